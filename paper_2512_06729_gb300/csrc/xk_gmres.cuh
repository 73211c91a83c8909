// Device state and host driver of the FP64 flexible GMRES used by the
// mixed-precision linear solve.
#pragma once

#include <functional>

#include "xk_internal.cuh"

namespace xk {

constexpr int kMaxBasis = 32;

struct GmState {
    double H[(kMaxBasis + 1) * kMaxBasis];   // column-major, leading dimension kMaxBasis + 1
    double g[kMaxBasis + 1];
    double cs[kMaxBasis], sn[kMaxBasis];
    double beta, bnorm, resid, tol, hnext;
    int j, iters, done, cycle_end, applied, failed;
    int idle;            // done || cycle_end: kernels of the remaining iterations return at once
};

using VecOp = std::function<void(const double *, double *, const int *skip, cudaStream_t)>;

struct GmArgs {
    long long N;
    int m, max_iter;
    double tol;
    const double *b;     // right-hand side (scaled)
    double *x;           // solution (scaled)
    double *V;           // (m + 1) x N basis
    double *Z;           // m x N preconditioned basis
    double *w;           // N work vector
    double *h1, *h2;     // kMaxBasis + 1 coefficients each
    double *red;         // reduction output
    double *partials;    // blocks x (kMaxBasis + 1)
    unsigned *counter;   // last-block counter (zero on entry)
    GmState *gm;
    Ctl *ctl;
    const int *skip_solve;   // this solve is skipped when *skip_solve != 0
    int role;                // 0: FP32-preconditioned attempt, 1: attempt with the reused FP64 factorization,
                             // 2: refinement around a fresh FP64 factorization (recorded, no routing)
    int reuse_max_iters;     // role 1: more iterations than this trigger a fresh factorization next step
    VecOp matvec;        // y = A x (FP64); must return at once while *skip != 0
    VecOp precond;       // z ~ A^-1 v (low precision); same skip rule
};

constexpr int kGmPartialBlocks = 304;

void enqueue_fgmres(const GmArgs &a, cudaStream_t st);

}  // namespace xk
