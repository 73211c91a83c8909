// Block cyclic reduction of the block-tridiagonal system on the tensor cores:
// the mixed path's FP32 factorization and its solve.
#pragma once

#include <vector>

#include "xk_tc.cuh"

namespace xk {

constexpr int kBcrLeafMax = 160;   // largest block inverted directly by one CTA

// One block inverted by Gauss-Jordan with partial pivoting in one CTA (n <= kBcrLeafMax).
struct BcrLeaf {
    const float *in;
    float *out;
    int ldin, ldout, n;
};

// y = base + sign * M v for the rows [0, Sp) of one block: M is Sp x K row-major (ld), v is
// [v0; v1] (K = Sp or 2 Sp), optionally v0 - d0 w0 - d1 w1 on the first S entries (level 0).
struct BcrMv {
    const float *M;
    const float *v0, *v1, *d0, *w0, *d1, *w1, *base;
    float *y;
    int ld, K;
    float sign;
};

struct BcrStage {
    int kind;          // BcrKind
    int off, count;    // range in the task list of that kind
    int tiles;         // GEMM: output tiles of the launch
    int level;         // the reduction level it belongs to
};
enum BcrKind { kBcrLeafStage = 0, kBcrGemm = 1, kBcrLevel0 = 2, kBcrMv = 3, kBcrFwd0 = 4, kBcrIn = 5, kBcrOut = 6 };

// The plan of one column's factorization and solve.  Built on the host once per workspace; the
// task lists live in the workspace.
struct BcrPlan {
    int L = 0, S = 0, Sp = 0, Wt = 0, Zt = 0, Ncp = 0, levels = 0;
    // arrays: D (the FP32 blocks, padded to Sp x Sp per layer), INV (inverses), TMP (inversion
    // temporaries), CP (dense couplings [L | U] of the levels >= 1), PQ (D^-1 [L | U])
    float *D = nullptr, *INV = nullptr, *TMP = nullptr, *CP = nullptr, *PQ = nullptr;
    float *bw = nullptr, *tw = nullptr, *xw = nullptr;      // [L][Sp] vectors of the solve
    const float *lo = nullptr, *up = nullptr;                // level-0 couplings [L][S] (FP32)
    std::vector<TcTask> gemm;
    std::vector<BcrLeaf> leaf;
    std::vector<BcrMv> mv;
    std::vector<BcrStage> fac, sol;
    std::vector<int> level0_kept;                            // even layers kept at level 0
    TcTask *gemm_d = nullptr;
    BcrLeaf *leaf_d = nullptr;
    BcrMv *mv_d = nullptr;
    CUtensorMap *maps_d = nullptr;
    std::vector<CUtensorMap> maps;
    int *l0_d = nullptr;
    BcrStage *sol_d = nullptr;     // the solve's stages, walked by one persistent kernel
    unsigned *bar = nullptr;       // its grid-barrier words (2, zero between calls)
    int solve_ctas = 0;            // CTAs of that kernel (0: as many as fit on the GPU)
};

// Sizes of the device arrays and task lists of an L-layer, S-species column (no pointers).
struct BcrSizes {
    int Sp, Wt, Zt, Ncp, ngemm, nleaf, nmv, nsol;
    size_t floats_D, floats_INV, floats_TMP, floats_CP, floats_PQ, floats_vec;
};
BcrSizes bcr_sizes(int L, int S);
// Fill the plan for arrays already laid out (p.D ... p.xw, p.lo, p.up, and the task storage
// pointers set); uploads task lists and tensor maps on st.  0 or -1.
int bcr_build(BcrPlan &p, int L, int S, cudaStream_t st);
// Pad rows of D to the identity (once per workspace).
void bcr_init_pad(const BcrPlan &p, cudaStream_t st);
// Optional marks around the factorization's launches (tracing).
struct BcrTimer {
    virtual void begin(int kind) = 0;
    virtual void end(int kind) = 0;
    virtual ~BcrTimer() = default;
};
// Factorization: every level's inversions and Schur updates (D is overwritten).
cudaError_t bcr_factor(const BcrPlan &p, const int *skip, Ctl *ctl, cudaStream_t st, BcrTimer *timer = nullptr);
// Flops of one factorization: 2 m n k over the products, 2 n^3 over the leaves.
void bcr_work(const BcrPlan &p, double *mma_flops, double *leaf_flops);
// x = M^-1 (b * bscale) (* xscale) with the factorization, FP64 in and out.
cudaError_t bcr_solve(const BcrPlan &p, const double *b, double *x, const double *bscale, const double *xscale,
                      const int *skip, Ctl *ctl, cudaStream_t st);

}  // namespace xk
