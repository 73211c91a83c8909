// Internal structures shared by the libxk translation units (CUDA path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/xk.h"

namespace xk {

// number of kernels this library has launched (all contexts), for reporting
void count_launches(long long n);
long long launches();

constexpr double kBoltz = 1.380649e-16;       // erg / K
constexpr double kAmu = 1.66053906660e-24;    // g
constexpr double kP0 = 1.0e6;                 // 1 bar in dyn / cm^2
constexpr double kBarToCgs = 1.0e6;

// Device-side view of one column: network, photolysis and atmosphere inputs,
// derived grid/transport arrays, per-step buffers.  All pointers are device
// pointers inside the caller-provided workspace.
struct Col {
    int S, E, R, L, W, Rph, Sabs;
    int ld;               // leading dimension of a dense S x S block (elements)
    // network
    const int *elem;      // [S][E] element counts
    const double *mass, *nasa, *dcoef, *arr, *troe;
    const int *rtype, *reac, *prod, *form, *prow;
    // species-major stoichiometry (residual gather): entries r * 16 + (nu + 8)
    const int *yp, *yent;
    // Jacobian pattern by row and column: row i's distinct columns jcol[jp[i] .. jp[i+1]), the terms of
    // column entry q in jrs[jtp[q] .. jtp[q+1]) as (reaction * 8 + slot) << 1 | (1: +d, 0: -d); jdq[i]
    // the diagonal entry of row i (-1: none)
    const int *jp, *jcol, *jtp, *jrs, *jdq;
    // photolysis
    const double *J0, *dlam, *sigma, *sig_abs;   // sig_abs: Sabs x W
    const int *abs_sp;
    double mu, tf;
    // Rayleigh scattering (Sec. 2.3.3): cross sections of the Ssca scattering species sca_sp,
    // Ssca x W; the diffuse field (diffuse = 1) with lower-boundary albedo; alpha_s [L][W] the
    // scattering coefficient; rt [4][L][W] the two-stream recursion's coefficients
    int Ssca, diffuse;
    // photolysis rates in the Jacobian (cfg.photo_jacobian): extinction along the J v direction
    // [L][W], the beam's change [L][W] and the rates' change [L][Rph]
    int photo_jac;
    double *pbeta, *pdJ, *pdk;
    const double *sig_sca;
    const int *sca_sp;
    double albedo;
    double *alpha_s, *rt;
    // atmosphere
    const double *P, *T, *Kzz;
    double g, mbar, alpha_T;
    // derived on the device
    double *ngas, *z, *dz, *dzi, *u, *v;
    // transport terms of row (k, y) of I/dt - dF/dn, per atmosphere: diagonal (u_k + v_{k-1}) / dz_k,
    // couplings -u_{k-1} / dz_k (to layer k-1) and -v_k / dz_k (to layer k+1); [L][S]
    double *tdg, *tlo, *tup;
    double *rs;           // [L][S] 1 / s of the current step's scaling
    // per step
    double *grt, *lnkc, *kf, *kr, *kph, *alpha, *Jw, *w, *d;
    double *dw;           // [L][R] directional derivative of each rate along a vector (J v)
    const double *fshift; // [L][S] subtracted from the residual when set (the BDF step's history terms)
    double *n, *F, *s, *b, *x, *delta, *tmp;
};

// Device control block: step-size state, decisions and counters.
struct Ctl {
    double dt, t, max_rel, dt_next, last_dt;
    unsigned long long max_rel_bits;
    int bad;              // non-finite or too negative
    int n_neg;
    int accepted, converged, status, finished;
    int steps, n_acc, n_rej;
    int solver_iters;
    double solver_resid;
    long long total_iters;
    int err_timeout;      // a bounded wait gave up
    unsigned long long wait_polls;   // polls before a bounded wait gives up (0: the default, about a second)
    int err_singular;     // zero pivot met
    // mixed precision routing: skip32 = this step goes straight to FP64; skip64 = FP64 solve not needed
    int skip32, skip64;
    int skip_reuse;       // 0: this step tries FGMRES preconditioned by the last FP64 factorization
    int have64;           // the FP64 factors in the workspace are valid
    int reuse_enabled;
    int used_fp64;        // this step was solved by the FP64 factorization
    long long refactors;  // FP64 factorizations made
    long long fp64_steps;
    double dt_fp64;       // smallest dt at which the FP32-preconditioned solve did not converge
};

struct Policy {
    double dt_max, rel_reject, rel_target, grow_max, shrink_min, neg_tol, f_floor, dt_min, ss_dt, ss_tol;
};

// Mass-action terms of reaction r in layer k at densities nk (Sec. 2.3): w = k_f prod n_reac -
// k_r prod n_prod, and d[slot] = d(k_f prod n_reac)/d n_reac[slot] (slots 0-2),
// -d(k_r prod n_prod)/d n_prod[slot] (slots 3-5).  Photolysis rows take k_f from kph, no reverse.
__device__ __forceinline__ void reaction_terms_at(const Col &c, int k, int r, const double *nk, double *w, double *d)
{
    const long long idx = (long long)k * c.R + r;
    double kfv, krv;
    if (c.rtype[r] == XK_RX_PHOTO) {
        kfv = c.kph[(long long)k * c.Rph + c.prow[r]];
        krv = 0.0;
    } else {
        kfv = c.kf[idx];
        krv = c.kr[idx];
    }
    int ra[3], pa[3];
    double na[3], pb[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        ra[s] = c.reac[3 * r + s];
        pa[s] = c.prod[3 * r + s];
        na[s] = ra[s] >= 0 ? nk[ra[s]] : 0.0;
        pb[s] = pa[s] >= 0 ? nk[pa[s]] : 0.0;
    }
    double wf = kfv, wb = krv;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (ra[s] >= 0) wf *= na[s];
        if (pa[s] >= 0) wb *= pb[s];
    }
    *w = wf - wb;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        double df = 0.0, db = 0.0;
        if (ra[s] >= 0) {
            df = kfv;
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (t != s && ra[t] >= 0) df *= na[t];
        }
        if (pa[s] >= 0) {
            db = -krv;
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (t != s && pa[t] >= 0) db *= pb[t];
        }
        d[s] = df;
        d[3 + s] = db;
    }
}

// Entry q of the Jacobian pattern (row-grouped): sum of its terms, -dF_i/dn_j of one layer, in a
// fixed order (dk: that layer's reaction derivatives [R][6]).
__device__ __forceinline__ double jac_entry(const Col &c, int q, const double *dk)
{
    double acc = 0.0;
    for (int t = c.jtp[q]; t < c.jtp[q + 1]; ++t) {
        const int code = c.jrs[t];
        const int rs = code >> 1;
        const double dv = dk[(long long)(rs >> 3) * 6 + (rs & 7)];
        acc += (code & 1) ? dv : -dv;
    }
    return acc;
}

// Reaction graph of the pathway analyser (Sec. 4), the same in every layer: species u's out-edges
// are grouped by target, groups gp[u] .. gp[u+1); group g leads to species gv[g] through the edge
// codes gcode[gs[g] .. gs[g+1]) (2 r + direction, 0 forward, 1 reverse) in increasing order.
struct PathGraph {
    const int *gp, *gv, *gs, *gcode;
};
// Sparse element structure for the equilibrium solve, built on the host: species y holds elements
// se[sp[y] .. sp[y+1]) with counts sc[..]; entry t of the Newton system (eij[t] = i * 32 + j for the
// element pair i <= j, -1 - i for element i's own sums) is a sum over the species ey[ep[t] ..
// ep[t+1]) (increasing) with coefficients ec[..] (a_iy a_jy, or a_iy).
struct EqIndex {
    const int *sp, *se, *ep, *ey, *eij;
    const double *sc, *ec;
    int nent;
};
// Equilibrium composition per layer (xk_analysis.cu): element totals b [L][E] (nullptr: from the
// state c.n); mole fractions into x [L][S] (may be nullptr) and, when nout is set, number densities
// x n_gas into nout; per layer the iterations taken and a status (0 converged, 1 not converged,
// -1 singular system).  Needs c.grt of the current atmosphere.
cudaError_t launch_equilibrium(const Col &c, const EqIndex &ix, const double *b, double *x, double *nout,
                               int max_iter, double tol, int *iters, int *status, cudaStream_t st);
// Forward and reverse rate of every reaction in every layer at state n: q [L][R][2].
void launch_fluxes(const Col &c, const double *n, double *q, cudaStream_t st);
// Dijkstra from each source src[j] (device, nsrc) in every layer of rates q [L][R][2]: outputs
// [nsrc][L][S] (any output pointer may be nullptr).  wbuf: L * R * 2 doubles of scratch for the edge
// weights 1/q.
cudaError_t launch_pathways(const Col &c, const PathGraph &g, const double *q, double *wbuf, int nsrc,
                            const int *src, double *dist, int *pred_sp, int *pred_edge, int *lim_edge,
                            double *lim_w, cudaStream_t st);

// Variable-order BDF (xk_bdf.cu): the history's linear combinations for one step attempt.
constexpr int kBdfHist = 7;      // states kept: order 5 plus the two needed by the order-6 predictor
struct BdfCombo {
    int m;                       // terms
    int slot[kBdfHist];          // history buffer of each term
    double w[kBdfHist];
};
struct BdfStepArgs {
    BdfCombo pred;               // predictor y_hat at t + h
    BdfCombo hist;               // sum_{j>=1} c_j y_j of the corrector
    double c0;
    BdfCombo lo, hi;             // predictors of one degree lower / higher (m = 0: not needed)
    double K, Klo, Khi;          // error constants q + 1, q, q + 2
    double rtol, neg_tol, f_floor;
    int newest;                  // buffer of y_n
};
struct BdfResult {
    unsigned long long err, err_lo, err_hi, relc;   // bit patterns of non-negative maxima
    int bad;
};
// y_hat and g = c0 y_hat + sum_{j>=1} c_j y_j (Y: kBdfHist buffers of L*S)
void launch_bdf_predict(long long N, const double *Y, const BdfStepArgs &a, double *yhat, double *g,
                        cudaStream_t st);
// y_new = y_hat + delta, its checks and error estimates into *res (cleared by the caller)
void launch_bdf_check(const Col &c, const double *Y, const BdfStepArgs &a, const double *yhat, const double *delta,
                      double *ynew, BdfResult *res, cudaStream_t st);
// accepted: Y[slot] = max(y_new, 0) and the state n = the same
void launch_bdf_accept(long long N, const double *ynew, double *Yslot, double *n, cudaStream_t st);

// Lagrangian parcel scheme (Sec. 2, Fig. 2): buffers and state of one global iteration.
struct ParcelState {
    double h;              // trial step, carried from visit to visit and across iterations
    long long steps, rejected;
    int status;            // 0, XK_ESINGULAR, XK_ENEG (step below dt_min), XK_ENOCONV (visit step cap)
    int visit;             // visit at which a failure happened
    double max_change;     // largest |N_new - N_old| / N_new over entries above f_floor mixing ratio
};
struct ParcelArgs {
    double *N;             // [L][S] stored profile (the column state), updated in place
    double *Nold;          // [L][S] the profile at the start of the iteration
    const double *um, *vm; // [L-1][S] molecular part of Eq. 2's interface coefficients
    double *A;             // 2 x S x S: the current implicit step's matrix and its LU factors (row-major)
    double *vmr;           // [S] the parcel's carried mixing ratios
    double *w, *dd;        // [R] rates, [R][6] their derivatives at the parcel's densities
    Policy pol;
    int max_visit_steps;
    ParcelState *st;
};
// One global iteration on one CTA (photolysis and rate coefficients already in c).
cudaError_t launch_parcel_iteration(const Col &c, const ParcelArgs &a, cudaStream_t st);

constexpr unsigned long long kSpinLimit = 1ull << 24;   // polls of a bounded wait: ~1-2 s with the sleep below

// Barrier over the nblk CTAs that share the counter pair bar[0..1] (the whole grid by default).
// The wait is bounded: after ctl->wait_polls polls (default kSpinLimit) the CTA records
// ctl->err_timeout and every CTA leaves at its next barrier.  The decision is taken by thread 0
// and shared through shared memory, so all threads of a CTA return the same value.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, Ctl *ctl, unsigned nblk = 0)
{
    __shared__ int s_go;
    if (nblk == 0) nblk = gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *vto = &ctl->err_timeout;
        int go = *vto == 0;
        if (go) {
            const unsigned long long limit = ctl->wait_polls ? ctl->wait_polls : kSpinLimit;
            volatile unsigned *vgen = bar + 1;
            unsigned gen = *vgen;
            __threadfence();
            unsigned prev = atomicAdd(bar, 1u);
            if (prev == nblk - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                unsigned long long spins = 0;
                while (*vgen == gen) {
                    if (++spins > limit || *vto) {
                        atomicExch(&ctl->err_timeout, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            go = *vto == 0;
        }
        s_go = go;
    }
    __syncthreads();
    return s_go != 0;
}

// Launch helpers implemented in xk_chem.cu
void launch_grid(const Col &c, cudaStream_t st);
void launch_thermo(const Col &c, cudaStream_t st);
void launch_rates(const Col &c, cudaStream_t st);
// u, v of Eq. 2 for the eddy profile Kzz (a zero profile leaves the molecular part only)
void launch_transport_coeffs(const Col &c, const double *Kzz, double *u, double *v, cudaStream_t st);
void launch_photolysis(const Col &c, const double *n, cudaStream_t st);
void launch_reaction_terms(const Col &c, const double *n, cudaStream_t st);
void launch_residual(const Col &c, const double *n, double *F, const Ctl *ctl, double f_floor, cudaStream_t st);
void launch_jacobian64(const Col &c, const double *n, const Ctl *ctl, double dt_override, int scaled,
                       double *A, double *lo, double *up, cudaStream_t st, const int *skip = nullptr);
// lstride: elements between consecutive layers' blocks (0: S * ld)
void launch_jacobian32(const Col &c, const double *n, const Ctl *ctl, float *A, float *lo, float *up, double *diag,
                       cudaStream_t st, const int *skip = nullptr, long long lstride = 0);
void launch_route(Ctl *ctl, cudaStream_t st);
void launch_jv(const Col &c, const Ctl *ctl, const double *xs, double *ys, const double *rowdiv, const int *skip,
               cudaStream_t st);
void launch_rowdiv(long long N, const double *x, const double *d, double *y, cudaStream_t st);
void launch_diag(const Col &c, const Ctl *ctl, double *diag, cudaStream_t st);
void launch_reuse_scales(long long N, const double *rowd, const double *s, const double *s64, double *pin, double *pout,
                         const Ctl *ctl, cudaStream_t st);
void launch_after_refactor(long long N, const double *s, double *s64, Ctl *ctl, cudaStream_t st);
void launch_check(const Col &c, Ctl *ctl, const Policy &pol, cudaStream_t st);
void launch_decide(const Col &c, Ctl *ctl, const Policy &pol, cudaStream_t st);
void launch_apply(const Col &c, Ctl *ctl, cudaStream_t st);
void launch_unscale(const Col &c, const double *xs, double *delta, cudaStream_t st);
void launch_begin(Ctl *ctl, cudaStream_t st);
void launch_set_mixing(const Col &c, const double *f, double *n, cudaStream_t st);
void launch_convert32(const double *src, size_t lds, float *dst, size_t ldd, size_t rows, size_t cols, cudaStream_t st);

// Block-Thomas factorization and solve (xk_factor.cu)
struct FactorPlan {
    int nb;          // panel width
    int ctas;        // persistent CTAs
    int threads;
    size_t smem;
    int twisted = 0;           // k_factor: eliminate from both ends on the two halves of the grid
    int preview = 0;           // FP64: each panel's pivots chosen first on one CTA (k_factor_pv)
    double *dinv = nullptr;    // that path: nb x nb LU factors of the panel's pivot block (global)
};
template <typename T>
struct BlockSys {
    T *D;            // [L][S][ld] diagonal blocks, overwritten by their inverses (row-pivoted form)
    const T *lo, *up;
    int *perm;       // [L][S] pivot row of each column
    int *iperm;      // [L][S] column each row was pivot of
    int *pinfo;      // panel scratch: pivot rows of the current panel
    unsigned *bar;   // grid barrier: [2]
    int L, S, ld;
};
int factor_plan(int S, int precision_bytes, int nb_hint, int ctas_hint, FactorPlan *out);
template <typename T>
cudaError_t launch_factor(const BlockSys<T> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                          const int *skip = nullptr);
// FP32 block inversion without pivoting (mixed-path preconditioner); gbuf: 2 x S x nb floats
cudaError_t launch_factor_nopivot(const BlockSys<float> &sys, const FactorPlan &plan, float *gbuf, Ctl *ctl,
                                  cudaStream_t st, const int *skip = nullptr);
// FP32 block inversion without pivoting on one thread-block cluster, each layer's
// block resident in distributed shared memory (xk_cluster.cu)
struct ClusterPlan {
    int C;           // CTAs in the cluster
    int nb;          // panel width
    int threads;
    int nslot;       // panels held per CTA
    int lds;         // shared-memory row stride (floats)
    size_t smem;
    int twisted = 0; // two clusters fit at once: eliminate from both ends (layers >= 3)
};
bool cluster_twisted(const ClusterPlan &plan, int L);
int cluster_plan(int S, int nb, int C, ClusterPlan *out);
// gU: cluster_ubuf_floats(plan) floats of global memory (the panel rows every CTA reads, two
// slots per cluster)
size_t cluster_ubuf_floats(const ClusterPlan &plan);
cudaError_t launch_factor_cluster(const BlockSys<float> &sys, const ClusterPlan &plan, float *gU, Ctl *ctl,
                                  cudaStream_t st, const int *skip = nullptr);
// sweeps with stored inverses on one cluster (xk_cluster.cu): FP32 inverses of the
// cluster factorization (identity pivots) or FP64 inverses with implicit pivoting
struct SolvePlan {
    int C;           // CTAs in the cluster
    int rpc;         // rows per CTA
    int lds;         // shared-memory row stride (elements)
    int nbuf;        // prefetch buffers (2, or 1 when two do not fit)
    int threads;
    size_t smem;
    int twisted = 0; // two clusters fit at once (sweeps after the twisted elimination)
};
int solve_cluster_plan(int S, int elem_bytes, SolvePlan *out);
// sweeps after the twisted elimination (two launches of two clusters); ymid: 2 x S doubles
template <typename T>
cudaError_t launch_solve_twisted(const BlockSys<T> &sys, const SolvePlan &plan, bool pivoted, const double *b,
                                 double *x, double *g, double *ymid, Ctl *ctl, cudaStream_t st,
                                 const double *bscale = nullptr, const int *skip = nullptr,
                                 const double *xscale = nullptr);
template <typename T>
cudaError_t launch_solve_cluster(const BlockSys<T> &sys, const SolvePlan &plan, bool pivoted, const double *b,
                                 double *x, double *g, Ctl *ctl, cudaStream_t st, const double *bscale = nullptr,
                                 const int *skip = nullptr, const double *xscale = nullptr);
template <typename T>
cudaError_t launch_solve(const BlockSys<T> &sys, const FactorPlan &plan, const double *b, double *x,
                         double *g, Ctl *ctl, cudaStream_t st, const double *bscale = nullptr,
                         const int *skip = nullptr, const double *xscale = nullptr);
size_t barrier_words();

}  // namespace xk
