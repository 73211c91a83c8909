// Flexible GMRES(m) in FP64 on the scaled system diag(1/s) (I/dt - J) diag(s) x = F / s,
// right-preconditioned by the FP32 block-Thomas inverse (mixed-precision
// iterative refinement in its Krylov form: the low-precision factorization
// handles the fast chemistry, the FP64 Krylov iteration on the exact FP64
// operator recovers the slow and conserved directions that FP32 cannot
// resolve).  Every kernel checks the device flags and returns at once when
// the solve has converged, so all iterations can be enqueued (or captured)
// without a host round trip.
#include <math.h>

#include "xk_gmres.cuh"

namespace xk {

namespace {

constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic multi-dot h[i] = <V_i, w>, i < nv (nv <= kMaxBasis), optionally
// also ||w||^2 into h[nv].  Partial sums per block; the last block to finish
// adds them in block order.
__global__ void k_dots(const double *V, int nv, const double *w, long long N, double *partials,
                       unsigned *counter, double *out, const GmState *gm, int with_norm)
{
    if (gm->done || gm->cycle_end) return;
    __shared__ double sacc[kRedThreads / 32][kMaxBasis + 1];
    __shared__ bool last;
    int nout = nv + (with_norm ? 1 : 0);
    double acc[kMaxBasis + 1];
#pragma unroll
    for (int i = 0; i <= kMaxBasis; ++i) acc[i] = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double wn = w[n];
#pragma unroll
        for (int i = 0; i < kMaxBasis; ++i)
            if (i < nv) acc[i] += V[(long long)i * N + n] * wn;
        if (with_norm) acc[kMaxBasis] += wn * wn;
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i <= kMaxBasis; ++i) {
        double v = warp_sum(acc[i]);
        if (lane == 0) sacc[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < nout) {
        int i = threadIdx.x < nv ? threadIdx.x : kMaxBasis;
        double s = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) s += sacc[q][i];
        partials[(long long)blockIdx.x * (kMaxBasis + 1) + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < nout) {
            double s = 0.0;
            for (int b = 0; b < gridDim.x; ++b) s += partials[(long long)b * (kMaxBasis + 1) + threadIdx.x];
            out[threadIdx.x] = s;
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// w -= sum_i h[i] V_i
__global__ void k_axpy_basis(const double *V, int nv, const double *h, double *w, long long N, const GmState *gm)
{
    if (gm->done || gm->cycle_end) return;
    __shared__ double sh[kMaxBasis];
    if (threadIdx.x < nv) sh[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double acc = w[n];
        for (int i = 0; i < nv; ++i) acc -= sh[i] * V[(long long)i * N + n];
        w[n] = acc;
    }
}

// v = w / nrm
__global__ void k_scale(const double *w, double *v, long long N, const double *nrm, const GmState *gm)
{
    if (gm->done || gm->cycle_end) return;
    double inv = 1.0 / *nrm;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        v[n] = w[n] * inv;
}

// r = b - y (restart residual); y holds A x
__global__ void k_sub(const double *b, const double *y, double *r, long long N, const GmState *gm)
{
    if (gm->done) return;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        r[n] = b[n] - y[n];
}

// Start of a cycle: beta = ||r|| of the true residual r = b - A x (computed
// into red[0]); V_0 = r / beta; g = beta e_1.  Convergence is decided here, on
// the true residual, never on the Givens recurrence alone.
__global__ void k_cycle_begin(GmState *gm, const double *red, int first, int max_iter)
{
    if (gm->done) return;
    double beta = sqrt(red[0]);
    if (first) gm->bnorm = beta;
    gm->beta = beta;
    gm->j = 0;
    gm->cycle_end = 0;
    gm->idle = 0;
    for (int i = 0; i <= kMaxBasis; ++i) gm->g[i] = 0.0;
    gm->g[0] = beta;
    double rel = (gm->bnorm > 0.0) ? beta / gm->bnorm : 0.0;
    gm->resid = rel;
    if (!(beta > 0.0) || rel <= gm->tol || !isfinite(beta) || gm->iters >= max_iter) {
        gm->done = 1;
        gm->cycle_end = 1;
        gm->idle = 1;
        if (!isfinite(beta)) gm->failed = 1;
    }
}

// After the two Gram-Schmidt passes: combine the coefficients, normalize, apply
// Givens rotations and test convergence.
__global__ void k_arnoldi_end(GmState *gm, const double *h1, const double *h2, int jj, int m, int max_iter)
{
    if (gm->done || gm->cycle_end) return;
    double *H = gm->H + (long long)jj * (kMaxBasis + 1);       // column jj
    for (int i = 0; i <= jj; ++i) H[i] = h1[i] + h2[i];
    double hn = sqrt(h2[jj + 1]);                               // ||w|| after the second pass
    H[jj + 1] = hn;
    gm->hnext = hn;
    for (int i = 0; i < jj; ++i) {
        double a = gm->cs[i] * H[i] + gm->sn[i] * H[i + 1];
        double b = -gm->sn[i] * H[i] + gm->cs[i] * H[i + 1];
        H[i] = a;
        H[i + 1] = b;
    }
    double a = H[jj], b = H[jj + 1];
    double r = hypot(a, b);
    double c = (r > 0.0) ? a / r : 1.0, s = (r > 0.0) ? b / r : 0.0;
    gm->cs[jj] = c;
    gm->sn[jj] = s;
    H[jj] = r;
    H[jj + 1] = 0.0;
    gm->g[jj + 1] = -s * gm->g[jj];
    gm->g[jj] = c * gm->g[jj];
    gm->iters += 1;
    gm->j = jj + 1;
    gm->resid = fabs(gm->g[jj + 1]) / gm->bnorm;
    if (!isfinite(gm->resid)) {
        gm->cycle_end = 1;
        gm->done = 1;
        gm->failed = 1;
        gm->idle = 1;
        return;
    }
    if (gm->resid <= gm->tol || gm->iters >= max_iter || jj + 1 >= m || !(hn > 0.0)) {
        gm->cycle_end = 1;
        gm->idle = 1;
    }
}

// x += Z y with H(0:j, 0:j) y = g(0:j); solved by the first thread of every block.
__global__ void k_update(GmState *gm, const double *Z, double *x, long long N, int max_iter)
{
    if (gm->done && !gm->cycle_end) return;
    if (gm->applied) return;
    __shared__ double y[kMaxBasis];
    int j = gm->j;
    if (threadIdx.x == 0) {
        for (int i = j - 1; i >= 0; --i) {
            double s = gm->g[i];
            for (int q = i + 1; q < j; ++q) s -= gm->H[(long long)q * (kMaxBasis + 1) + i] * y[q];
            y[i] = s / gm->H[(long long)i * (kMaxBasis + 1) + i];
        }
    }
    __syncthreads();
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double acc = x[n];
        for (int i = 0; i < j; ++i) acc += y[i] * Z[(long long)i * N + n];
        x[n] = acc;
    }
    (void)max_iter;
}

__global__ void k_update_done(GmState *gm, int max_iter)
{
    if (gm->applied) return;
    (void)max_iter;
    if (gm->failed) gm->done = 1;        // otherwise the next cycle start checks the true residual
    gm->cycle_end = 0;
    gm->idle = gm->done;
    if (gm->done) gm->applied = 1;
}

// Record the true relative residual of a solve that ended without a checked convergence.
__global__ void k_final(GmState *gm, const double *red)
{
    if (gm->done) return;
    gm->resid = (gm->bnorm > 0.0) ? sqrt(red[0]) / gm->bnorm : 0.0;
    gm->done = 1;
    gm->idle = 1;
}

__global__ void k_gm_init(GmState *gm, double tol)
{
    gm->done = 0;
    gm->cycle_end = 0;
    gm->applied = 0;
    gm->failed = 0;
    gm->iters = 0;
    gm->idle = 0;
    gm->j = 0;
    gm->tol = tol;
    gm->resid = 0.0;
    gm->bnorm = 0.0;
}

__global__ void k_zero(double *x, long long N, const GmState *gm)
{
    if (gm->done) return;               // a skipped solve leaves x to the solve that ran
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        x[n] = 0.0;
}

__global__ void k_gm_skip_if_finished(GmState *gm, const Ctl *ctl, const int *skip_solve)
{
    if (ctl->finished || (skip_solve && *skip_solve)) { gm->done = 1; gm->applied = 1; gm->idle = 1; }
}

// Record the solve; a solve that did not reach the tolerance hands the step to
// the FP64 factorization, and so does every later step at this dt or above.
// Refinement around a fresh FP64 factorization (role 2) is only recorded.
__global__ void k_gm_report(const GmState *gm, Ctl *ctl, const int *skip_solve, int role, int reuse_max_iters)
{
    if (ctl->finished || (skip_solve && *skip_solve)) return;
    ctl->solver_iters = gm->iters;
    ctl->solver_resid = gm->resid;
    ctl->total_iters += gm->iters;
    if (role == 2) return;             // refinement of a fresh FP64 factorization: the best FP64 can do
    if (gm->failed || !(gm->resid <= gm->tol)) {
        ctl->skip64 = 0;               // refactor in FP64 and solve directly
        ctl->used_fp64 = 1;
        if (role == 0 && ctl->dt < ctl->dt_fp64) ctl->dt_fp64 = ctl->dt;
    } else if (role == 1 && gm->iters > reuse_max_iters) {
        ctl->have64 = 0;               // the reused factorization has drifted: refactor at the next step
    }
}

}  // namespace

void enqueue_fgmres(const GmArgs &a, cudaStream_t st)
{
    const long long N = a.N;
    const int m = a.m < kMaxBasis ? a.m : kMaxBasis;
    // iteration slots: the budget max_iter split into cycles of m, then a short spare cycle for a
    // restart after a cycle that ended on the recurrence estimate without true convergence;
    // slots past convergence cost one early-exit launch per kernel
    const int full = (a.max_iter + m - 1) / m;
    const int spare = m < 8 ? m : 8;
    const int cycles = full + 1;
    int eb = (int)((N + kRedThreads - 1) / kRedThreads);
    if (eb > 4 * kRedBlocks) eb = 4 * kRedBlocks;
    count_launches(1); k_gm_init<<<1, 1, 0, st>>>(a.gm, a.tol);
    count_launches(1); k_gm_skip_if_finished<<<1, 1, 0, st>>>(a.gm, a.ctl, a.skip_solve);
    count_launches(1); k_zero<<<eb, kRedThreads, 0, st>>>(a.x, N, a.gm);
    for (int cyc = 0; cyc < cycles; ++cyc) {
        double *r = a.V;                       // V_0 slot holds the residual before scaling
        if (cyc == 0) {
            count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, 0, a.b, N, a.partials, a.counter, a.red, a.gm, 1);
            // red[0] = ||b||^2 (nv = 0: the norm lands in out[0])
            count_launches(1); k_cycle_begin<<<1, 1, 0, st>>>(a.gm, a.red, 1, a.max_iter);
            count_launches(1); k_scale<<<eb, kRedThreads, 0, st>>>(a.b, a.V, N, &a.gm->beta, a.gm);
        } else {
            a.matvec(a.x, a.w, &a.gm->done, st);
            count_launches(1); k_sub<<<eb, kRedThreads, 0, st>>>(a.b, a.w, r, N, a.gm);
            count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, 0, r, N, a.partials, a.counter, a.red, a.gm, 1);
            count_launches(1); k_cycle_begin<<<1, 1, 0, st>>>(a.gm, a.red, 0, a.max_iter);
            count_launches(1); k_scale<<<eb, kRedThreads, 0, st>>>(r, a.V, N, &a.gm->beta, a.gm);
        }
        const int mc = cyc < full ? (a.max_iter - cyc * m < m ? a.max_iter - cyc * m : m) : spare;
        for (int jj = 0; jj < mc; ++jj) {
            double *vj = a.V + (long long)jj * N;
            double *zj = a.Z + (long long)jj * N;
            a.precond(vj, zj, &a.gm->idle, st);
            a.matvec(zj, a.w, &a.gm->idle, st);
            count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, jj + 1, a.w, N, a.partials, a.counter, a.h1, a.gm, 0);
            count_launches(1); k_axpy_basis<<<eb, kRedThreads, 0, st>>>(a.V, jj + 1, a.h1, a.w, N, a.gm);
            count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, jj + 1, a.w, N, a.partials, a.counter, a.h2, a.gm, 0);
            count_launches(1); k_axpy_basis<<<eb, kRedThreads, 0, st>>>(a.V, jj + 1, a.h2, a.w, N, a.gm);
            // ||w||^2 into h2[jj + 1]
            count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, 0, a.w, N, a.partials, a.counter, a.h2 + jj + 1, a.gm, 1);
            count_launches(1); k_arnoldi_end<<<1, 1, 0, st>>>(a.gm, a.h1, a.h2, jj, mc, a.max_iter);
            count_launches(1); k_scale<<<eb, kRedThreads, 0, st>>>(a.w, a.V + (long long)(jj + 1) * N, N, &a.gm->hnext, a.gm);
        }
        count_launches(1); k_update<<<eb, kRedThreads, 0, st>>>(a.gm, a.Z, a.x, N, a.max_iter);
        count_launches(1); k_update_done<<<1, 1, 0, st>>>(a.gm, a.max_iter);
    }
    // final check on the true residual (a cycle may have ended on the recurrence estimate)
    a.matvec(a.x, a.w, &a.gm->done, st);
    count_launches(1); k_sub<<<eb, kRedThreads, 0, st>>>(a.b, a.w, a.w, N, a.gm);
    count_launches(1); k_dots<<<kRedBlocks, kRedThreads, 0, st>>>(a.V, 0, a.w, N, a.partials, a.counter, a.red, a.gm, 1);
    count_launches(1); k_final<<<1, 1, 0, st>>>(a.gm, a.red);
    count_launches(1); k_gm_report<<<1, 1, 0, st>>>(a.gm, a.ctl, a.skip_solve, a.role, a.reuse_max_iters);
}

}  // namespace xk
