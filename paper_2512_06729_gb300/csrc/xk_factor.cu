// Block-tridiagonal solve by block Thomas elimination with explicit block
// inverses.  For layer k the Schur complement D'_k = A_k - diag(lo_k)
// D'^-1_{k-1} diag(up_{k-1}) is formed and inverted in place by blocked
// Gauss-Jordan elimination with partial (row) pivoting.  One persistent,
// cooperatively launched kernel runs all layers; phases are separated by a
// grid barrier whose waits are bounded (on timeout the kernel records the
// error in the control block and returns).
//
// Storage after factorization: D holds B_k = (P_k D'_k)^-1, where P_k is the
// row permutation chosen by pivoting; ridx_k[i] is the original row now at
// position i, so D'^-1_k g = B_k (g[ridx_k]) and D'^-1_k[:, j] = B_k[:, sig_k(j)]
// with sig_k the inverse of ridx_k.
#include <cooperative_groups.h>
#include <math.h>

#include "xk_internal.cuh"

namespace xk {

namespace {

constexpr int kFactorThreads = 512;
constexpr int kSolveThreads = 512;
constexpr unsigned long long kSpinLimit = 1ull << 24;   // ~1-2 s with the sleep below

__device__ __forceinline__ bool grid_barrier(unsigned *bar, Ctl *ctl)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == gen) {
                if (++spins > kSpinLimit) {
                    atomicExch(&ctl->err_timeout, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)&ctl->err_timeout == 0;
}

// max |value| with the lowest row index on ties, over a block
__device__ __forceinline__ void argmax_combine(double &v, int &i, double ov, int oi)
{
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
}

// Gauss-Jordan on the panel columns [c0, c0 + nb) of D (all S rows), by one CTA.
template <typename T, int NB>
__device__ void panel_factor(T *D, int *ridx, int *pinfo, int S, int ld, int c0, int nb, Ctl *ctl,
                             unsigned char *smem)
{
    constexpr int PS = NB + 1;                 // padded row stride (no bank conflicts)
    T *P = (T *)smem;
    int *src = (int *)(P + (size_t)S * PS);
    int *tmp = src + S;
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ int s_piv, s_cnt;
    const int tid = threadIdx.x, nthr = blockDim.x;

    for (int e = tid; e < S * nb; e += nthr) {
        int r = e / nb, j = e - r * nb;
        P[r * PS + j] = D[(size_t)r * ld + c0 + j];
    }
    for (int r = tid; r < S; r += nthr) src[r] = r;
    __syncthreads();

    for (int lc = 0; lc < nb; ++lc) {
        const int c = c0 + lc;
        double best = -1.0;
        int bi = S;
        for (int r = c + tid; r < S; r += nthr) {
            double v = fabs((double)P[r * PS + lc]);
            argmax_combine(best, bi, v, r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_combine(best, bi, ov, oi);
        }
        if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid < 32) {
            int nw = nthr >> 5;
            double v = tid < nw ? red_v[tid] : -1.0;
            int i = tid < nw ? red_i[tid] : S;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, i, o);
                argmax_combine(v, i, ov, oi);
            }
            if (tid == 0) {
                if (!(v > 0.0) || i >= S) {       // zero (or NaN) column: singular block
                    atomicExch(&ctl->err_singular, 1);
                    i = c;
                }
                s_piv = i;
            }
        }
        __syncthreads();
        const int piv = s_piv;
        if (piv != c) {
            for (int j = tid; j < nb; j += nthr) {
                T t = P[c * PS + j];
                P[c * PS + j] = P[piv * PS + j];
                P[piv * PS + j] = t;
            }
            if (tid == 0) { int t = src[c]; src[c] = src[piv]; src[piv] = t; }
        }
        __syncthreads();
        const T dinv = (T)1 / P[c * PS + lc];
        __syncthreads();
        for (int j = tid; j < nb; j += nthr)
            P[c * PS + j] = (j == lc) ? dinv : P[c * PS + j] * dinv;
        __syncthreads();
        for (int r = tid; r < S; r += nthr) {
            if (r == c) continue;
            T f = P[r * PS + lc];
            if (f != (T)0) {
#pragma unroll 8
                for (int j = 0; j < nb; ++j)
                    if (j != lc) P[r * PS + j] -= f * P[c * PS + j];
                P[r * PS + lc] = -f * dinv;
            }
        }
        __syncthreads();
    }

    for (int e = tid; e < S * nb; e += nthr) {
        int r = e / nb, j = e - r * nb;
        D[(size_t)r * ld + c0 + j] = P[r * PS + j];
    }
    // pinfo: [0] displaced count, [1..nb] source rows of panel positions,
    // [1+nb ..] pairs (row, source) of rows outside the panel that moved
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int lc = tid; lc < nb; lc += nthr) pinfo[1 + lc] = src[c0 + lc];
    for (int r = tid; r < S; r += nthr) {
        if ((r < c0 || r >= c0 + nb) && src[r] != r) {
            int slot = atomicAdd(&s_cnt, 1);
            pinfo[1 + nb + 2 * slot] = r;
            pinfo[2 + nb + 2 * slot] = src[r];
        }
    }
    // ridx follows the same row moves
    for (int r = tid; r < S; r += nthr) tmp[r] = ridx[src[r]];
    __syncthreads();
    for (int r = tid; r < S; r += nthr) ridx[r] = tmp[r];
    if (tid == 0) pinfo[0] = s_cnt;
    __threadfence();
}

// Apply the panel's row moves and eliminations to the other columns:
// rows outside the panel: D[r][j] += sum_l G[r][l] U[l][j]; panel rows: D[r][j] = sum_l G[r][l] U[l][j],
// with U the (moved) panel rows and G the panel columns.
template <typename T, int NB>
__device__ void trailing_update(T *D, const int *pinfo, int S, int ld, int c0, int nb, unsigned char *smem)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int others = S - nb;
    const int cw = (others + gridDim.x - 1) / gridDim.x;
    const int q0 = blockIdx.x * cw;
    const int q1 = min(others, q0 + cw);
    const int ncols = q1 - q0;
    if (ncols <= 0) return;
    T *G = (T *)smem;                                  // S x NB
    T *U = G + (size_t)S * NB;                         // NB x cw
    T *DV = U + (size_t)NB * cw;                       // NB x cw (displaced rows' old values)
    int *meta = (int *)(DV + (size_t)NB * cw);         // [0..nb) sources, then pairs
    int *dmap = meta + 1 + 3 * NB;                     // S: index into DV or -1
    const int ndisp = pinfo[0];
    for (int e = tid; e < 1 + nb + 2 * ndisp; e += nthr) meta[e] = pinfo[e];
    for (int r = tid; r < S; r += nthr) dmap[r] = -1;
    for (int e = tid; e < S * nb; e += nthr) {
        int r = e / nb, l = e - r * nb;
        G[r * NB + l] = D[(size_t)r * ld + c0 + l];
    }
    __syncthreads();
    for (int t = tid; t < ndisp; t += nthr) dmap[meta[1 + nb + 2 * t]] = t;
    for (int e = tid; e < nb * ncols; e += nthr) {
        int l = e / ncols, jj = e - l * ncols;
        int q = q0 + jj;
        int j = q < c0 ? q : q + nb;
        U[l * cw + jj] = D[(size_t)meta[1 + l] * ld + j];
    }
    for (int e = tid; e < ndisp * ncols; e += nthr) {
        int t = e / ncols, jj = e - t * ncols;
        int q = q0 + jj;
        int j = q < c0 ? q : q + nb;
        DV[t * cw + jj] = D[(size_t)meta[2 + nb + 2 * t] * ld + j];
    }
    __syncthreads();
    for (int e = tid; e < S * ncols; e += nthr) {
        int r = e / ncols, jj = e - r * ncols;
        int q = q0 + jj;
        int j = q < c0 ? q : q + nb;
        T base;
        if (r >= c0 && r < c0 + nb) base = (T)0;
        else if (dmap[r] >= 0) base = DV[dmap[r] * cw + jj];
        else base = D[(size_t)r * ld + j];
        T acc = base;
        const T *g = G + r * NB;
#pragma unroll 8
        for (int l = 0; l < nb; ++l) acc += g[l] * U[l * cw + jj];
        D[(size_t)r * ld + j] = acc;
    }
    __syncthreads();
}

template <typename T, int NB>
__global__ void __launch_bounds__(kFactorThreads, 1) k_factor(BlockSys<T> a, Ctl *ctl, const int *skip)
{
    if (ctl->finished || (skip && *skip)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = a.S, ld = a.ld, L = a.L;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = 0; k < L; ++k) {
        T *D = a.D + (size_t)k * S * ld;
        int *ridx = a.ridx + (size_t)k * S;
        if (k > 0) {
            const T *Bp = a.D + (size_t)(k - 1) * S * ld;
            const int *sg = a.sig + (size_t)(k - 1) * S;
            const T *lo = a.lo + (size_t)k * S;
            const T *upp = a.up + (size_t)(k - 1) * S;
            for (long long e = gtid; e < (long long)S * S; e += gstride) {
                int i = (int)(e / S), j = (int)(e - (long long)i * S);
                D[(size_t)i * ld + j] -= lo[i] * Bp[(size_t)i * ld + sg[j]] * upp[j];
            }
        }
        for (long long i = gtid; i < S; i += gstride) ridx[i] = (int)i;
        if (!grid_barrier(a.bar, ctl)) return;
        for (int c0 = 0; c0 < S; c0 += NB) {
            const int nb = min(NB, S - c0);
            if (blockIdx.x == 0) panel_factor<T, NB>(D, ridx, a.pinfo, S, ld, c0, nb, ctl, smem);
            if (!grid_barrier(a.bar, ctl)) return;
            trailing_update<T, NB>(D, a.pinfo, S, ld, c0, nb, smem);
            if (!grid_barrier(a.bar, ctl)) return;
        }
        for (long long i = gtid; i < S; i += gstride) a.sig[(size_t)k * S + ridx[i]] = (int)i;
        if (!grid_barrier(a.bar, ctl)) return;
    }
}

// Forward and back substitution sweeps with the stored inverses.
//   g_0 = b_0; g_k = b_k - lo_k * (D'^-1_{k-1} g_{k-1})
//   x_{L-1} = D'^-1_{L-1} g_{L-1}; x_k = D'^-1_k (g_k - up_k * x_{k+1})
template <typename T>
__global__ void __launch_bounds__(kSolveThreads, 1) k_solve(BlockSys<T> a, const double *b, double *x, double *g, Ctl *ctl,
                                                                  const double *bscale, const int *skip)
{
    if (ctl->finished || (skip && *skip)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    T *vec = (T *)smem;
    const int S = a.S, ld = a.ld, L = a.L;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * warps + warp, nw = gridDim.x * warps;
    for (int k = 0; k < L; ++k) {
        if (k == 0) {
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x)
                g[i] = bscale ? b[i] * bscale[i] : b[i];
        } else {
            const int *rp = a.ridx + (size_t)(k - 1) * S;
            const double *gp = g + (size_t)(k - 1) * S;
            for (int m = threadIdx.x; m < S; m += blockDim.x) vec[m] = (T)gp[rp[m]];
            __syncthreads();
            const T *B = a.D + (size_t)(k - 1) * S * ld;
            for (int i = gw; i < S; i += nw) {
                const T *Bi = B + (size_t)i * ld;
                T acc = 0;
                for (int m = lane; m < S; m += 32) acc += Bi[m] * vec[m];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) {
                    double bi = b[(size_t)k * S + i];
                    if (bscale) bi *= bscale[(size_t)k * S + i];
                    g[(size_t)k * S + i] = bi - (double)a.lo[(size_t)k * S + i] * (double)acc;
                }
            }
        }
        if (!grid_barrier(a.bar, ctl)) return;
    }
    for (int k = L - 1; k >= 0; --k) {
        const int *rp = a.ridx + (size_t)k * S;
        const double *gk = g + (size_t)k * S;
        for (int m = threadIdx.x; m < S; m += blockDim.x) {
            int o = rp[m];
            double h = gk[o];
            if (k + 1 < L) h -= (double)a.up[(size_t)k * S + o] * x[(size_t)(k + 1) * S + o];
            vec[m] = (T)h;
        }
        __syncthreads();
        const T *B = a.D + (size_t)k * S * ld;
        for (int i = gw; i < S; i += nw) {
            const T *Bi = B + (size_t)i * ld;
            T acc = 0;
            for (int m = lane; m < S; m += 32) acc += Bi[m] * vec[m];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) x[(size_t)k * S + i] = (double)acc;
        }
        if (!grid_barrier(a.bar, ctl)) return;
    }
}

template <typename T, int NB>
size_t factor_smem(int S, int ctas)
{
    size_t panel = (size_t)S * (NB + 1) * sizeof(T) + 2 * (size_t)S * sizeof(int);
    int cw = (S + ctas - 1) / ctas;
    size_t trail = (size_t)S * NB * sizeof(T) + 2 * (size_t)NB * cw * sizeof(T)
                 + (1 + 3 * NB + (size_t)S) * sizeof(int);
    size_t m = panel > trail ? panel : trail;
    return (m + 255) & ~(size_t)255;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

size_t barrier_words() { return 2; }

int factor_plan(int S, int precision_bytes, int nb_hint, int ctas_hint, FactorPlan *out)
{
    FactorPlan p;
    p.threads = kFactorThreads;
    p.nb = precision_bytes == 8 ? 8 : 32;
    if (nb_hint > 0) p.nb = nb_hint;
    int sms = sm_count();
    // FP64 is ALU-bound on every SM; FP32 reads the panel per CTA, so fewer and wider slices
    int want = precision_bytes == 8 ? sms : (S + 15) / 16;
    if (ctas_hint > 0) want = ctas_hint;
    if (want > sms) want = sms;
    if (want < 1) want = 1;
    p.ctas = want;
    if (precision_bytes == 8) {
        if (p.nb == 8) p.smem = factor_smem<double, 8>(S, p.ctas);
        else if (p.nb == 16) p.smem = factor_smem<double, 16>(S, p.ctas);
        else return -1;
    } else {
        if (p.nb == 16) p.smem = factor_smem<float, 16>(S, p.ctas);
        else if (p.nb == 32) p.smem = factor_smem<float, 32>(S, p.ctas);
        else return -1;
    }
    if (p.smem > 227 * 1024) return -1;
    *out = p;
    return 0;
}

template <typename T, int NB>
static cudaError_t launch_factor_nb(const BlockSys<T> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                                    const int *skip)
{
    auto fn = k_factor<T, NB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return e;
    BlockSys<T> a = sys;
    void *args[] = {(void *)&a, (void *)&ctl, (void *)&skip};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(plan.ctas), dim3(plan.threads), args, plan.smem, st);
}

template <>
cudaError_t launch_factor<double>(const BlockSys<double> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                                  const int *skip)
{
    if (plan.nb == 8) return launch_factor_nb<double, 8>(sys, plan, ctl, st, skip);
    if (plan.nb == 16) return launch_factor_nb<double, 16>(sys, plan, ctl, st, skip);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_factor<float>(const BlockSys<float> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                                 const int *skip)
{
    if (plan.nb == 16) return launch_factor_nb<float, 16>(sys, plan, ctl, st, skip);
    if (plan.nb == 32) return launch_factor_nb<float, 32>(sys, plan, ctl, st, skip);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_solve(const BlockSys<T> &sys, const FactorPlan &plan, const double *b, double *x,
                         double *g, Ctl *ctl, cudaStream_t st, const double *bscale, const int *skip)
{
    (void)plan;
    auto fn = k_solve<T>;
    size_t smem = ((size_t)sys.S * sizeof(T) + 255) & ~(size_t)255;
    int warps = kSolveThreads / 32;
    int ctas = (sys.S + warps - 1) / warps;
    if (ctas > sm_count()) ctas = sm_count();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BlockSys<T> a = sys;
    void *args[] = {(void *)&a, (void *)&b, (void *)&x, (void *)&g, (void *)&ctl, (void *)&bscale, (void *)&skip};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(ctas), dim3(kSolveThreads), args, smem, st);
}

template cudaError_t launch_solve<double>(const BlockSys<double> &, const FactorPlan &, const double *, double *,
                                          double *, Ctl *, cudaStream_t, const double *, const int *);
template cudaError_t launch_solve<float>(const BlockSys<float> &, const FactorPlan &, const double *, double *,
                                         double *, Ctl *, cudaStream_t, const double *, const int *);

}  // namespace xk
