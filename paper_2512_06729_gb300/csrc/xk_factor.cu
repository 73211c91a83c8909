// Block-tridiagonal solve by block Thomas elimination with explicit block
// inverses.  For layer k the Schur complement D'_k = A_k - diag(lo_k)
// D'^-1_{k-1} diag(up_{k-1}) is formed and inverted in place by blocked
// Gauss-Jordan elimination with partial (row) pivoting.  One persistent,
// cooperatively launched kernel runs all layers; phases are separated by a
// grid barrier whose waits are bounded (on timeout the kernel records the
// error in the control block and returns).
//
// Pivoting is implicit: rows never move, perm_k[c] is the row that served as
// pivot of column c and iperm_k its inverse.  After factorization D holds B_k
// with D'^-1_k[i][j] = B_k[perm_k(i)][iperm_k(j)], so that
// (D'^-1_k g)[i] = sum_b B_k[perm_k(i)][b] g[perm_k(b)].
#include <cooperative_groups.h>
#include <math.h>

#include "xk_internal.cuh"

namespace xk {

namespace {

constexpr int kFactorThreads = 512;
constexpr int kSolveThreads = 512;

// Pivot search key: the magnitude's bit pattern is monotonic for |x|, so the
// comparison runs on the integer pipes (FP64 compares are slow on this part).
// High 32 bits: magnitude (float bits, or the top 32 bits of the double's
// magnitude); low 32 bits: ~row, so that among equal keys the lowest row wins.
__device__ __forceinline__ unsigned long long pivot_key(float v, int row)
{
    unsigned mag = __float_as_uint(v) & 0x7fffffffu;
    return ((unsigned long long)mag << 32) | (unsigned)(~row);
}
__device__ __forceinline__ unsigned long long pivot_key(double v, int row)
{
    unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return ((bits >> 31) << 32) | (unsigned)(~row);
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

constexpr int kRowsPerThread = 2;        // rows per thread in the trailing update: S <= 2 * kFactorThreads

// Gauss-Jordan on the panel columns [c0, c0 + nb) of D (all S rows), by one CTA,
// with implicit partial pivoting: rows are never moved; the pivot of column c
// is the unused row of largest |value|, recorded as perm[c] = row and
// iperm[row] = c (iperm = -1 marks rows not used as pivots yet).  The panel is
// staged in shared memory; per column two block barriers, with the elimination
// of column c-1 fused into the pivot search of column c.
template <typename T, int NB>
__device__ void panel_factor(T *D, int *perm, int *iperm, int *pinfo, int S, int ld, int c0, int nb, Ctl *ctl,
                             unsigned char *smem)
{
    constexpr int PS = NB + 1;                 // padded row stride (no bank conflicts)
    T *P = (T *)smem;                          // S x PS panel
    T *prow = P + (size_t)S * PS;              // normalized pivot row (PS); prow[c] = 1 / pivot
    int *ip = (int *)(prow + PS);              // S: iperm of this layer
    __shared__ unsigned long long red[32];
    __shared__ int s_piv;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;

    for (int e = tid; e < S * nb; e += nthr) {
        int r = e / nb, j = e - r * nb;
        P[r * PS + j] = D[(size_t)r * ld + c0 + j];
    }
    for (int r = tid; r < S; r += nthr) ip[r] = iperm[r];
    __syncthreads();

    int piv_prev = -1;
    for (int lc = 0; lc <= nb; ++lc) {
        unsigned long long best = 0ull;
        for (int r = tid; r < S; r += nthr) {
            T *Pr = P + r * PS;
            if (lc > 0 && r != piv_prev) {
                const T f = Pr[lc - 1];
                if (f != (T)0) {
#pragma unroll
                    for (int j = 0; j < NB; ++j)
                        if (j < nb && j != lc - 1) Pr[j] -= f * prow[j];
                    Pr[lc - 1] = -f * prow[lc - 1];
                }
            }
            if (lc < nb && ip[r] < 0) best = umax64(best, pivot_key(Pr[lc], r));
        }
        if (lc == nb) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            unsigned long long all = lane < nw ? red[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) all = umax64(all, __shfl_xor_sync(0xffffffffu, all, o));
            int piv = (int)(~(unsigned)(all & 0xffffffffull));
            if ((all >> 32) == 0ull || piv < 0 || piv >= S) {
                // zero column: singular block; keep the bookkeeping consistent with the first unused row
                if (lane == 0) atomicExch(&ctl->err_singular, 1);
                piv = -1;
                for (int r = 0; r < S && piv < 0; ++r)
                    if (ip[r] < 0) piv = r;
                if (piv < 0) piv = 0;
            }
            const T pv = P[piv * PS + lc];
            const T di = (pv != (T)0) ? (T)1 / pv : (T)0;
            for (int j = lane; j < nb; j += 32) {
                T val = (j == lc) ? di : P[piv * PS + j] * di;
                prow[j] = val;
                P[piv * PS + j] = val;
            }
            if (lane == 0) {
                s_piv = piv;
                ip[piv] = c0 + lc;
                perm[c0 + lc] = piv;
                pinfo[lc] = piv;
            }
        }
        __syncthreads();
        piv_prev = s_piv;
    }
    __syncthreads();
    for (int e = tid; e < S * nb; e += nthr) {
        int r = e / nb, j = e - r * nb;
        D[(size_t)r * ld + c0 + j] = P[r * PS + j];
    }
    for (int r = tid; r < S; r += nthr) iperm[r] = ip[r];
    __threadfence();
}

// Apply the panel's eliminations to the other columns j: with G the panel
// columns and U the panel's pivot rows (values before this update),
//   pivot rows of this panel: D[r][j] = sum_l G[r][l] U[l][j]
//   all other rows:           D[r][j] += sum_l G[r][l] U[l][j].
// Each CTA owns a slice of columns; each thread owns whole rows and keeps its
// row of G in registers.
template <typename T, int NB>
__device__ void trailing_update(T *D, const int *pinfo, const int *iperm, int S, int ld, int c0, int nb,
                                unsigned char *smem, int bid, int nblk)
{
    constexpr int MAXC = 8;                            // columns per CTA handled in registers
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int others = S - nb;
    const int cw = (others + nblk - 1) / nblk;
    T *U = (T *)smem;                                  // NB x cw
    for (int q0 = bid * cw, qend = min(others, (bid + 1) * cw); q0 < qend; q0 += MAXC) {
        const int ncols = min(MAXC, qend - q0);
        // rows nb..NB-1 of U (ragged last panel) are zero: the update below runs over all NB
        for (int e = tid; e < NB * ncols; e += nthr) {
            int l = e / ncols, jj = e - l * ncols;
            int q = q0 + jj;
            int j = q < c0 ? q : q + nb;
            U[l * MAXC + jj] = l < nb ? D[(size_t)pinfo[l] * ld + j] : (T)0;
        }
        __syncthreads();
#pragma unroll 1
        for (int rr = 0; rr < kRowsPerThread; ++rr) {
            const int r = tid + rr * nthr;
            if (r >= S) break;
            const int ip = iperm[r];
            const bool pivot_row = ip >= c0 && ip < c0 + nb;
            T g[NB];
            const T *Gr = D + (size_t)r * ld + c0;
#pragma unroll
            for (int l = 0; l < NB; ++l) g[l] = (l < nb) ? Gr[l] : (T)0;
            T acc[MAXC];
#pragma unroll
            for (int jj = 0; jj < MAXC; ++jj) {
                int q = q0 + jj;
                int j = q < c0 ? q : q + nb;
                acc[jj] = (jj < ncols && !pivot_row) ? D[(size_t)r * ld + j] : (T)0;
            }
#pragma unroll
            for (int l = 0; l < NB; ++l)
#pragma unroll
                for (int jj = 0; jj < MAXC; ++jj) acc[jj] += g[l] * U[l * MAXC + jj];
#pragma unroll
            for (int jj = 0; jj < MAXC; ++jj) {
                int q = q0 + jj;
                int j = q < c0 ? q : q + nb;
                if (jj < ncols) D[(size_t)r * ld + j] = acc[jj];
            }
        }
        __syncthreads();
    }
}

// mode 0: all layers top-down on the whole grid.  mode 1 (twisted): the grid splits in two halves
// with their own barrier counters and panel scratch; the first half eliminates layers 0..mid-1
// top-down, the second layers L-1..mid+1 bottom-up (E'_k = A_k - diag(up_k) E'^-1_{k+1}
// diag(lo_{k+1})).  mode 2: the middle layer on the whole grid, with both Schur terms.
template <typename T, int NB>
__global__ void __launch_bounds__(kFactorThreads, 1) k_factor(BlockSys<T> a, Ctl *ctl, const int *skip, int mode,
                                                               int mid)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = a.S, ld = a.ld, L = a.L;
    const int half = mode == 1 ? (int)(blockIdx.x >= gridDim.x / 2) : 0;
    const int nblk = mode == 1 ? (int)gridDim.x / 2 : (int)gridDim.x;
    const int bid = (int)blockIdx.x - half * nblk;
    unsigned *bar = a.bar + 2 * half;
    int *pinfo = a.pinfo + 64 * half;
    const long long gstride = (long long)nblk * blockDim.x;
    const long long gtid = (long long)bid * blockDim.x + threadIdx.x;
    int nsteps = L, k0 = 0, dk = 1;
    if (mode == 1) {
        nsteps = half == 0 ? mid : L - 1 - mid;
        k0 = half == 0 ? 0 : L - 1;
        dk = half == 0 ? 1 : -1;
    } else if (mode == 2) {
        nsteps = 1;
        k0 = mid;
        dk = 0;
    }
    for (int step = 0; step < nsteps; ++step) {
        const int k = k0 + step * dk;
        T *D = a.D + (size_t)k * S * ld;
        int *perm = a.perm + (size_t)k * S;
        int *iperm = a.iperm + (size_t)k * S;
        // Schur terms: D'^-1 of a neighbour n is B_n[perm_n(i)][iperm_n(j)]
        auto schur = [&](int nbr, const T *rowc, const T *colc) {
            const T *Bn = a.D + (size_t)nbr * S * ld;
            const int *pn = a.perm + (size_t)nbr * S;
            const int *ipn = a.iperm + (size_t)nbr * S;
            for (long long e = gtid; e < (long long)S * S; e += gstride) {
                int i = (int)(e / S), j = (int)(e - (long long)i * S);
                D[(size_t)i * ld + j] -= rowc[i] * Bn[(size_t)pn[i] * ld + ipn[j]] * colc[j];
            }
        };
        if (mode == 2) {
            if (k > 0) schur(k - 1, a.lo + (size_t)k * S, a.up + (size_t)(k - 1) * S);
            if (k + 1 < L) schur(k + 1, a.up + (size_t)k * S, a.lo + (size_t)(k + 1) * S);
        } else if (step > 0) {
            if (dk > 0) schur(k - 1, a.lo + (size_t)k * S, a.up + (size_t)(k - 1) * S);
            else schur(k + 1, a.up + (size_t)k * S, a.lo + (size_t)(k + 1) * S);
        }
        for (long long i = gtid; i < S; i += gstride) iperm[i] = -1;
        if (!grid_barrier(bar, ctl, nblk)) return;
        for (int c0 = 0; c0 < S; c0 += NB) {
            const int nb = min(NB, S - c0);
            if (bid == 0) panel_factor<T, NB>(D, perm, iperm, pinfo, S, ld, c0, nb, ctl, smem);
            if (!grid_barrier(bar, ctl, nblk)) return;
            trailing_update<T, NB>(D, pinfo, iperm, S, ld, c0, nb, smem, bid, nblk);
            if (!grid_barrier(bar, ctl, nblk)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 block inversion with partial pivoting, each panel's pivots chosen first.
//
// In panel_factor the sequential part of each panel -- nb columns of pivot
// search plus Gauss-Jordan elimination of every row over all nb panel columns
// -- runs in FP64 on one SM, whose FP64 rate (about 2 FMA per clock) makes it
// the critical path: about S * nb^2 / 2 clocks per panel.  Here CTA 0 only
// chooses the nb pivot rows: right-looking elimination of the panel restricted
// to the rows not yet used as pivots and to the columns right of the current
// one (the same candidates and values as partial pivoting in panel_factor, at
// about a quarter of the FP64 work), keeping the multipliers, so that the
// eliminated rows of the pivots are the LU factors of the nb x nb pivot block
// M.  Every CTA then forms G_r = -D[r][panel] M^-1 for its slice of rows by two
// triangular solves with those factors (an explicit M^-1 loses accuracy on
// nearly singular blocks), and the trailing update of the other columns is
// the one of the column-by-column kernel.
// ---------------------------------------------------------------------------
template <int NB>
__device__ void panel_preview(const double *D, int *perm, int *iperm, int *pinfo, double *lu, int S, int ld,
                              int c0, int nb, Ctl *ctl, unsigned char *smem)
{
    constexpr int PS = NB + 1;
    double *P = (double *)smem;                // S x PS: the panel
    int *ip = (int *)(P + (size_t)S * PS);     // S: iperm of this layer (-1: not a pivot yet)
    __shared__ int s_piv[NB];
    __shared__ unsigned long long red[32];
    __shared__ int s_cur;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;

    for (int r = tid; r < S; r += nthr) ip[r] = iperm[r];
    for (int e = tid; e < S * nb; e += nthr) {
        const int r = e / nb, j = e - r * nb;
        P[r * PS + j] = D[(size_t)r * ld + c0 + j];
    }
    __syncthreads();

    __shared__ double s_rcp;                   // 1 / pivot of the previous column (one FP64 division per column)
    int piv_prev = -1;
    for (int lc = 0; lc <= nb; ++lc) {
        unsigned long long best = 0ull;
        const double rcp = lc > 0 ? s_rcp : 0.0;
        for (int r = tid; r < S; r += nthr) {
            if (ip[r] >= 0) continue;              // pivot of an earlier panel or column
            double *Pr = P + r * PS;
            if (lc > 0) {
                const double f = Pr[lc - 1] * rcp;
#pragma unroll
                for (int j = 1; j < NB; ++j)
                    if (j >= lc && j < nb) Pr[j] = fma(-f, P[piv_prev * PS + j], Pr[j]);
                Pr[lc - 1] = f;                    // the multiplier L[r][lc - 1]
            }
            if (lc < nb) best = umax64(best, pivot_key(Pr[lc], r));
        }
        if (lc == nb) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            unsigned long long all = lane < nw ? red[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) all = umax64(all, __shfl_xor_sync(0xffffffffu, all, o));
            if (lane == 0) {
                int piv = (int)(~(unsigned)(all & 0xffffffffull));
                if ((all >> 32) == 0ull || piv < 0 || piv >= S) {
                    // no nonzero candidate: singular block; keep the bookkeeping consistent
                    atomicExch(&ctl->err_singular, 1);
                    piv = -1;
                    for (int r = 0; r < S && piv < 0; ++r)
                        if (ip[r] < 0) piv = r;
                    if (piv < 0) piv = 0;
                }
                ip[piv] = c0 + lc;
                s_piv[lc] = piv;
                s_cur = piv;
                const double pv = P[piv * PS + lc];
                s_rcp = pv != 0.0 ? 1.0 / pv : 0.0;
            }
        }
        __syncthreads();
        piv_prev = s_cur;
    }
    if (tid < nb) {
        const int pr = s_piv[tid];
        perm[c0 + tid] = pr;
        iperm[pr] = c0 + tid;
        pinfo[tid] = pr;
    }
    // LU factors of the pivot block M[i][l] = D[s_piv[i]][c0 + l] in the chosen order: row i of
    // the eliminated panel holds L[i][0..i) (multipliers) and U[i][i..nb)
    __syncthreads();
    for (int e = tid; e < nb * nb; e += nthr) {
        const int i = e / nb, l = e - i * nb;
        lu[i * NB + l] = P[s_piv[i] * PS + l];
    }
    __threadfence();
}

template <int NB>
__global__ void __launch_bounds__(kFactorThreads, 1) k_factor_pv(BlockSys<double> a, double *lu, Ctl *ctl,
                                                                  const int *skip)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double Ds[NB * NB];
    __shared__ double Dr_rcp[NB];
    const int S = a.S, ld = a.ld, L = a.L;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int rs = (S + gridDim.x - 1) / gridDim.x, r0 = blockIdx.x * rs, r1 = min(S, r0 + rs);
    for (int k = 0; k < L; ++k) {
        double *D = a.D + (size_t)k * S * ld;
        int *perm = a.perm + (size_t)k * S;
        int *iperm = a.iperm + (size_t)k * S;
        if (k > 0) {
            // D'_k = A_k - diag(lo_k) D'^-1_{k-1} diag(up_{k-1}), D'^-1[i][j] = B[perm(i)][iperm(j)]
            const double *Bp = a.D + (size_t)(k - 1) * S * ld;
            const int *pp = a.perm + (size_t)(k - 1) * S;
            const int *ipp = a.iperm + (size_t)(k - 1) * S;
            const double *lo = a.lo + (size_t)k * S;
            const double *upp = a.up + (size_t)(k - 1) * S;
            for (long long e = gtid; e < (long long)S * S; e += gstride) {
                int i = (int)(e / S), j = (int)(e - (long long)i * S);
                D[(size_t)i * ld + j] -= lo[i] * Bp[(size_t)pp[i] * ld + ipp[j]] * upp[j];
            }
        }
        for (long long i = gtid; i < S; i += gstride) iperm[i] = -1;
        if (!grid_barrier(a.bar, ctl)) return;
        for (int c0 = 0; c0 < S; c0 += NB) {
            const int nb = min(NB, S - c0);
            if (blockIdx.x == 0) panel_preview<NB>(D, perm, iperm, a.pinfo, lu, S, ld, c0, nb, ctl, smem);
            if (!grid_barrier(a.bar, ctl)) return;
            // G_r = -D[r][panel] M^-1 (pivot row p_i of the panel: row i of M^-1), from the LU
            // factors of M by two triangular solves, G L U = rhs: w U = rhs, then G L = w
            for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
                const int i = e / NB, l = e - i * NB;
                Ds[e] = (i < nb && l < nb) ? lu[i * NB + l] : 0.0;
            }
            if (threadIdx.x < NB) {
                const double u = threadIdx.x < nb ? lu[threadIdx.x * NB + threadIdx.x] : 0.0;
                Dr_rcp[threadIdx.x] = u != 0.0 ? 1.0 / u : 0.0;
            }
            __syncthreads();
#pragma unroll 1
            for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
                double *Dr = D + (size_t)r * ld + c0;
                const int ipr = iperm[r];
                const bool piv_row = ipr >= c0 && ipr < c0 + nb;
                double w[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j >= nb) { w[j] = 0.0; continue; }
                    double acc = piv_row ? (ipr - c0 == j ? 1.0 : 0.0) : -Dr[j];
#pragma unroll
                    for (int k = 0; k < j; ++k) acc = fma(-w[k], Ds[k * NB + j], acc);
                    w[j] = acc * Dr_rcp[j];
                }
#pragma unroll
                for (int i = NB - 1; i >= 0; --i) {
                    if (i >= nb) continue;
                    double g = w[i];
#pragma unroll
                    for (int k = i + 1; k < NB; ++k)
                        if (k < nb) g = fma(-w[k], Ds[k * NB + i], g);
                    w[i] = g;
                }
#pragma unroll
                for (int l = 0; l < NB; ++l)
                    if (l < nb) Dr[l] = w[l];
            }
            if (!grid_barrier(a.bar, ctl)) return;
            trailing_update<double, NB>(D, a.pinfo, iperm, S, ld, c0, nb, smem, blockIdx.x, gridDim.x);
            if (!grid_barrier(a.bar, ctl)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 block inversion without pivoting (preconditioner of the mixed path).
//
// Blocked Gauss-Jordan with panels of NB columns and no row exchanges: the
// diagonal NB x NB block of each panel is inverted by one warp, every other
// row r of the panel becomes G_r = -D[r][panel] Dpp^-1, and the other columns
// are updated with the panel's rows.  Look-ahead: CTA 0 owns the next panel's
// columns in each update and inverts the next diagonal block right after, so
// each panel costs one grid barrier.  G of a panel is written to a two-slot
// buffer; the CTA that owns those columns in the next panel reads it there.
// The FGMRES iteration on the exact FP64 operator (and, when it does not
// converge, the pivoted FP64 factorization) is what guarantees the solution;
// this factorization only has to be a good approximate inverse.
// ---------------------------------------------------------------------------

// Invert the nb x nb block at (c0, c0) of D in place with one warp (no pivoting).
template <int NB>
__device__ void diag_inverse_warp(float *D, int ld, int c0, int nb, float *Bs, Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    // Bs: NB x (NB + 1) staging in shared memory
    for (int r = 0; r < nb; ++r)
        if (lane < nb) Bs[r * (NB + 1) + lane] = D[(size_t)(c0 + r) * ld + c0 + lane];
    __syncwarp();
    for (int c = 0; c < nb; ++c) {
        const float d = Bs[c * (NB + 1) + c];
        const float inv = (d != 0.f) ? 1.f / d : 0.f;
        if (d == 0.f && lane == 0) atomicExch(&ctl->err_singular, 1);
        float f[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) f[r] = (r < nb) ? Bs[r * (NB + 1) + c] : 0.f;
        const float bc = (lane < nb) ? ((lane == c) ? inv : Bs[c * (NB + 1) + lane] * inv) : 0.f;
        __syncwarp();
        if (lane < nb) {
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                if (r >= nb) break;
                if (r == c) Bs[r * (NB + 1) + lane] = bc;
                else Bs[r * (NB + 1) + lane] = (lane == c) ? -f[r] * inv : Bs[r * (NB + 1) + lane] - f[r] * bc;
            }
        }
        __syncwarp();
    }
    for (int r = 0; r < nb; ++r)
        if (lane < nb) D[(size_t)(c0 + r) * ld + c0 + lane] = Bs[r * (NB + 1) + lane];
    __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(kFactorThreads, 1) k_factor_np(BlockSys<float> a, float *gbuf, Ctl *ctl,
                                                                  const int *skip)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    constexpr int MAXC = 8;
    __shared__ float Dinv[NB * (NB + 1)];
    __shared__ float U[NB * MAXC];
    __shared__ float Bs[NB * (NB + 1)];
    const int S = a.S, ld = a.ld, L = a.L;
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, nw = nthr >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const long long gstride = (long long)G * blockDim.x;
    const long long gtid = (long long)b * blockDim.x + threadIdx.x;
    const int npan = (S + NB - 1) / NB;
    for (int k = 0; k < L; ++k) {
        float *D = a.D + (size_t)k * S * ld;
        int *perm = a.perm + (size_t)k * S;
        int *iperm = a.iperm + (size_t)k * S;
        if (k > 0) {
            // D'_k = A_k - diag(lo_k) D'^-1_{k-1} diag(up_{k-1}) (no permutation here)
            const float *Bp = a.D + (size_t)(k - 1) * S * ld;
            const float *lo = a.lo + (size_t)k * S;
            const float *upp = a.up + (size_t)(k - 1) * S;
            for (long long e = gtid; e < (long long)S * S; e += gstride) {
                int i = (int)(e / S), j = (int)(e - (long long)i * S);
                D[(size_t)i * ld + j] -= lo[i] * Bp[(size_t)i * ld + j] * upp[j];
            }
        }
        for (long long i = gtid; i < S; i += gstride) { perm[i] = (int)i; iperm[i] = (int)i; }
        if (!grid_barrier(a.bar, ctl)) return;
        if (b == 0 && warp == 0) diag_inverse_warp<NB>(D, ld, 0, min(NB, S), Bs, ctl);
        if (!grid_barrier(a.bar, ctl)) return;
        for (int p = 0; p < npan; ++p) {
            const int c0 = p * NB, nb = min(NB, S - c0), c1 = c0 + nb;
            const int nbn = (p + 1 < npan) ? min(NB, S - c1) : 0;
            const int cp = c0 - NB, nbp = (p > 0) ? NB : 0;
            const float *gprev = gbuf + (size_t)((p + 1) & 1) * S * NB;
            float *gcur = gbuf + (size_t)(p & 1) * S * NB;
            // value of D[r][j] before this panel: the previous panel's G lives in its buffer slot
            auto val = [&](int r, int j) -> float {
                return (j >= cp && j < cp + nbp) ? gprev[(size_t)r * NB + (j - cp)] : D[(size_t)r * ld + j];
            };
            for (int e = tid; e < nb * nb; e += nthr) {
                int l = e / nb, m = e - l * nb;
                Dinv[l * (NB + 1) + m] = D[(size_t)(c0 + l) * ld + c0 + m];
            }
            __syncthreads();
            // phase A: G rows of this CTA's row slice: pivot rows take Dinv, the others -D[r][panel] Dinv
            const int rs = (S + G - 1) / G, r0 = b * rs, r1 = min(S, r0 + rs);
            for (int e = tid; e < (r1 - r0) * nb; e += nthr) {
                const int r = r0 + e / nb, l = e - (e / nb) * nb;
                float gv;
                if (r >= c0 && r < c1) {
                    gv = Dinv[(r - c0) * (NB + 1) + l];
                } else {
                    float acc = 0.f;
                    for (int m = 0; m < nb; ++m) acc += val(r, c0 + m) * Dinv[m * (NB + 1) + l];
                    gv = -acc;
                }
                gcur[(size_t)r * NB + l] = gv;
            }
            if (!grid_barrier(a.bar, ctl)) return;
            // phase B: update this CTA's columns; CTA 0 takes the next panel's columns (look-ahead)
            const int others = S - nb;
            int base, count, skipq;
            if (G == 1 || nbn == 0) {
                const int cw = (others + G - 1) / G;
                base = b * cw; count = max(0, min(others, base + cw) - base); skipq = 0;
            } else if (b == 0) {
                base = c0; count = nbn; skipq = 0;
            } else {
                const int rest = others - nbn, cw = (rest + G - 2) / (G - 1);
                base = (b - 1) * cw; count = max(0, min(rest, base + cw) - base); skipq = nbn;
            }
            auto col_of = [&](int i) -> int {
                int q = base + i;
                if (skipq > 0 && q >= c0) q += skipq;
                return q < c0 ? q : q + nb;
            };
            for (int i0 = 0; i0 < count; i0 += MAXC) {
                const int ncols = min(MAXC, count - i0);
                // rows nb..NB-1 of U (ragged last panel) are zero: the update below runs over all NB
                for (int e = tid; e < NB * ncols; e += nthr) {
                    int l = e / ncols, jj = e - l * ncols;
                    U[l * MAXC + jj] = l < nb ? val(c0 + l, col_of(i0 + jj)) : 0.f;
                }
                __syncthreads();
#pragma unroll 1
                for (int rr = 0; rr < kRowsPerThread; ++rr) {
                    const int r = tid + rr * nthr;
                    if (r >= S) break;
                    const bool pivot_row = r >= c0 && r < c1;
                    float g[NB];
                    const float *gr = gcur + (size_t)r * NB;
#pragma unroll
                    for (int l = 0; l < NB; ++l) g[l] = (l < nb) ? gr[l] : 0.f;
                    float acc[MAXC];
#pragma unroll
                    for (int jj = 0; jj < MAXC; ++jj)
                        acc[jj] = (jj < ncols && !pivot_row) ? val(r, col_of(i0 + jj)) : 0.f;
#pragma unroll
                    for (int l = 0; l < NB; ++l)
#pragma unroll
                        for (int jj = 0; jj < MAXC; ++jj) acc[jj] += g[l] * U[l * MAXC + jj];
#pragma unroll
                    for (int jj = 0; jj < MAXC; ++jj)
                        if (jj < ncols) D[(size_t)r * ld + col_of(i0 + jj)] = acc[jj];
                }
                __syncthreads();
            }
            // look-ahead: CTA 0 inverts the next diagonal block it has just updated
            if (b == 0 && nbn > 0 && warp == 0) diag_inverse_warp<NB>(D, ld, c1, nbn, Bs, ctl);
            (void)nw;
            if (!grid_barrier(a.bar, ctl)) return;
        }
        // the last panel's columns are not updated by any later panel: store its G
        {
            const int c0 = (npan - 1) * NB, nb = S - c0;
            const float *glast = gbuf + (size_t)((npan - 1) & 1) * S * NB;
            for (long long e = gtid; e < (long long)S * nb; e += gstride) {
                int r = (int)(e / nb), l = (int)(e - (long long)r * nb);
                D[(size_t)r * ld + c0 + l] = glast[(size_t)r * NB + l];
            }
        }
        if (!grid_barrier(a.bar, ctl)) return;
    }
}

// Forward and back substitution sweeps with the stored inverses.
//   g_0 = b_0; g_k = b_k - lo_k * (D'^-1_{k-1} g_{k-1})
//   x_{L-1} = D'^-1_{L-1} g_{L-1}; x_k = D'^-1_k (g_k - up_k * x_{k+1})
template <typename T>
__global__ void __launch_bounds__(kSolveThreads, 1) k_solve(BlockSys<T> a, const double *b, double *x, double *g, Ctl *ctl,
                                                                  const double *bscale, const int *skip,
                                                                  const double *xscale)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
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
            const int *rp = a.perm + (size_t)(k - 1) * S;
            const double *gp = g + (size_t)(k - 1) * S;
            for (int m = threadIdx.x; m < S; m += blockDim.x) vec[m] = (T)gp[rp[m]];
            __syncthreads();
            const T *B = a.D + (size_t)(k - 1) * S * ld;
            for (int i = gw; i < S; i += nw) {
                const T *Bi = B + (size_t)rp[i] * ld;
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
        const int *rp = a.perm + (size_t)k * S;
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
            const T *Bi = B + (size_t)rp[i] * ld;
            T acc = 0;
            for (int m = lane; m < S; m += 32) acc += Bi[m] * vec[m];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) x[(size_t)k * S + i] = (double)acc;
        }
        if (!grid_barrier(a.bar, ctl)) return;
    }
    if (xscale) {
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)L * S;
             e += (long long)gridDim.x * blockDim.x)
            x[e] *= xscale[e];
    }
}

template <typename T, int NB>
size_t factor_smem(int S, int ctas)
{
    (void)ctas;
    size_t panel = (size_t)S * (NB + 1) * sizeof(T) + (NB + 1) * sizeof(T) + (size_t)S * sizeof(int) + 64;
    size_t trail = (size_t)NB * 8 * sizeof(T) + 64;
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
    if (S > kRowsPerThread * kFactorThreads) return -1;
    int want = sms;
    if (ctas_hint > 0) want = ctas_hint;
    if (want > sms) want = sms;
    if (want < 1) want = 1;
    p.ctas = want;
    if (precision_bytes == 8) {
        if (p.nb == 8) p.smem = factor_smem<double, 8>(S, p.ctas);
        else if (p.nb == 16) p.smem = factor_smem<double, 16>(S, p.ctas);
        else if (p.nb == 32) p.smem = 0;
        else return -1;
        // the pivot choice: S x (nb + 1) doubles and S ints; the trailing update: nb x 8 doubles
        size_t pv = (size_t)S * (p.nb + 1) * sizeof(double) + (size_t)S * sizeof(int) + 64;
        size_t tr = (size_t)p.nb * 8 * sizeof(double) + 64;
        pv = pv > tr ? pv : tr;
        pv = (pv + 255) & ~(size_t)255;
        if (pv > p.smem) p.smem = pv;
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
    auto go = [&](int mode, int mid, int ctas) -> cudaError_t {
        void *args[] = {(void *)&a, (void *)&ctl, (void *)&skip, (void *)&mode, (void *)&mid};
        count_launches(1);
        return cudaLaunchCooperativeKernel((const void *)fn, dim3(ctas), dim3(plan.threads), args, plan.smem, st);
    };
    if (!(plan.twisted && sys.L >= 3 && plan.ctas >= 2)) return go(0, 0, plan.ctas);
    // twisted elimination: both ends at once on the two halves of the grid, then the middle layer
    const int mid = sys.L / 2;
    e = go(1, mid, plan.ctas & ~1);
    if (e == cudaSuccess) e = go(2, mid, plan.ctas);
    return e;
}

template <int NB>
static cudaError_t launch_factor_pv_nb(const BlockSys<double> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                                       const int *skip)
{
    auto fn = k_factor_pv<NB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return e;
    BlockSys<double> a = sys;
    double *lu = plan.dinv;
    void *args[] = {(void *)&a, (void *)&lu, (void *)&ctl, (void *)&skip};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(plan.ctas), dim3(plan.threads), args, plan.smem, st);
}

template <>
cudaError_t launch_factor<double>(const BlockSys<double> &sys, const FactorPlan &plan, Ctl *ctl, cudaStream_t st,
                                  const int *skip)
{
    if (plan.preview && plan.dinv) {
        if (plan.nb == 8) return launch_factor_pv_nb<8>(sys, plan, ctl, st, skip);
        if (plan.nb == 16) return launch_factor_pv_nb<16>(sys, plan, ctl, st, skip);
        if (plan.nb == 32) return launch_factor_pv_nb<32>(sys, plan, ctl, st, skip);
        return cudaErrorInvalidValue;
    }
    if (plan.nb == 8) return launch_factor_nb<double, 8>(sys, plan, ctl, st, skip);
    if (plan.nb == 16) return launch_factor_nb<double, 16>(sys, plan, ctl, st, skip);
    return cudaErrorInvalidValue;
}

cudaError_t launch_factor_nopivot(const BlockSys<float> &sys, const FactorPlan &plan, float *gbuf, Ctl *ctl,
                                  cudaStream_t st, const int *skip)
{
    BlockSys<float> a = sys;
    void *args[] = {(void *)&a, (void *)&gbuf, (void *)&ctl, (void *)&skip};
    count_launches(1);
    if (plan.nb == 32)
        return cudaLaunchCooperativeKernel((const void *)k_factor_np<32>, dim3(plan.ctas), dim3(plan.threads), args, 0, st);
    if (plan.nb == 16)
        return cudaLaunchCooperativeKernel((const void *)k_factor_np<16>, dim3(plan.ctas), dim3(plan.threads), args, 0, st);
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
                         double *g, Ctl *ctl, cudaStream_t st, const double *bscale, const int *skip,
                         const double *xscale)
{
    auto fn = k_solve<T>;
    size_t smem = ((size_t)sys.S * sizeof(T) + 255) & ~(size_t)255;
    int warps = kSolveThreads / 32;
    int ctas = (sys.S + warps - 1) / warps;
    if (ctas > sm_count()) ctas = sm_count();
    if (plan.ctas > 0 && ctas > plan.ctas) ctas = plan.ctas;    // stay within the column's share of the SMs
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BlockSys<T> a = sys;
    void *args[] = {(void *)&a, (void *)&b, (void *)&x, (void *)&g, (void *)&ctl, (void *)&bscale, (void *)&skip,
                    (void *)&xscale};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(ctas), dim3(kSolveThreads), args, smem, st);
}

template cudaError_t launch_solve<double>(const BlockSys<double> &, const FactorPlan &, const double *, double *,
                                          double *, Ctl *, cudaStream_t, const double *, const int *,
                                          const double *);
template cudaError_t launch_solve<float>(const BlockSys<float> &, const FactorPlan &, const double *, double *,
                                         double *, Ctl *, cudaStream_t, const double *, const int *, const double *);

}  // namespace xk
