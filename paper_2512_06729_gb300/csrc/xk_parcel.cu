// Lagrangian parcel scheme (Sec. 2, Fig. 1 and Fig. 2): one global iteration carries an air
// parcel from the bottom layer to the top and back (layers 0 .. L-1, then L-2 .. 0).  In layer k
// the parcel's densities x evolve for the eddy mixing time tau_k = dz_k^2 / K_zz,k under that
// layer's chemistry (Sec. 2.3) and molecular diffusion written as a pseudo-reaction pair with the
// stored densities of layers k -+ 1 (Sec. 2.1, after Eq. 4: the molecular part of Eq. 2's flux);
// eddy diffusion is the parcel's motion and has no term.  Within a visit: linearly implicit Euler
// steps (I/h - dF/dx) delta = F under the step controller of the Eulerian path, each solved by
// Gaussian elimination with partial pivoting plus two sweeps of FP64 iterative refinement.  The
// parcel keeps its mixing ratios from layer to layer, and each visit leaves its densities as the
// layer's.
//
// The sweep is sequential in the layers, so one CTA runs a whole iteration: every reduction,
// pivot search and elimination step stays inside the block (no grid-wide wait).  The step's
// vectors live in shared memory, and so do its two S x S matrices (the system and its factors)
// when they fit (S up to 111); larger systems keep them in global memory, where they stay in L2.
#include <cfloat>

#include "xk_internal.cuh"

namespace xk {

namespace {

constexpr int kMaxWarps = 32;
constexpr int kRefineSweeps = 2;          // FP64 iterative-refinement sweeps of every implicit step
constexpr size_t kSmemLimit = 200 * 1024; // dynamic shared memory the kernel may ask for

struct Shared {
    double red[kMaxWarps];
    int ired[kMaxWarps];
    double h, t, hs;
    int last, done;
};

__device__ __forceinline__ int nwarps() { return blockDim.x >> 5; }

// max over the block; every thread gets the result
__device__ double block_max(double v, Shared &sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    v = lane < nwarps() ? sh.red[lane] : -DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ int block_or(int v, Shared &sh)
{
    v = __any_sync(0xffffffffu, v) ? 1 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh.ired[warp] = v;
    __syncthreads();
    v = lane < nwarps() ? sh.ired[lane] : 0;
    return __any_sync(0xffffffffu, v) ? 1 : 0;
}

// Row of the largest |A[i][c]|, i >= c (the first on ties, as a sequential scan picks it), or -1.
__device__ int pivot_row(const double *A, int S, int c, Shared &sh)
{
    double best = -1.0;
    int bi = S;
    for (int i = c + threadIdx.x; i < S; i += blockDim.x) {
        const double v = fabs(A[(long long)i * S + c]);
        if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { sh.red[warp] = best; sh.ired[warp] = bi; }
    __syncthreads();
    best = lane < nwarps() ? sh.red[lane] : -1.0;
    bi = lane < nwarps() ? sh.ired[lane] : S;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    return best > 0.0 ? bi : -1;
}

// A <- its LU factors with partial pivoting (whole rows swapped; row c of the factors came from
// row piv[c] of the rows as they stood at step c).  0, or -1 on a zero pivot column.
__device__ int lu_factor(double *A, int *piv, int S, Shared &sh)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nwarps();
    for (int c = 0; c < S; ++c) {
        const int p = pivot_row(A, S, c, sh);
        if (p < 0) return -1;
        if (threadIdx.x == 0) piv[c] = p;
        if (p != c)
            for (int j = threadIdx.x; j < S; j += blockDim.x) {
                const double t = A[(long long)c * S + j];
                A[(long long)c * S + j] = A[(long long)p * S + j];
                A[(long long)p * S + j] = t;
            }
        __syncthreads();
        const double inv = 1.0 / A[(long long)c * S + c];
        // a warp per row below the pivot: its multiplier, then the row update along the lanes
        for (int i = c + 1 + warp; i < S; i += nw) {
            double *Ai = A + (long long)i * S;
            const double l = Ai[c] * inv;
            __syncwarp();
            if (lane == 0) Ai[c] = l;
            for (int j = c + 1 + lane; j < S; j += 32) Ai[j] -= l * A[(long long)c * S + j];
        }
        __syncthreads();
    }
    return 0;
}

// x <- (LU)^-1 P x with the factors of lu_factor.
__device__ void lu_solve(const double *A, const int *piv, double *x, int S)
{
    if (threadIdx.x == 0)
        for (int c = 0; c < S; ++c) {
            const int p = piv[c];
            if (p != c) { const double t = x[c]; x[c] = x[p]; x[p] = t; }
        }
    __syncthreads();
    for (int c = 0; c < S; ++c) {            // unit lower triangle, column by column
        const double xc = x[c];
        for (int i = c + 1 + threadIdx.x; i < S; i += blockDim.x) x[i] -= A[(long long)i * S + c] * xc;
        __syncthreads();
    }
    for (int c = S - 1; c >= 0; --c) {       // upper triangle
        const double xc = x[c] * (1.0 / A[(long long)c * S + c]);
        __syncthreads();
        if (threadIdx.x == 0) x[c] = xc;
        for (int i = threadIdx.x; i < c; i += blockDim.x) x[i] -= A[(long long)i * S + c] * xc;
        __syncthreads();
    }
}

// d <- A0^-1 F: LU with partial pivoting of A (a copy of A0), then kRefineSweeps sweeps of FP64
// iterative refinement r = F - A0 d, d += (LU)^-1 P r.  0, or -1 on a zero pivot column.
__device__ int dense_solve(const double *A0, double *A, int *piv, const double *F, double *d, double *r, int S,
                           Shared &sh)
{
    for (long long e = threadIdx.x; e < (long long)S * S; e += blockDim.x) A[e] = A0[e];
    for (int y = threadIdx.x; y < S; y += blockDim.x) d[y] = F[y];
    __syncthreads();
    if (lu_factor(A, piv, S, sh) != 0) return -1;
    lu_solve(A, piv, d, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nwarps();
    for (int sweep = 0; sweep < kRefineSweeps; ++sweep) {
        for (int i = warp; i < S; i += nw) {
            const double *Ai = A0 + (long long)i * S;
            double acc = 0.0;
            for (int j = lane; j < S; j += 32) acc += Ai[j] * d[j];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) r[i] = F[i] - acc;
        }
        __syncthreads();
        lu_solve(A, piv, r, S);
        for (int y = threadIdx.x; y < S; y += blockDim.x) d[y] += r[y];
        __syncthreads();
    }
    return 0;
}

__global__ void __launch_bounds__(1024, 1) k_parcel_iteration(Col c, ParcelArgs a, int mats_in_smem)
{
    __shared__ Shared sh;
    extern __shared__ double dyn[];
    const int S = c.S, L = c.L, R = c.R;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nwarps();
    const Policy &pol = a.pol;
    ParcelState *st = a.st;
    // vectors always in shared memory; the two S x S matrices there too when they fit
    double *x = dyn, *F = x + S, *d = F + S, *r = d + S;
    int *piv = (int *)(r + S);
    double *mats = (double *)(piv + ((S + 1) & ~1));
    double *A0 = mats_in_smem ? mats : a.A;
    double *A = mats_in_smem ? mats + (long long)S * S : a.A + (long long)S * S;
    for (long long i = tid; i < (long long)L * S; i += nt) a.Nold[i] = a.N[i];
    for (int y = tid; y < S; y += nt) a.vmr[y] = a.N[y] / c.ngas[0];
    if (tid == 0) sh.h = st->h;
    long long steps = 0, rejected = 0;
    __syncthreads();
    for (int v = 0; v < 2 * L - 1; ++v) {
        const int k = v < L ? v : 2 * L - 2 - v;
        const double nk = c.ngas[k], dzk = c.dz[k];
        const double tau = dzk * dzk / c.Kzz[k];
        for (int y = tid; y < S; y += nt) x[y] = a.vmr[y] * nk;
        if (tid == 0) sh.t = 0.0;
        __syncthreads();
        int visit_steps = 0;
        while (sh.t < tau) {
            if (tid == 0) {
                const double rest = tau - sh.t;
                double hs = sh.h < rest ? sh.h : rest;
                if (hs > pol.dt_max) hs = pol.dt_max;
                sh.hs = hs;
                sh.last = hs >= rest;
            }
            __syncthreads();
            const double hs = sh.hs;
            // reaction terms at the parcel's densities (Sec. 2.3)
            for (int rr = tid; rr < R; rr += nt) reaction_terms_at(c, k, rr, x, a.w + rr, a.dd + (long long)rr * 6);
            __syncthreads();
            // right-hand side: chemistry plus the molecular-diffusion pair
            for (int y = tid; y < S; y += nt) {
                double f = 0.0;
                for (int e = c.yp[y]; e < c.yp[y + 1]; ++e) {
                    const int code = c.yent[e];
                    if ((code & 15) - 8 < 0) f -= a.w[code >> 4];
                    else f += a.w[code >> 4];
                }
                double loss = 0.0, gain = 0.0;
                if (k + 1 < L) {
                    loss += a.um[(long long)k * S + y];
                    gain += a.vm[(long long)k * S + y] * a.N[(long long)(k + 1) * S + y];
                }
                if (k > 0) {
                    loss += a.vm[(long long)(k - 1) * S + y];
                    gain += a.um[(long long)(k - 1) * S + y] * a.N[(long long)(k - 1) * S + y];
                }
                F[y] = f + (gain - loss * x[y]) / dzk;
            }
            // matrix I/h - dF/dx: one warp per row, entries of the pattern summed in a fixed order
            for (int i = warp; i < S; i += nw) {
                double *Ar = A0 + (long long)i * S;
                for (int j = lane; j < S; j += 32) Ar[j] = 0.0;
                __syncwarp();
                for (int q = c.jp[i] + lane; q < c.jp[i + 1]; q += 32) Ar[c.jcol[q]] = jac_entry(c, q, a.dd);
                __syncwarp();
                if (lane == 0) {
                    double loss = 0.0;
                    if (k + 1 < L) loss += a.um[(long long)k * S + i];
                    if (k > 0) loss += a.vm[(long long)(k - 1) * S + i];
                    Ar[i] += 1.0 / hs + loss / dzk;
                }
            }
            __syncthreads();
            if (dense_solve(A0, A, piv, F, d, r, S, sh) != 0) {
                if (tid == 0) { st->status = XK_ESINGULAR; st->visit = v; }
                return;
            }
            // the Eulerian step controller: reject on a negative or a too large relative change
            double mr = 0.0;
            int bad = 0;
            for (int y = tid; y < S; y += nt) {
                const double xv = x[y], dv = d[y], nn = xv + dv;
                if (!isfinite(nn) || nn < -pol.neg_tol * nk) bad = 1;
                if (xv > pol.f_floor * nk) mr = fmax(mr, fabs(dv) / xv);
            }
            bad = block_or(bad, sh);
            mr = block_max(mr, sh);
            const int ok = !bad && !(mr > pol.rel_reject);
            if (ok)
                for (int y = tid; y < S; y += nt) {
                    const double nn = x[y] + d[y];
                    x[y] = nn < 0.0 ? 0.0 : nn;
                }
            __syncthreads();
            if (tid == 0) {
                if (ok) {
                    sh.t = sh.last ? tau : sh.t + hs;
                    double fac = mr > 0.0 ? pol.rel_target / mr : pol.grow_max;
                    if (fac > pol.grow_max) fac = pol.grow_max;
                    if (fac < pol.shrink_min) fac = pol.shrink_min;
                    double next = hs * fac;
                    if (hs < sh.h && fac >= 1.0 && next < sh.h) next = sh.h;   // cut short by the visit's end
                    sh.h = next;
                    sh.done = 0;
                } else {
                    sh.h = 0.5 * hs;
                    sh.done = sh.h < pol.dt_min ? XK_ENEG : 0;
                }
                if (++visit_steps > a.max_visit_steps && !sh.done) sh.done = XK_ENOCONV;
            }
            if (ok) ++steps;
            else ++rejected;
            __syncthreads();
            if (sh.done) {
                if (tid == 0) { st->status = sh.done; st->visit = v; st->steps += steps; st->rejected += rejected; }
                return;
            }
        }
        for (int y = tid; y < S; y += nt) {
            a.N[(long long)k * S + y] = x[y];
            a.vmr[y] = x[y] / nk;
        }
        __syncthreads();
    }
    double ch = 0.0;
    for (long long i = tid; i < (long long)L * S; i += nt) {
        const int k = (int)(i / S);
        const double nv = a.N[i];
        if (nv > pol.f_floor * c.ngas[k]) ch = fmax(ch, fabs(nv - a.Nold[i]) / nv);
    }
    ch = block_max(ch, sh);
    if (tid == 0) {
        st->max_change = ch;
        st->h = sh.h;
        st->steps += steps;
        st->rejected += rejected;
        st->status = 0;
    }
}

}  // namespace

size_t parcel_vector_bytes(int S) { return sizeof(double) * 4 * (size_t)S + sizeof(int) * (size_t)((S + 1) & ~1); }

bool parcel_mats_in_smem(int S)
{
    return parcel_vector_bytes(S) + 2 * sizeof(double) * (size_t)S * S <= kSmemLimit;
}

cudaError_t launch_parcel_iteration(const Col &c, const ParcelArgs &a, cudaStream_t st)
{
    const int S = c.S;
    const bool in_smem = parcel_mats_in_smem(S);
    const size_t smem = parcel_vector_bytes(S) + (in_smem ? 2 * sizeof(double) * (size_t)S * S : 0);
    // small systems: fewer warps, so that each barrier waits on less; large ones: the whole SM
    const int threads = S <= 160 ? 256 : 1024;
    cudaError_t e = cudaFuncSetAttribute(k_parcel_iteration, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_parcel_iteration<<<1, threads, smem, st>>>(c, a, in_smem ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace xk
