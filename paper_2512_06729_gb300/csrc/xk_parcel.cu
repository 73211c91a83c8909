// Lagrangian parcel scheme (Sec. 2, Fig. 1 and Fig. 2): one global iteration carries an air
// parcel from the bottom layer to the top and back (layers 0 .. L-1, then L-2 .. 0).  In layer k
// the parcel's densities x evolve for the eddy mixing time tau_k = dz_k^2 / K_zz,k under that
// layer's chemistry (Sec. 2.3) and molecular diffusion written as a pseudo-reaction pair with the
// stored densities of layers k -+ 1 (Sec. 2.1, after Eq. 4: the molecular part of Eq. 2's flux);
// eddy diffusion is the parcel's motion and has no term.  Within a visit: linearly implicit Euler
// steps (I/h - dF/dx) delta = F under the step controller of the Eulerian path, each solved by
// Gaussian elimination with partial pivoting.  The parcel keeps its mixing ratios from layer to
// layer, and each visit leaves its densities as the layer's.
//
// The sweep is sequential in the layers, so one CTA runs a whole iteration: every reduction,
// pivot search and elimination step stays inside the block (no grid-wide wait), and the only
// global traffic is the S x S matrix of the current step, which lives in L2.
#include <cfloat>

#include "xk_internal.cuh"

namespace xk {

namespace {

constexpr int kParcelThreads = 1024;
constexpr int kParcelWarps = kParcelThreads / 32;

struct Shared {
    double red[kParcelWarps];
    int ired[kParcelWarps];
    double h, t, hs;
    int last, done;
};

// max over the block; every thread gets the result
__device__ double block_max(double v, Shared &sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    v = lane < kParcelWarps ? sh.red[lane] : -DBL_MAX;
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
    v = lane < kParcelWarps ? sh.ired[lane] : 0;
    return __any_sync(0xffffffffu, v) ? 1 : 0;
}

// Row of the largest |A[i][c]|, i >= c (the first on ties, as a sequential scan picks it).
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
    best = lane < kParcelWarps ? sh.red[lane] : -1.0;
    bi = lane < kParcelWarps ? sh.ired[lane] : S;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    return best > 0.0 ? bi : -1;
}

// F <- A^-1 F by Gaussian elimination with partial pivoting (A is overwritten).  0, or -1 on a
// zero pivot column.
__device__ int dense_solve(double *A, double *F, int S, Shared &sh)
{
    for (int c = 0; c < S; ++c) {
        const int p = pivot_row(A, S, c, sh);
        if (p < 0) return -1;
        if (p != c) {
            for (int j = c + threadIdx.x; j < S; j += blockDim.x) {
                const double t = A[(long long)c * S + j];
                A[(long long)c * S + j] = A[(long long)p * S + j];
                A[(long long)p * S + j] = t;
            }
            if (threadIdx.x == 0) {
                const double t = F[c];
                F[c] = F[p];
                F[p] = t;
            }
        }
        __syncthreads();
        const double inv = 1.0 / A[(long long)c * S + c];
        const double fc = F[c];
        // multipliers first (column c is read by every row's update)
        for (int i = c + 1 + threadIdx.x; i < S; i += blockDim.x) {
            const double l = A[(long long)i * S + c] * inv;
            A[(long long)i * S + c] = l;
            F[i] -= l * fc;
        }
        __syncthreads();
        // trailing update: a warp per row, lanes along the row (coalesced)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = c + 1 + warp; i < S; i += kParcelWarps) {
            double *Ai = A + (long long)i * S;
            const double l = Ai[c];
            for (int j = c + 1 + lane; j < S; j += 32) Ai[j] -= l * A[(long long)c * S + j];
        }
        __syncthreads();
    }
    // back substitution, column by column
    for (int c = S - 1; c >= 0; --c) {
        const double xc = F[c] * (1.0 / A[(long long)c * S + c]);
        __syncthreads();
        if (threadIdx.x == 0) F[c] = xc;
        for (int i = threadIdx.x; i < c; i += blockDim.x) F[i] -= A[(long long)i * S + c] * xc;
        __syncthreads();
    }
    return 0;
}

__global__ void __launch_bounds__(kParcelThreads, 1) k_parcel_iteration(Col c, ParcelArgs a)
{
    __shared__ Shared sh;
    const int S = c.S, L = c.L, R = c.R;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const Policy &pol = a.pol;
    ParcelState *st = a.st;
    for (long long i = tid; i < (long long)L * S; i += nt) a.Nold[i] = a.N[i];
    for (int y = tid; y < S; y += nt) a.vmr[y] = a.N[y] / c.ngas[0];
    if (tid == 0) sh.h = st->h;
    long long steps = 0, rejected = 0;
    __syncthreads();
    for (int v = 0; v < 2 * L - 1; ++v) {
        const int k = v < L ? v : 2 * L - 2 - v;
        const double nk = c.ngas[k], dzk = c.dz[k];
        const double tau = dzk * dzk / c.Kzz[k];
        for (int y = tid; y < S; y += nt) a.x[y] = a.vmr[y] * nk;
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
            for (int r = tid; r < R; r += nt) reaction_terms_at(c, k, r, a.x, a.w + r, a.dd + (long long)r * 6);
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
                a.F[y] = f + (gain - loss * a.x[y]) / dzk;
            }
            // matrix I/h - dF/dx: one warp per row, entries of the pattern summed in a fixed order
            for (int i = warp; i < S; i += kParcelWarps) {
                double *Ar = a.A + (long long)i * S;
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
            if (dense_solve(a.A, a.F, S, sh) != 0) {
                if (tid == 0) { st->status = XK_ESINGULAR; st->visit = v; }
                return;
            }
            // the Eulerian step controller: reject on a negative or a too large relative change
            double mr = 0.0;
            int bad = 0;
            for (int y = tid; y < S; y += nt) {
                const double xv = a.x[y], d = a.F[y], nn = xv + d;
                if (!isfinite(nn) || nn < -pol.neg_tol * nk) bad = 1;
                if (xv > pol.f_floor * nk) mr = fmax(mr, fabs(d) / xv);
            }
            bad = block_or(bad, sh);
            mr = block_max(mr, sh);
            const int ok = !bad && !(mr > pol.rel_reject);
            if (ok)
                for (int y = tid; y < S; y += nt) {
                    const double nn = a.x[y] + a.F[y];
                    a.x[y] = nn < 0.0 ? 0.0 : nn;
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
            a.N[(long long)k * S + y] = a.x[y];
            a.vmr[y] = a.x[y] / nk;
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

void launch_parcel_iteration(const Col &c, const ParcelArgs &a, cudaStream_t st)
{
    count_launches(1);
    k_parcel_iteration<<<1, kParcelThreads, 0, st>>>(c, a);
}

}  // namespace xk
