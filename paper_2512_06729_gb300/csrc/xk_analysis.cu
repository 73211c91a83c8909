// Chemical-equilibrium initial state (Sec. 2.5, option (i)) and the reaction-pathway analyser
// (Sec. 4) on the GPU.
//
// Equilibrium: one CTA per layer finds the ideal-gas mixture of minimum Gibbs energy at the layer's
// T and P for given element totals.  The unknowns are ln N_y of every species, the total ln N and
// one potential pi_e per element; each Newton iteration reduces to an (E+1) x (E+1) system (the
// reduced Gibbs iteration of the NASA equilibrium program, Gordon & McBride 1994).  The species
// loop (exp, chemical potentials, the update) is spread over the CTA's threads, each of the
// system's sums over species is taken by one thread in species order, and one warp solves the
// small system with partial pivoting.  At convergence the mole fractions are rebuilt from the
// potentials, x_y = exp(sum_e pi_e a_ey - G_y/RT - ln P), so trace species keep full relative
// accuracy however small.
//
// Pathways: one warp per (source, layer) runs Dijkstra on the layer's reaction graph with edge
// weights 1/rate (the kinetically fastest route minimises the summed inverse rates).  The graph is
// the same in every layer (built on the host from the network); the weights come from that
// layer's forward and reverse rates.  Distances, the predecessor tree and each path's slowest step
// are kept in shared memory until the warp writes them out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "xk_internal.cuh"

namespace xk {
namespace {

constexpr int kEqThreads = 256;
constexpr int kEqMaxE = 31;              // E + 1 rows of the Newton system fit one warp
constexpr double kLnMajor = -18.420680743952367;   // ln 1e-8: species above this fraction are "major"
constexpr double kTraceCap = 9.2103;               // a trace species may rise to about 1e-4 of N per step

struct EqShared {
    double A[kEqMaxE + 1][kEqMaxE + 2];  // the (E+1) x (E+1) system with its right-hand side
    double sol[kEqMaxE + 1];
    double bk[kEqMaxE];
    double red[3][kEqThreads / 32];
    double lntot, bsum, sn, snm;
    int eact[kEqMaxE];
    int done, singular, nact;
};

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
    for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide reduction of three values (max, min, sum) with one barrier pair; every thread gets them.
__device__ void block_reduce3(EqShared &sh, double &mx, double &mn, double &sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    mx = warp_max(mx);
    mn = warp_min(mn);
    sm = warp_sum(sm);
    if (lane == 0) {
        sh.red[0][w] = mx;
        sh.red[1][w] = mn;
        sh.red[2][w] = sm;
    }
    __syncthreads();
    mx = -INFINITY;
    mn = INFINITY;
    sm = 0.0;
    for (int i = 0; i < nw; ++i) {   // same order in every thread: identical results everywhere
        mx = fmax(mx, sh.red[0][i]);
        mn = fmin(mn, sh.red[1][i]);
        sm += sh.red[2][i];
    }
    __syncthreads();
}

// Block-wide sums of two values, the same in every thread.
__device__ void block_sum2(EqShared &sh, double &a, double &b)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        sh.red[0][w] = a;
        sh.red[1][w] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int i = 0; i < nw; ++i) {
        a += sh.red[0][i];
        b += sh.red[1][i];
    }
    __syncthreads();
}

// Gaussian elimination with partial pivoting of the M x (M+1) augmented system on warp 0: lane r
// owns row r; the pivot is the first row of largest magnitude in the column.
__device__ void warp_solve(EqShared &sh, int M)
{
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < M; ++c) {
        double v = (lane >= c && lane < M) ? fabs(sh.A[lane][c]) : -1.0;
        int idx = lane;
        for (int o = 16; o; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) {
                v = ov;
                idx = oi;
            }
        }
        if (!(v > 0.0)) {
            if (lane == 0) sh.singular = 1;
            __syncwarp();
            return;
        }
        if (idx != c && lane <= M) {
            const double t = sh.A[c][lane];
            sh.A[c][lane] = sh.A[idx][lane];
            sh.A[idx][lane] = t;
        }
        __syncwarp();
        if (lane > c && lane < M) {
            const double l = sh.A[lane][c] / sh.A[c][c];
            for (int j = c; j <= M; ++j) sh.A[lane][j] -= l * sh.A[c][j];
        }
        __syncwarp();
    }
    if (lane == 0)
        for (int i = M - 1; i >= 0; --i) {
            double s = sh.A[i][M];
            for (int j = i + 1; j < M; ++j) s -= sh.A[i][j] * sh.sol[j];
            sh.sol[i] = s / sh.A[i][i];
        }
    __syncwarp();
}

// Dynamic shared memory: lnN, nj, mu [S] doubles, then the activity flags [S] as bytes.
__global__ void __launch_bounds__(kEqThreads) k_equilibrium(Col c, EqIndex ix, const double *b, double *x,
                                                             double *nout, int max_iter, double tol, int *iters,
                                                             int *status)
{
    __shared__ EqShared sh;
    extern __shared__ double eq_dyn[];
    const int S = c.S, E = c.E, M = c.E + 1, k = blockIdx.x, tid = threadIdx.x;
    double *lnN = eq_dyn, *nj = lnN + S, *mu = nj + S;
    unsigned char *act = (unsigned char *)(mu + S);
    const double *g = c.grt + (size_t)k * S;
    const double lnP = log(c.P[k]);

    if (tid < E) {
        double v = 0.0;
        if (b) v = b[(size_t)k * E + tid];
        else
            for (int y = 0; y < S; ++y) v += (double)c.elem[y * E + tid] * c.n[(size_t)k * S + y];
        sh.bk[tid] = v;
        sh.eact[tid] = v > 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int e = 0; e < E; ++e)
            if (sh.eact[e]) s += sh.bk[e];
        sh.bsum = s;
        sh.lntot = 0.0;
        sh.done = 0;
        sh.singular = 0;
    }
    int cnt = 0;
    for (int y = tid; y < S; y += blockDim.x) {
        int on = 1;
        for (int q = ix.sp[y]; q < ix.sp[y + 1]; ++q)
            if (!sh.eact[ix.se[q]]) on = 0;
        act[y] = (unsigned char)on;
        cnt += on;
    }
    double d0 = -INFINITY, d1 = INFINITY, d2 = cnt;
    block_reduce3(sh, d0, d1, d2);
    const int nact = (int)d2;
    if (nact == 0 || !(sh.bsum > 0.0)) {
        if (tid == 0) {
            iters[k] = 0;
            status[k] = -1;
        }
        return;
    }
    for (int y = tid; y < S; y += blockDim.x) lnN[y] = act[y] ? log(1.0 / nact) : 0.0;
    __syncthreads();

    int it = 0;
    for (; it < max_iter; ++it) {
        const double lntot = sh.lntot, ntot = exp(lntot);
        double sn = 0.0, snm = 0.0;
        for (int y = tid; y < S; y += blockDim.x) {
            if (act[y]) {
                nj[y] = exp(lnN[y]);
                mu[y] = g[y] + lnP + lnN[y] - lntot;
            } else {
                nj[y] = 0.0;
                mu[y] = 0.0;
            }
            sn += nj[y];
            snm += nj[y] * mu[y];
        }
        // the system starts from zero (pairs of elements no species shares stay zero)
        for (int t = tid; t < M * (M + 1); t += blockDim.x) sh.A[t / (M + 1)][t % (M + 1)] = 0.0;
        block_sum2(sh, sn, snm);
        // each entry's sparse sum over the species holding its elements, in species order
        for (int t = tid; t < ix.nent; t += blockDim.x) {
            const int code = ix.eij[t];
            double sv = 0.0, dv = 0.0;
            for (int q = ix.ep[t]; q < ix.ep[t + 1]; ++q) {
                const int y = ix.ey[q];
                const double v = ix.ec[q] * nj[y];
                sv += v;
                if (code < 0) dv += v * mu[y];
            }
            if (code >= 0) {
                const int i = code >> 5, j = code & 31;
                if (sh.eact[i] && sh.eact[j]) {
                    sh.A[i][j] = sv;
                    sh.A[j][i] = sv;
                }
            } else {
                const int i = -1 - code;
                if (sh.eact[i]) {
                    sh.A[i][E] = sv;
                    sh.A[E][i] = sv;
                    sh.A[i][M] = sh.bk[i] / sh.bsum - sv + dv;
                }
            }
        }
        if (tid == 0) {
            sh.A[E][E] = sn - ntot;
            sh.sn = sn;
            sh.snm = snm;
        }
        __syncthreads();
        if (tid < E && !sh.eact[tid]) sh.A[tid][tid] = 1.0;
        if (tid == 0) sh.A[E][M] = ntot - sh.sn + sh.snm;
        __syncthreads();
        if (tid < 32) warp_solve(sh, M);
        __syncthreads();
        if (sh.singular) break;
        const double dlntot = sh.sol[E];
        // step limit and convergence measure
        double big = 5.0 * fabs(dlntot), lam2 = 1.0, conv = 0.0;
        for (int y = tid; y < S; y += blockDim.x) {
            if (!act[y]) continue;
            double d = -mu[y] + dlntot;
            for (int q = ix.sp[y]; q < ix.sp[y + 1]; ++q) d += sh.sol[ix.se[q]] * ix.sc[q];
            mu[y] = d;
            const double lx = lnN[y] - lntot;
            if (lx > kLnMajor) big = fmax(big, fabs(d));
            else if (d - dlntot > 0.0) lam2 = fmin(lam2, fabs((-lx - kTraceCap) / (d - dlntot)));
            conv += nj[y] * fabs(d);
        }
        block_reduce3(sh, big, lam2, conv);
        conv /= sh.sn;
        double lam = big > 2.0 ? 2.0 / big : 1.0;
        lam = fmin(lam, lam2);
        for (int y = tid; y < S; y += blockDim.x)
            if (act[y]) lnN[y] += lam * mu[y];
        __syncthreads();
        if (tid == 0) sh.lntot = lntot + lam * dlntot;
        if (conv < tol && fabs(dlntot) < tol) {
            ++it;
            sh.done = 1;   // same decision in every thread (block-reduced values)
            break;
        }
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
        iters[k] = it;
        status[k] = sh.singular ? -1 : (sh.done ? 0 : 1);
    }
    if (sh.singular) return;
    // mole fractions from the potentials of the last solve, normalised
    double amax = -INFINITY;
    for (int y = tid; y < S; y += blockDim.x) {
        if (!act[y]) continue;
        double v = -g[y] - lnP;
        for (int q = ix.sp[y]; q < ix.sp[y + 1]; ++q) v += sh.sol[ix.se[q]] * ix.sc[q];
        mu[y] = v;
        amax = fmax(amax, v);
    }
    double dummy = INFINITY, zero = 0.0;
    block_reduce3(sh, amax, dummy, zero);
    double z = 0.0;
    for (int y = tid; y < S; y += blockDim.x)
        if (act[y]) z += exp(mu[y] - amax);
    double mx2 = -INFINITY, mn2 = INFINITY;
    block_reduce3(sh, mx2, mn2, z);
    const double lz = log(z);
    const double ng = c.ngas[k];
    for (int y = tid; y < S; y += blockDim.x) {
        const double v = act[y] ? exp(mu[y] - amax - lz) : 0.0;
        if (x) x[(size_t)k * S + y] = v;
        if (nout) nout[(size_t)k * S + y] = v * ng;
    }
}

__global__ void k_fluxes(Col c, const double *n, double *q)
{
    const long long total = (long long)c.L * c.R;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / c.R), r = (int)(i % c.R);
        const double *nk = n + (size_t)k * c.S;
        double wf, wb;
        if (c.rtype[r] == XK_RX_PHOTO) {
            wf = c.kph[(size_t)k * c.Rph + c.prow[r]];
            wb = 0.0;
        } else {
            wf = c.kf[i];
            wb = c.kr[i];
        }
        for (int s = 0; s < 3; ++s) {
            const int a = c.reac[3 * r + s], p = c.prod[3 * r + s];
            if (a >= 0) wf *= nk[a];
            if (p >= 0) wb *= nk[p];
        }
        q[2 * i] = wf;
        q[2 * i + 1] = wb;
    }
}

// Edge weight of every reaction direction in every layer: 1/q for q > 0, +inf otherwise (no edge).
// Computed once per layer and shared by every source's search.
__global__ void k_path_weights(long long n, const double *q, double *wq)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double r = q[i];
        wq[i] = r > 0.0 ? 1.0 / r : INFINITY;
    }
}

// Distances are non-negative doubles (or +inf): their bit patterns order like the values, so the
// search compares them on the integer pipes (FP64 compares are scarce on this GPU).
__device__ __forceinline__ unsigned long long key_of(double d) { return (unsigned long long)__double_as_longlong(d); }

// Per-warp shared memory of the pathway search: dist [S] doubles, then pred_sp, pred_e, order [S]
// ints and done [S] bytes.
__host__ __device__ inline size_t path_warp_bytes(int S)
{
    return ((size_t)S * (8 + 4 + 4 + 4 + 1) + 15) / 16 * 16;
}

__global__ void k_pathways(Col c, PathGraph gr, const double *wq, int nsrc, const int *src, int wpb,
                           double *dist_out, int *pred_out, int *edge_out, int *lim_out, double *limw_out)
{
    extern __shared__ double path_dyn[];
    const int S = c.S, L = c.L, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long prob = (long long)blockIdx.x * wpb + w;
    if (w >= wpb || prob >= (long long)nsrc * L) return;
    const int j = (int)(prob / L), k = (int)(prob % L);
    const int s0 = src[j];
    char *base = (char *)path_dyn + path_warp_bytes(S) * w;
    double *dist = (double *)base;
    int *pred = (int *)(dist + S), *pe = pred + S, *order = pe + S;
    unsigned char *done = (unsigned char *)(order + S);
    const double *wk = wq + (size_t)k * c.R * 2;
    for (int y = lane; y < S; y += 32) {
        dist[y] = INFINITY;
        pred[y] = -1;
        pe[y] = -1;
        done[y] = 0;
    }
    __syncwarp();
    if (lane == 0) dist[s0] = 0.0;
    __syncwarp();
    int nord = 0;
    for (;;) {
        // the unfinished species of least distance, the lower index on ties
        const unsigned long long kinf = key_of(INFINITY);
        unsigned long long bd = kinf;
        int bi = S;
        for (int y = lane; y < S; y += 32) {
            const unsigned long long ky = key_of(dist[y]);
            if (!done[y] && ky < bd) {
                bd = ky;
                bi = y;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (od < bd || (od == bd && oi < bi)) {
                bd = od;
                bi = oi;
            }
        }
        if (!(bd < kinf)) break;
        const int u = bi;
        if (lane == 0) {
            done[u] = 1;
            order[nord] = u;
        }
        ++nord;
        __syncwarp();
        // relax: one lane per target species, its parallel edges in increasing code, strict decrease
        const double du = dist[u];
        for (int g = gr.gp[u] + lane; g < gr.gp[u + 1]; g += 32) {
            const int v = gr.gv[g];
            double best = dist[v];
            unsigned long long kb = key_of(best);
            int be = -1;
            for (int t = gr.gs[g]; t < gr.gs[g + 1]; ++t) {
                const int e = gr.gcode[t];
                const double cand = du + wk[e];   // +inf for a direction without rate
                const unsigned long long kc = key_of(cand);
                if (kc < kb) {
                    kb = kc;
                    best = cand;
                    be = e;
                }
            }
            if (be >= 0) {
                dist[v] = best;
                pred[v] = u;
                pe[v] = be;
            }
        }
        __syncwarp();
    }
    const size_t o = ((size_t)j * L + k) * S;
    for (int y = lane; y < S; y += 32) {
        if (dist_out) dist_out[o + y] = dist[y];
        if (pred_out) pred_out[o + y] = pred[y];
        if (edge_out) edge_out[o + y] = pe[y];
        if (lim_out) {
            lim_out[o + y] = -1;
            limw_out[o + y] = 0.0;
        }
    }
    __syncwarp();
    // slowest step of each path, in the order the species were finished
    if (lim_out && lane == 0)
        for (int i = 0; i < nord; ++i) {
            const int v = order[i], u = pred[v];
            if (u < 0) continue;
            const int e = pe[v];
            const double wv = wk[e];
            if (u == s0 || wv > limw_out[o + u]) {
                lim_out[o + v] = e;
                limw_out[o + v] = wv;
            } else {
                lim_out[o + v] = lim_out[o + u];
                limw_out[o + v] = limw_out[o + u];
            }
        }
}

}  // namespace

cudaError_t launch_equilibrium(const Col &c, const EqIndex &ix, const double *b, double *x, double *nout,
                               int max_iter, double tol, int *iters, int *status, cudaStream_t st)
{
    if (c.E + 1 > kEqMaxE) return cudaErrorInvalidValue;
    const size_t smem = (size_t)c.S * 3 * sizeof(double) + (size_t)c.S;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_equilibrium, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_equilibrium<<<c.L, kEqThreads, smem, st>>>(c, ix, b, x, nout, max_iter, tol, iters, status);
    count_launches(1);
    return cudaGetLastError();
}

void launch_fluxes(const Col &c, const double *n, double *q, cudaStream_t st)
{
    const long long total = (long long)c.L * c.R;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
    k_fluxes<<<std::max(blocks, 1), 256, 0, st>>>(c, n, q);
    count_launches(1);
}

cudaError_t launch_pathways(const Col &c, const PathGraph &g, const double *q, double *wbuf, int nsrc,
                            const int *src, double *dist, int *pred_sp, int *pred_edge, int *lim_edge,
                            double *lim_w, cudaStream_t st)
{
    const long long nw = (long long)c.L * c.R * 2;
    if (nw > 0) {
        k_path_weights<<<(int)std::min<long long>((nw + 255) / 256, 152LL * 8), 256, 0, st>>>(nw, q, wbuf);
        count_launches(1);
    }
    const size_t per = path_warp_bytes(c.S);
    const size_t cap = 96 * 1024;
    if (per > 200 * 1024) return cudaErrorInvalidValue;
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, cap / per));
    const size_t smem = per * wpb;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pathways, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long probs = (long long)nsrc * c.L;
    const int blocks = (int)((probs + wpb - 1) / wpb);
    k_pathways<<<blocks, 32 * wpb, smem, st>>>(c, g, wbuf, nsrc, src, wpb, dist, pred_sp, pred_edge, lim_edge,
                                              lim_w);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace xk
