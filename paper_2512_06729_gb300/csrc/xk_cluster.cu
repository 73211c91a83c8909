// FP32 block inversions of the block-Thomas elimination on one thread-block
// cluster, with every layer's block resident in the cluster's distributed
// shared memory.
//
// The grid-wide kernels in xk_factor.cu keep the block in global memory and
// pay two grid barriers and several L2 round trips per panel; on a 594-species
// block that is ~40 us per panel for ~0.1 us of arithmetic per SM.  Here the
// S x S block of one layer is split by panels of NB rows over the C CTAs of one
// cluster (panel p on CTA p mod C) and stays in shared memory from the Schur
// update to the stored inverse.  Gauss-Jordan elimination without pivoting
// then needs, per panel, only the owner's NB new rows
//   U = D_pp^-1 [D_p,*]   (with the panel columns replaced by D_pp^-1),
// and one hardware cluster barrier (~0.2 us).  The owner publishes U through
// a two-slot buffer in global memory, read by every CTA from L2: reading it
// from the owner's shared memory instead serializes on that one SM
// (38 KB x 12 CTAs took ~10 us per panel, against ~1.7 us from L2).  Every
// other row r is updated locally:
//   D[r][j] <- (j in panel ? 0 : D[r][j]) - sum_l D[r][c0 + l] U[l][j].
// The Schur update of the next layer, D'_k = A_k - diag(lo_k) D'^-1_{k-1}
// diag(up_{k-1}), uses the same rows of the previous inverse, so it is local
// too.  Global memory sees one read of A_k and one write of the inverse per
// layer.
//
// As in k_factor_np there is no pivoting: this inverse preconditions the FP64
// FGMRES iteration on the exact operator, which (with the pivoted FP64
// factorization behind it) guarantees the solution.  A zero diagonal pivot sets
// err_singular and continues with a zero reciprocal; no thread leaves the
// layer loop early, so every cluster barrier is reached by all CTAs.
#include <cooperative_groups.h>

#include "xk_internal.cuh"

namespace xk {
namespace {

namespace cg = cooperative_groups;

constexpr int kClusterMaxThreads = 512;
constexpr int kClusterMaxSize = 16;

// Invert the NB x NB diagonal block of panel rows R (lds-strided, columns
// c0 .. c0 + nb) with one warp: lane j < NB holds column j in registers; rows
// and columns at or above nb are treated as identity.  Result into Bs
// (NB x (NB + 1)).
template <int NB>
__device__ __forceinline__ void diag_inverse_regs(const float *R, int lds, int c0, int nb, float *Bs, Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    const int j = lane < NB ? lane : NB - 1;
    float b[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r)
        b[r] = (r < nb && j < nb) ? R[(size_t)r * lds + c0 + j] : (r == j ? 1.f : 0.f);
    bool singular = false;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        const float d = __shfl_sync(0xffffffffu, b[c], c);
        singular |= (d == 0.f);
        const float inv = (d != 0.f) ? 1.f / d : 0.f;
        const float rowc = (j == c) ? inv : b[c] * inv;       // new row c, column j
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            if (r == c) continue;
            const float f = __shfl_sync(0xffffffffu, b[r], c);   // old B[r][c]
            b[r] = (j == c) ? -f * inv : fmaf(-f, rowc, b[r]);
        }
        b[c] = rowc;
    }
    if (lane < NB) {
#pragma unroll
        for (int r = 0; r < NB; ++r) Bs[r * (NB + 1) + lane] = b[r];
    }
    if (singular && lane == 0) atomicExch(&ctl->err_singular, 1);
    __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(kClusterMaxThreads, 1)
k_factor_cluster(BlockSys<float> a, float *gU, Ctl *ctl, const int *skip, int nslot, int lds, int mode, int mid)
{
    // the flags are written by earlier kernels on the stream: every CTA of the
    // cluster takes the same branch
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int me = (int)cl.block_rank();
    extern __shared__ __align__(16) float sm[];
    const int nloc = nslot * NB;                  // local rows (some may not exist)
    float *Dl = sm;                               // nloc x lds: this CTA's rows of the block
    float *Ub = Dl + (size_t)nloc * lds;          // NB x lds: U of the panel this CTA owns (gU: 2 x NB x lds)
    float *Gs = Ub + (size_t)NB * lds;            // nloc x NB: panel columns before the update
    float *Bs = Gs + (size_t)nloc * NB;           // NB x (NB + 1): diagonal-block inverse

    const int S = a.S, ld = a.ld, L = a.L;
    const int Q = lds / 4;                        // column quads of a row
    const int T = blockDim.x / Q;                 // row teams; thread = (team, quad)
    const int tid = threadIdx.x;
    const int team = tid / Q, q = tid - team * Q;
    const bool active = team < T;
    const int npan = (S + NB - 1) / NB;
    auto grow = [&](int lr) -> int {              // global row of local row lr, or -1
        const int p = (lr / NB) * C + me;
        const int r = p * NB + (lr % NB);
        return (p < npan && r < S) ? r : -1;
    };

    // layers this cluster factors: mode 0 all, top-down; mode 1 (two clusters, the twisted
    // elimination) cluster 0 top-down to mid - 1 and cluster 1 bottom-up to mid + 1, with
    // E'_k = A_k - diag(up_k) E'^-1_{k+1} diag(lo_{k+1}); mode 2 the middle layer alone,
    // D'_mid = A_mid - diag(lo) D'^-1_{mid-1} diag(up_{mid-1}) - diag(up) E'^-1_{mid+1} diag(lo_{mid+1})
    const int cq = blockIdx.x / C;
    int nsteps = L, k0 = 0, dk = 1;
    if (mode == 1) {
        nsteps = cq == 0 ? mid : L - 1 - mid;
        k0 = cq == 0 ? 0 : L - 1;
        dk = cq == 0 ? 1 : -1;
    } else if (mode == 2) {
        nsteps = 1;
        k0 = mid;
        dk = 0;
    }
    gU += (size_t)cq * 2 * NB * lds;
    for (int step = 0; step < nsteps; ++step) {
        const int k = k0 + step * dk;
        float *D = a.D + (size_t)k * S * ld;
        // rows of A_k minus the Schur terms of the neighbour(s) already inverted
        {
            const float *cl = nullptr, *cr = nullptr;          // chain: previous inverse, in place
            if (mode != 2 && step > 0) {
                cl = dk > 0 ? a.lo + (size_t)k * S : a.up + (size_t)k * S;
                cr = dk > 0 ? a.up + (size_t)(k - 1) * S : a.lo + (size_t)(k + 1) * S;
            }
            const float *Bd = (mode == 2 && k > 0) ? a.D + (size_t)(k - 1) * S * ld : nullptr;
            const float *Bu = (mode == 2 && k + 1 < L) ? a.D + (size_t)(k + 1) * S * ld : nullptr;
            for (int e = tid; e < nloc * Q; e += blockDim.x) {
                const int lr = e / Q, qq = e - lr * Q;
                const int r = grow(lr);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r >= 0) {
                    const int j0 = qq * 4;
                    const float *src = D + (size_t)r * ld + j0;
                    float4 x = *reinterpret_cast<const float4 *>(src);
                    float w[4] = {x.x, x.y, x.z, x.w};
                    const float *prev = Dl + (size_t)lr * lds + j0;
                    float4 bd = make_float4(0.f, 0.f, 0.f, 0.f), bu = bd;
                    if (Bd) bd = *reinterpret_cast<const float4 *>(Bd + (size_t)r * ld + j0);
                    if (Bu) bu = *reinterpret_cast<const float4 *>(Bu + (size_t)r * ld + j0);
                    const float bdv[4] = {bd.x, bd.y, bd.z, bd.w}, buv[4] = {bu.x, bu.y, bu.z, bu.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = j0 + t;
                        if (j >= S) {
                            w[t] = 0.f;
                            continue;
                        }
                        if (cl) w[t] -= cl[r] * prev[t] * cr[j];
                        if (Bd) w[t] -= a.lo[(size_t)k * S + r] * bdv[t] * a.up[(size_t)(k - 1) * S + j];
                        if (Bu) w[t] -= a.up[(size_t)k * S + r] * buv[t] * a.lo[(size_t)(k + 1) * S + j];
                    }
                    v = make_float4(w[0], w[1], w[2], w[3]);
                }
                *reinterpret_cast<float4 *>(Dl + (size_t)lr * lds + qq * 4) = v;
            }
            for (int i = me * blockDim.x + tid; i < S; i += C * blockDim.x) {
                a.perm[(size_t)k * S + i] = i;
                a.iperm[(size_t)k * S + i] = i;
            }
        }
        __syncthreads();

        for (int p = 0; p < npan; ++p) {
            const int owner = p % C, slot = p / C;
            const int c0 = p * NB, nb = min(NB, S - c0);
            const int cq0 = c0 / 4;                       // first quad of the panel (c0 is a multiple of 4)
            if (me == owner) {
                const float *R = Dl + (size_t)slot * NB * lds;
                if (tid < 32) diag_inverse_regs<NB>(R, lds, c0, nb, Bs, ctl);
                __syncthreads();
                // U[l][j] = sum_m Dinv[l][m] D[c0 + m][j]; panel columns take Dinv itself
                for (int e = tid; e < NB * Q; e += blockDim.x) {
                    const int l = e / Q, qq = e - l * Q;
                    float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (l < nb) {
                        if (qq >= cq0 && qq < cq0 + NB / 4) {
                            float w[4];
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int jj = qq * 4 + t - c0;
                                w[t] = jj < nb ? Bs[l * (NB + 1) + jj] : 0.f;
                            }
                            u = make_float4(w[0], w[1], w[2], w[3]);
                        } else {
#pragma unroll 4
                            for (int m = 0; m < nb; ++m) {
                                const float dlm = Bs[l * (NB + 1) + m];
                                const float4 x = *reinterpret_cast<const float4 *>(R + (size_t)m * lds + qq * 4);
                                u.x = fmaf(dlm, x.x, u.x);
                                u.y = fmaf(dlm, x.y, u.y);
                                u.z = fmaf(dlm, x.z, u.z);
                                u.w = fmaf(dlm, x.w, u.w);
                            }
                        }
                    }
                    *reinterpret_cast<float4 *>(Ub + (size_t)l * lds + qq * 4) = u;
                    *reinterpret_cast<float4 *>(gU + ((size_t)(p & 1) * NB + l) * lds + qq * 4) = u;
                }
            }
            // U of panel p is complete in global memory (the barrier releases and acquires at
            // cluster scope; the slot of panel p + 2 is written only after every CTA has passed
            // the barrier of panel p + 1, i.e. has read this one)
            cl.sync();

            float4 u[NB];
            if (active) {
                const float4 *Ug = reinterpret_cast<const float4 *>(gU + (size_t)(p & 1) * NB * lds) + q;
#pragma unroll
                for (int l = 0; l < NB; ++l) u[l] = __ldcg(Ug + (size_t)l * (lds / 4));
            }
            for (int e = tid; e < nloc * NB; e += blockDim.x) {
                const int lr = e / NB, l = e - lr * NB;
                Gs[e] = (l < nb) ? Dl[(size_t)lr * lds + c0 + l] : 0.f;
            }
            __syncthreads();
            if (active) {
                const bool pq = (q >= cq0 && q < cq0 + NB / 4);
                for (int lr = team; lr < nloc; lr += T) {
                    if (grow(lr) < 0) continue;
                    if (me == owner && lr / NB == slot) continue;   // the panel rows become U
                    float4 *dst = reinterpret_cast<float4 *>(Dl + (size_t)lr * lds) + q;
                    float4 v = pq ? make_float4(0.f, 0.f, 0.f, 0.f) : *dst;
                    const float4 *g4 = reinterpret_cast<const float4 *>(Gs + (size_t)lr * NB);
#pragma unroll
                    for (int l4 = 0; l4 < NB / 4; ++l4) {
                        const float4 g = g4[l4];
                        const float gg[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const float4 uu = u[l4 * 4 + t];
                            v.x = fmaf(-gg[t], uu.x, v.x);
                            v.y = fmaf(-gg[t], uu.y, v.y);
                            v.z = fmaf(-gg[t], uu.z, v.z);
                            v.w = fmaf(-gg[t], uu.w, v.w);
                        }
                    }
                    *dst = v;
                }
            }
            if (me == owner) {
                float *R = Dl + (size_t)slot * NB * lds;
                for (int e = tid; e < nb * Q; e += blockDim.x) {
                    const int l = e / Q, qq = e - l * Q;
                    *reinterpret_cast<float4 *>(R + (size_t)l * lds + qq * 4) =
                        *reinterpret_cast<const float4 *>(Ub + (size_t)l * lds + qq * 4);
                }
            }
            __syncthreads();
        }

        // store the inverse for the solve sweeps (it stays in shared memory for the next Schur update)
        for (int e = tid; e < nloc * Q; e += blockDim.x) {
            const int lr = e / Q, qq = e - lr * Q;
            const int r = grow(lr);
            if (r < 0) continue;
            *reinterpret_cast<float4 *>(D + (size_t)r * ld + qq * 4) =
                *reinterpret_cast<const float4 *>(Dl + (size_t)lr * lds + qq * 4);
        }
        // no CTA rewrites its U buffer (next layer) or exits while another may still read it
        cl.sync();
    }
}


// ---------------------------------------------------------------------------
// Forward and back sweeps with the stored inverses on one cluster:
//   g_0 = b_0;  g_k = b_k - lo_k * (D'^-1_{k-1} g_{k-1})
//   x_{L-1} = D'^-1_{L-1} g_{L-1};  x_k = D'^-1_k (g_k - up_k * x_{k+1})
// With implicit pivoting (perm != null) D'^-1_k[i][j] = B_k[perm(i)][iperm(j)],
// so (D'^-1_k v)[i] = sum_b B_k[perm(i)][b] v[perm(b)]; without it B_k is the
// inverse.  CTA c owns output rows [c*rpc, (c+1)*rpc) of every product.  The
// B rows a CTA needs next are copied into shared memory (cp.async) while the
// current layer finishes: with two buffers before its products, with one
// right after them, overlapping the cluster barrier and the exchange.  The new
// vector's rows go through distributed shared memory, one cluster barrier per
// layer and sweep.  Vectors are FP64 in global memory and rounded to T for the
// products, as in the grid-wide solve.
// ---------------------------------------------------------------------------
constexpr int kSolveClusterThreads = 512;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(kSolveClusterThreads, 1)
k_solve_cluster(BlockSys<T> a, const int *perm, const double *b, double *x, double *g, Ctl *ctl,
                const double *bscale, const int *skip, const double *xscale, int rpc, int lds, int nbuf)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    const int S = a.S, ld = a.ld, L = a.L;
    const int r0 = me * rpc, r1 = min(S, r0 + rpc), nr = max(0, r1 - r0);
    constexpr int E = 16 / sizeof(T);                   // elements per 16-byte copy
    const int Q = lds / E;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *buf = (T *)smraw;                                // nbuf x rpc x lds: B rows
    T *vec = buf + (size_t)nbuf * rpc * lds;            // lds: the vector the products take
    double *mine = (double *)(vec + lds);               // 2 x rpc: this CTA's rows of the newest vector

    // matrices in order of use: forward layers 1..L-1 take B_0..B_{L-2}, back layers L-1..0 take B_{L-1}..B_0
    const int nuse = 2 * L - 1;
    auto use_layer = [&](int t) -> int { return t < L - 1 ? t : 2 * L - 2 - t; };
    auto stage = [&](int t) {
        if (t < nuse) {
            const int layer = use_layer(t);
            const T *B = a.D + (size_t)layer * S * ld;
            const int *pk = perm ? perm + (size_t)layer * S : nullptr;
            T *dst = buf + (size_t)(t % nbuf) * rpc * lds;
            for (int e = tid; e < nr * Q; e += blockDim.x) {
                const int i = e / Q, qq = e - i * Q;
                const int row = pk ? pk[r0 + i] : r0 + i;
                cp_async16(dst + (size_t)i * lds + qq * E, B + (size_t)row * ld + qq * E);
            }
        }
        cp_async_commit();
    };
    // wait for use t (issued earlier), then clear the padding columns that were copied with it
    auto ready = [&](int t) {
        if (nbuf == 2) cp_async_wait1(); else cp_async_wait0();
        __syncthreads();
        T *Bt = buf + (size_t)(t % nbuf) * rpc * lds;
        if (lds > S)
            for (int e = tid; e < nr * (lds - S); e += blockDim.x) {
                const int i = e / (lds - S), j = S + (e - i * (lds - S));
                Bt[(size_t)i * lds + j] = (T)0;
            }
        __syncthreads();
    };
    auto rowdot = [&](const T *Bi) -> T {
        T acc = (T)0;
        for (int j = lane; j < S; j += 32) acc = fma(Bi[j], vec[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        return acc;
    };
    // vec[m] = the newest vector's entry perm(m) (or m), taken from its owner's slot
    auto gather = [&](int slot, int layer) {
        const int *pk = perm ? perm + (size_t)layer * S : nullptr;
        for (int m = tid; m < lds; m += blockDim.x) {
            T v = (T)0;
            if (m < S) {
                const int src_row = pk ? pk[m] : m;
                const int o = src_row / rpc;
                const double *src = cl.map_shared_rank(mine, o);
                v = (T)src[(size_t)slot * rpc + (src_row - o * rpc)];
            }
            vec[m] = v;
        }
    };

    int t = 0;                      // next use
    stage(0);
    if (nbuf == 2) stage(1);
    // forward sweep
    for (int k = 0; k < L; ++k) {
        const int slot = k & 1;
        if (k == 0) {
            for (int i = tid; i < nr; i += blockDim.x) {
                const int r = r0 + i;
                const double gi = bscale ? b[r] * bscale[r] : b[r];
                g[r] = gi;
                mine[(size_t)slot * rpc + i] = gi;
            }
        } else {
            ready(t);
            const T *Bk = buf + (size_t)(t % nbuf) * rpc * lds;
            for (int i = warp; i < nr; i += nw) {
                const T acc = rowdot(Bk + (size_t)i * lds);
                if (lane == 0) {
                    const size_t e = (size_t)k * S + r0 + i;
                    double bi = b[e];
                    if (bscale) bi *= bscale[e];
                    const double gi = bi - (double)a.lo[e] * (double)acc;
                    g[e] = gi;
                    mine[(size_t)slot * rpc + i] = gi;
                }
            }
            __syncthreads();                  // buffer t % nbuf is free again
            stage(t + nbuf);
            ++t;
        }
        cl.sync();
        if (k + 1 < L) {                      // the last forward vector is never read back through mine
            gather(slot, k);
            __syncthreads();
        }
    }
    // back sweep
    for (int k = L - 1; k >= 0; --k) {
        const int slot = k & 1;
        // h = g_k - up_k * x_{k+1}; x_{k+1}'s rows come from their owners, entry perm(m) into vec[m]
        const int *pk = perm ? perm + (size_t)k * S : nullptr;
        for (int m = tid; m < lds; m += blockDim.x) {
            T v = (T)0;
            if (m < S) {
                const int o_row = pk ? pk[m] : m;
                double h = g[(size_t)k * S + o_row];
                if (k + 1 < L) {
                    const int o = o_row / rpc;
                    const double *src = cl.map_shared_rank(mine, o);
                    h -= (double)a.up[(size_t)k * S + o_row] * src[(size_t)((k + 1) & 1) * rpc + (o_row - o * rpc)];
                }
                v = (T)h;
            }
            vec[m] = v;
        }
        ready(t);          // includes the block barrier that publishes vec
        const T *Bk = buf + (size_t)(t % nbuf) * rpc * lds;
        // (the slot written below was last read remotely before the previous cluster barrier)
        for (int i = warp; i < nr; i += nw) {
            const T acc = rowdot(Bk + (size_t)i * lds);
            if (lane == 0) {
                x[(size_t)k * S + r0 + i] = (double)acc;
                mine[(size_t)slot * rpc + i] = (double)acc;
            }
        }
        __syncthreads();
        stage(t + nbuf);
        ++t;
        cl.sync();
    }
    cp_async_wait0();
    if (xscale) {
        for (int k = 0; k < L; ++k)
            for (int i = tid; i < nr; i += blockDim.x) x[(size_t)k * S + r0 + i] *= xscale[(size_t)k * S + r0 + i];
    }
}

// Sweeps after the twisted elimination, on two clusters.
// phase 0 (forward, both ends at once):
//   cluster 0: g_0 = b_0, g_k = b_k - lo_k (B_{k-1} g_{k-1}) for 0 < k < mid, y_top = B_{mid-1} g_{mid-1}
//   cluster 1: h_{L-1} = b_{L-1}, h_k = b_k - up_k (C_{k+1} h_{k+1}) for mid < k < L-1,
//              y_bot = C_{mid+1} h_{mid+1}
// phase 1 (back, from the middle outwards):
//   both:      x_mid = B_mid (b_mid - lo_mid y_top - up_mid y_bot)
//   cluster 0: x_k = B_k (g_k - up_k x_{k+1}) for k < mid
//   cluster 1: x_k = C_k (h_k - lo_k x_{k-1}) for k > mid
// (B: inverses from the top, C: from the bottom, both stored in place of the blocks; g and h share
// the vector g; y_top and y_bot go through ymid.)  With implicit pivots (perm != null) a product
// with layer k's stored block reads rows perm_k(i) and takes the vector in the order perm_k, as in
// k_solve_cluster.  Prefetch and exchange as there.
template <typename T>
__global__ void __launch_bounds__(kSolveClusterThreads, 1)
k_solve_twisted(BlockSys<T> a, const int *perm, const double *b, double *x, double *g, double *ymid, Ctl *ctl,
                const double *bscale, const int *skip, const double *xscale, int rpc, int lds, int nbuf, int phase,
                int mid)
{
    if (ctl->finished || ctl->err_timeout || (skip && *skip)) return;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int me = (int)cl.block_rank();
    const int cq = blockIdx.x / C;
    const int S = a.S, ld = a.ld, L = a.L;
    const int r0 = me * rpc, r1 = min(S, r0 + rpc), nr = max(0, r1 - r0);
    constexpr int E = 16 / sizeof(T);
    const int Q = lds / E;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *buf = (T *)smraw;                                // nbuf x rpc x lds
    T *vec = buf + (size_t)nbuf * rpc * lds;            // lds
    double *mine = (double *)(vec + lds);               // 2 x rpc
    const int dk = cq == 0 ? 1 : -1;
    const int nuse = phase == 0 ? (cq == 0 ? mid : L - 1 - mid) : (cq == 0 ? mid + 1 : L - mid);
    auto use_layer = [&](int t) -> int {
        if (phase == 0) return cq == 0 ? t : L - 1 - t;
        return cq == 0 ? mid - t : mid + t;
    };
    auto pk = [&](int layer, int m) -> int { return perm ? perm[(size_t)layer * S + m] : m; };
    auto stage = [&](int t) {
        if (t < nuse) {
            const int layer = use_layer(t);
            const T *B = a.D + (size_t)layer * S * ld;
            T *dst = buf + (size_t)(t % nbuf) * rpc * lds;
            for (int e = tid; e < nr * Q; e += blockDim.x) {
                const int i = e / Q, qq = e - i * Q;
                cp_async16(dst + (size_t)i * lds + qq * E, B + (size_t)pk(layer, r0 + i) * ld + qq * E);
            }
        }
        cp_async_commit();
    };
    auto ready = [&](int t) {
        if (nbuf == 2) cp_async_wait1(); else cp_async_wait0();
        __syncthreads();
        T *Bt = buf + (size_t)(t % nbuf) * rpc * lds;
        if (lds > S)
            for (int e = tid; e < nr * (lds - S); e += blockDim.x) {
                const int i = e / (lds - S), j = S + (e - i * (lds - S));
                Bt[(size_t)i * lds + j] = (T)0;
            }
        __syncthreads();
    };
    auto rowdot = [&](const T *Bi) -> T {
        T acc = (T)0;
        for (int j = lane; j < S; j += 32) acc = fma(Bi[j], vec[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        return acc;
    };
    auto remote = [&](int slot, int row) -> double {
        const int o = row / rpc;
        const double *src = cl.map_shared_rank(mine, o);
        return src[(size_t)slot * rpc + (row - o * rpc)];
    };
    auto bval = [&](int k, int r) -> double {
        const size_t e = (size_t)k * S + r;
        return bscale ? b[e] * bscale[e] : b[e];
    };

    stage(0);
    if (nbuf == 2) stage(1);
    if (phase == 0) {
        const int ks = cq == 0 ? 0 : L - 1;
        for (int i = tid; i < nr; i += blockDim.x) {
            const double gi = bval(ks, r0 + i);
            g[(size_t)ks * S + r0 + i] = gi;
            mine[i] = gi;
        }
        cl.sync();
        for (int m = tid; m < lds; m += blockDim.x) vec[m] = m < S ? (T)remote(0, pk(use_layer(0), m)) : (T)0;
        for (int t = 0; t < nuse; ++t) {
            ready(t);
            const T *Bt = buf + (size_t)(t % nbuf) * rpc * lds;
            const bool last = t == nuse - 1;
            const int kn = use_layer(t) + dk;          // the layer whose vector this product feeds
            const T *cf = dk > 0 ? a.lo : a.up;
            for (int i = warp; i < nr; i += nw) {
                const T acc = rowdot(Bt + (size_t)i * lds);
                if (lane == 0) {
                    if (last) {
                        ymid[(size_t)cq * S + r0 + i] = (double)acc;
                    } else {
                        const size_t e = (size_t)kn * S + r0 + i;
                        const double gi = bval(kn, r0 + i) - (double)cf[e] * (double)acc;
                        g[e] = gi;
                        mine[(size_t)((t + 1) & 1) * rpc + i] = gi;
                    }
                }
            }
            __syncthreads();
            stage(t + nbuf);
            cl.sync();
            if (!last) {
                const int ln = use_layer(t + 1);
                for (int m = tid; m < lds; m += blockDim.x)
                    vec[m] = m < S ? (T)remote((t + 1) & 1, pk(ln, m)) : (T)0;
            }
        }
    } else {
        for (int m = tid; m < lds; m += blockDim.x) {
            T v = (T)0;
            if (m < S) {
                const int o = pk(mid, m);
                const size_t e = (size_t)mid * S + o;
                v = (T)(bval(mid, o) - (double)a.lo[e] * ymid[o] - (double)a.up[e] * ymid[(size_t)S + o]);
            }
            vec[m] = v;
        }
        for (int t = 0; t < nuse; ++t) {
            const int k = use_layer(t);
            if (t > 0) {
                // h = g_k - c_k x_prev, x_prev's rows from their owners (slot of the previous use)
                const T *cb = cq == 0 ? a.up : a.lo;
                for (int m = tid; m < lds; m += blockDim.x) {
                    T v = (T)0;
                    if (m < S) {
                        const int o = pk(k, m);
                        const size_t e = (size_t)k * S + o;
                        v = (T)(g[e] - (double)cb[e] * remote((t - 1) & 1, o));
                    }
                    vec[m] = v;
                }
            }
            ready(t);                 // includes the block barrier that publishes vec
            const T *Bt = buf + (size_t)(t % nbuf) * rpc * lds;
            for (int i = warp; i < nr; i += nw) {
                const T acc = rowdot(Bt + (size_t)i * lds);
                if (lane == 0) {
                    if (t > 0 || cq == 0) x[(size_t)k * S + r0 + i] = (double)acc;
                    mine[(size_t)(t & 1) * rpc + i] = (double)acc;
                }
            }
            __syncthreads();
            stage(t + nbuf);
            cl.sync();
        }
        if (xscale) {
            const int ka = cq == 0 ? 0 : mid + 1, kb = cq == 0 ? mid + 1 : L;
            for (int k = ka; k < kb; ++k)
                for (int i = tid; i < nr; i += blockDim.x) x[(size_t)k * S + r0 + i] *= xscale[(size_t)k * S + r0 + i];
        }
    }
    cp_async_wait0();
}

size_t cluster_smem(int S, int NB, int C, int *nslot, int *lds)
{
    const int npan = (S + NB - 1) / NB;
    *nslot = (npan + C - 1) / C;
    *lds = (S + 3) / 4 * 4;
    const size_t nloc = (size_t)*nslot * NB;
    return (nloc * *lds + (size_t)NB * *lds + nloc * NB + (size_t)NB * (NB + 1)) * sizeof(float);
}

template <int NB>
cudaError_t set_attrs(size_t smem)
{
    auto fn = k_factor_cluster<NB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int NB>
cudaError_t launch_nb(const BlockSys<float> &sys, const ClusterPlan &plan, float *gU, Ctl *ctl, cudaStream_t st,
                      const int *skip, int mode, int mid, int nclusters)
{
    // the shared-memory limit is a property of the function: contexts of other sizes may have set it
    cudaError_t ea = set_attrs<NB>(plan.smem);
    if (ea != cudaSuccess) return ea;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.C * nclusters);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, k_factor_cluster<NB>, sys, gU, ctl, skip, plan.nslot, plan.lds, mode, mid);
}

template <int NB>
int plan_nb(int S, int C, ClusterPlan *out)
{
    ClusterPlan p;
    p.nb = NB;
    p.C = C;
    p.smem = cluster_smem(S, NB, C, &p.nslot, &p.lds);
    if (p.smem > 227 * 1024) return -1;
    const int Q = p.lds / 4;
    int teams = kClusterMaxThreads / Q;
    if (teams < 1) return -1;
    const int rows = p.nslot * NB;
    if (teams > rows) teams = rows;
    p.threads = (teams * Q + 31) / 32 * 32;
    if (p.threads > kClusterMaxThreads) p.threads = kClusterMaxThreads;
    if (set_attrs<NB>(p.smem) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    // the cluster must fit on one GPC with this shared memory
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_factor_cluster<NB>, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return -1;
    }
    p.twisted = nclusters >= 2 ? 1 : 0;
    *out = p;
    return 0;
}

}  // namespace

int cluster_plan(int S, int nb, int C, ClusterPlan *out)
{
    if (S <= 0 || S > 65535) return -1;
    if (nb <= 0) nb = 16;
    if (C > kClusterMaxSize) return -1;
    const int npan = (S + nb - 1) / nb;
    if (C <= 0) {
        // automatic: the largest cluster that leaves every CTA at least one panel
        for (int c = (npan < kClusterMaxSize ? npan : kClusterMaxSize); c >= 1; --c)
            if (cluster_plan(S, nb, c, out) == 0) return 0;
        return -1;
    }
    if (C > npan) C = npan;
    if (nb == 16) return plan_nb<16>(S, C, out);
    if (nb == 8) return plan_nb<8>(S, C, out);
    return -1;
}

size_t cluster_ubuf_floats(const ClusterPlan &plan) { return (size_t)4 * plan.nb * plan.lds; }

bool cluster_twisted(const ClusterPlan &plan, int L) { return plan.twisted && L >= 3; }

cudaError_t launch_factor_cluster(const BlockSys<float> &sys, const ClusterPlan &plan, float *gU, Ctl *ctl,
                                  cudaStream_t st, const int *skip)
{
    auto go = [&](int mode, int mid, int n) -> cudaError_t {
        if (plan.nb == 16) return launch_nb<16>(sys, plan, gU, ctl, st, skip, mode, mid, n);
        if (plan.nb == 8) return launch_nb<8>(sys, plan, gU, ctl, st, skip, mode, mid, n);
        return cudaErrorInvalidValue;
    };
    if (!cluster_twisted(plan, sys.L)) return go(0, 0, 1);
    // twisted elimination: both ends at once on two clusters, then the middle layer
    const int mid = sys.L / 2;
    cudaError_t e = go(1, mid, 2);
    if (e == cudaSuccess) e = go(2, mid, 1);
    return e;
}

namespace {

template <typename T>
int solve_plan_t(int S, SolvePlan *out)
{
    SolvePlan p;
    const int E = 16 / (int)sizeof(T);
    p.lds = (S + E - 1) / E * E;
    auto fn = k_solve_cluster<T>;
    for (int C = kClusterMaxSize; C >= 1; --C) {
        if (C > 1 && (S + C - 1) / C < 8) continue;        // at least 8 rows per CTA
        for (int nbuf = 2; nbuf >= 1; --nbuf) {
            p.C = C;
            p.nbuf = nbuf;
            p.rpc = (S + C - 1) / C;
            p.smem = ((size_t)nbuf * p.rpc * p.lds + p.lds) * sizeof(T) + (size_t)2 * p.rpc * sizeof(double);
            if (p.smem > 227 * 1024) continue;
            p.threads = kSolveClusterThreads;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess ||
                cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(p.threads);
            cfg.dynamicSmemBytes = p.smem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
                cudaGetLastError();
                continue;
            }
            p.twisted = 0;
            if (nclusters >= 2) {
                int n2 = 0;
                auto ft = k_solve_twisted<T>;
                if (cudaFuncSetAttribute(ft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) == cudaSuccess &&
                    cudaFuncSetAttribute(ft, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
                    cudaOccupancyMaxActiveClusters(&n2, ft, &cfg) == cudaSuccess && n2 >= 2)
                    p.twisted = 1;
                cudaGetLastError();
            }
            *out = p;
            return 0;
        }
    }
    return -1;
}

}  // namespace

int solve_cluster_plan(int S, int elem_bytes, SolvePlan *out)
{
    if (S <= 0 || S > 65535) return -1;
    return elem_bytes == 8 ? solve_plan_t<double>(S, out) : solve_plan_t<float>(S, out);
}

template <typename T>
cudaError_t launch_solve_cluster(const BlockSys<T> &sys, const SolvePlan &plan, bool pivoted, const double *b,
                                 double *x, double *g, Ctl *ctl, cudaStream_t st, const double *bscale,
                                 const int *skip, const double *xscale)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.C);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    const int *perm = pivoted ? sys.perm : nullptr;
    // the shared-memory limit is a property of the function: contexts of other sizes may have set it
    cudaError_t ea = cudaFuncSetAttribute(k_solve_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (ea != cudaSuccess) return ea;
    return cudaLaunchKernelEx(&cfg, k_solve_cluster<T>, sys, perm, b, x, g, ctl, bscale, skip, xscale, plan.rpc,
                              plan.lds, plan.nbuf);
}

template <typename T>
cudaError_t launch_solve_twisted(const BlockSys<T> &sys, const SolvePlan &plan, bool pivoted, const double *b,
                                 double *x, double *g, double *ymid, Ctl *ctl, cudaStream_t st, const double *bscale,
                                 const int *skip, const double *xscale)
{
    const int mid = sys.L / 2;
    const int *perm = pivoted ? sys.perm : nullptr;
    cudaError_t ea = cudaFuncSetAttribute(k_solve_twisted<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (ea != cudaSuccess) return ea;
    for (int phase = 0; phase < 2; ++phase) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * plan.C);
        cfg.blockDim = dim3(plan.threads);
        cfg.dynamicSmemBytes = plan.smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = plan.C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        count_launches(1);
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve_twisted<T>, sys, perm, b, x, g, ymid, ctl, bscale, skip,
                                           xscale, plan.rpc, plan.lds, plan.nbuf, phase, mid);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_solve_twisted<float>(const BlockSys<float> &, const SolvePlan &, bool, const double *,
                                                 double *, double *, double *, Ctl *, cudaStream_t, const double *,
                                                 const int *, const double *);
template cudaError_t launch_solve_twisted<double>(const BlockSys<double> &, const SolvePlan &, bool, const double *,
                                                  double *, double *, double *, Ctl *, cudaStream_t,
                                                  const double *, const int *, const double *);

template cudaError_t launch_solve_cluster<float>(const BlockSys<float> &, const SolvePlan &, bool, const double *,
                                                 double *, double *, Ctl *, cudaStream_t, const double *,
                                                 const int *, const double *);
template cudaError_t launch_solve_cluster<double>(const BlockSys<double> &, const SolvePlan &, bool, const double *,
                                                  double *, double *, Ctl *, cudaStream_t, const double *,
                                                  const int *, const double *);

}  // namespace xk
