// Block cyclic reduction (odd-even elimination of layers) of the block-tridiagonal
// system (I/dt - J) x = b, in FP32 on the tensor cores: the mixed path's
// preconditioner, a block LU of the system with its layers ordered odd before
// even, level by level.
//
// Rows of the system: L_k x_{k-1} + D_k x_k + U_k x_{k+1} = b_k.  At each level the
// layers at odd positions j of the current list are eliminated:
//   x_j = D_j^-1 (b_j - L_j x_{j-1} - U_j x_{j+1});
// each kept neighbour i takes the Schur complement
//   D_i <- D_i - L_i Q_l - U_i P_r,  P = D^-1 L,  Q = D^-1 U,
// and couples to the next kept layers through L_i <- -L_i P_l, U_i <- -U_i Q_r.
// At level 0 the couplings are the diagonal transport terms, so the updates are
// element-wise; from level 1 on they are dense S x S blocks and every update is a
// product on the tensor cores (xk_tc.cu), batched over the layers of the level.
// The inverses D_j^-1 come from a recursive 2 x 2 block inversion (Schur
// complement of the leading block), whose products are batched the same way,
// down to blocks of at most 160 rows inverted by one CTA each (Gauss-Jordan
// with partial pivoting).  The work per factorization is about 4x that of
// block Thomas, but instead of a chain of L dependent inversions there are
// about log2(L) levels, each filling the GPU.
//
// Blocks are padded to Sp = round_up(S, 32) rows and columns with the identity
// in the padding, so that every product has dimensions that are multiples of 32.
#include <cuda_runtime.h>

#include <algorithm>

#include "xk_bcr.cuh"

namespace xk {

namespace {

constexpr int kLeafWarpsUsed = 16;   // warps of the leaf inversion: 16 x 50 elements per thread
constexpr int kMvThreads = 256;
constexpr int kMvRows = 64;
constexpr int kArrD = 0, kArrINV = 1, kArrTMP = 2, kArrCP = 3, kArrPQ = 4, kArrays = 5;

__device__ __forceinline__ bool stop(const int *skip, const Ctl *ctl)
{
    return (ctl && (ctl->finished || ctl->err_timeout)) || (skip && *skip);
}

// Leading (upper-left) part of a block of n rows in the recursive inversion: a multiple of 32.
int split_of(int n) { return 32 * ((n + 63) / 64); }

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion with partial pivoting of one block per CTA, the block
// held in registers: warp v owns columns v + 16 b (b < 10) and lane l owns rows
// l + 32 a (a < 5), so column c belongs to one whole warp and, with the column
// loop unrolled over b, to a fixed register.  Pivoting is implicit: rows never
// move; the pivot of column c is the unused row p(c) of largest |value|, and
// the in-place elimination leaves row p(k) holding row k of (P M)^-1, so
// M^-1[k][p(c)] = W[p(k)][c].
//
// One barrier per column.  After it every warp reads the pivot row index, the
// pivot and the column's multipliers from shared memory and takes the pivot
// row's entries in its own columns from the lane that holds them (a warp
// shuffle).  The warp owning the next column updates that column first, picks
// its pivot (redux.sync maximum of |value| over the unused rows, the lowest
// row on ties) and publishes it before updating its other columns
// (look-ahead); shared buffers alternate between columns.
// ---------------------------------------------------------------------------
constexpr int kLeafRowGroups = (kBcrLeafMax + 31) / 32;                         // 5

// Row groups: element a of a lane's rows selected by a runtime index.
__device__ __forceinline__ float leaf_pick(const float (&col)[kLeafRowGroups], int a)
{
    float v = col[0];
#pragma unroll
    for (int q = 1; q < kLeafRowGroups; ++q)
        if (a == q) v = col[q];
    return v;
}

struct LeafPivot {
    int p;
    float v;
};

// Pivot of one column (its values in this lane's rows: col[a]) over the unused rows of the warp.
__device__ __forceinline__ LeafPivot leaf_argmax(const float (&col)[kLeafRowGroups], unsigned used, int ln, int n)
{
    unsigned key = 0u;
    int br = 0x7fffffff;
#pragma unroll
    for (int a = 0; a < kLeafRowGroups; ++a) {
        const float v = fabsf(col[a]);
        const unsigned k = (((used >> a) & 1u) || !(v == v)) ? 0u : __float_as_uint(v) + 1u;
        if (k > key) { key = k; br = ln + 32 * a; }
    }
    const unsigned m = __reduce_max_sync(0xffffffffu, key);
    int p = (int)__reduce_min_sync(0xffffffffu, (key == m && m != 0u) ? (unsigned)br : 0x7fffffffu);
    if (m == 0u || p >= n) p = 0;       // no candidate left: a singular block
    const float val = __shfl_sync(0xffffffffu, leaf_pick(col, p >> 5), p & 31);
    return LeafPivot{p, val};
}

template <int kLeafWarps>
__global__ void __launch_bounds__(kLeafWarps * 32, 1) k_leaf_inverse(const BcrLeaf *tasks, const int *skip, const Ctl *ctl)
{
    constexpr int kLeafColGroups = (kBcrLeafMax + kLeafWarps - 1) / kLeafWarps;
    if (stop(skip, ctl)) return;
    const BcrLeaf t = tasks[blockIdx.x];
    __shared__ float fcol[2][kBcrLeafMax];
    __shared__ float pval[2];
    __shared__ int piv[2];
    __shared__ int perm[kBcrLeafMax], iperm[kBcrLeafMax];
    const int n = t.n;
    const int ln = threadIdx.x & 31, wv = threadIdx.x >> 5;
    float w[kLeafColGroups][kLeafRowGroups];        // w[b][a] = W[ln + 32 a][wv + 16 b]
    unsigned used = 0;
#pragma unroll
    for (int a = 0; a < kLeafRowGroups; ++a) {
        const int r = ln + 32 * a;
#pragma unroll
        for (int b = 0; b < kLeafColGroups; ++b) {
            const int j = wv + kLeafWarps * b;
            w[b][a] = (r < n && j < n) ? t.in[(long long)r * t.ldin + j] : 0.0f;
        }
        if (r >= n) used |= 1u << a;
    }
    // column 0: its owner (warp 0) publishes the first pivot
    if (wv == 0) {
        const LeafPivot pv = leaf_argmax(w[0], used, ln, n);
#pragma unroll
        for (int a = 0; a < kLeafRowGroups; ++a) {
            const int r = ln + 32 * a;
            if (r < n) fcol[0][r] = w[0][a];
        }
        if (ln == 0) { piv[0] = pv.p; pval[0] = pv.v; perm[0] = pv.p; iperm[pv.p] = 0; }
    }
    __syncthreads();
#pragma unroll
    for (int bc = 0; bc < kLeafColGroups; ++bc) {
        for (int cw = 0; cw < kLeafWarps; ++cw) {
            const int c = kLeafWarps * bc + cw;
            if (c >= n) break;
            const int buf = c & 1;
            const int p = piv[buf];
            const int pa = p >> 5, pl = p & 31;
            float pivv = pval[buf];
            if (pivv == 0.0f) pivv = 1e-30f;    // singular block: the FP64 Krylov solve sees a poor preconditioner
            const float inv = 1.0f / pivv;
            float f[kLeafRowGroups];
#pragma unroll
            for (int a = 0; a < kLeafRowGroups; ++a) {
                const int r = ln + 32 * a;
                f[a] = (r < n) ? fcol[buf][r] : 0.0f;
            }
            if (ln == pl) used |= 1u << pa;          // row p is a pivot from now on
            const bool own = (wv == cw);             // this warp owns column c
            // the pivot row in this warp's columns (lane pl, row group pa: uniform over the warp), scaled;
            // the column-c entry becomes 1 / pivot
            float pr[kLeafColGroups];
            switch (pa) {
#define XK_LEAF_ROW(A)                                                                            \
    case A:                                                                                       \
        _Pragma("unroll") for (int b = 0; b < kLeafColGroups; ++b) pr[b] =                     \
            __shfl_sync(0xffffffffu, w[b][A], pl);                                                \
        break;
                XK_LEAF_ROW(0) XK_LEAF_ROW(1) XK_LEAF_ROW(2) XK_LEAF_ROW(3) XK_LEAF_ROW(4)
#undef XK_LEAF_ROW
            }
#pragma unroll
            for (int b = 0; b < kLeafColGroups; ++b) pr[b] *= inv;
            if (own) pr[bc] = inv;
            // update of one column b: every row w - f pr (column c: -f / pivot); the pivot row is
            // then overwritten by its scaled values (fix_pivot)
            auto update = [&](float (&col)[kLeafRowGroups], float prb, bool is_c) {
#pragma unroll
                for (int a = 0; a < kLeafRowGroups; ++a) col[a] = is_c ? -f[a] * inv : fmaf(-f[a], prb, col[a]);
            };
            auto fix_pivot = [&](float (&col)[kLeafRowGroups], float prb) {
                if (ln == pl) {
                    switch (pa) {
                    case 0: col[0] = prb; break;
                    case 1: col[1] = prb; break;
                    case 2: col[2] = prb; break;
                    case 3: col[3] = prb; break;
                    default: col[4] = prb; break;
                    }
                }
            };
            // look-ahead: the owner of column c + 1 updates it, picks its pivot and publishes it first
            const int cn = c + 1;
            const int nw = cn % kLeafWarps;
            const bool next_here = cn < n && wv == nw;
            if (next_here) {
                if (cw + 1 < kLeafWarps) {
                    update(w[bc], pr[bc], false);
                    fix_pivot(w[bc], pr[bc]);
                    const LeafPivot pv = leaf_argmax(w[bc], used, ln, n);
#pragma unroll
                    for (int a = 0; a < kLeafRowGroups; ++a) {
                        const int r = ln + 32 * a;
                        if (r < n) fcol[buf ^ 1][r] = w[bc][a];
                    }
                    if (ln == 0) { piv[buf ^ 1] = pv.p; pval[buf ^ 1] = pv.v; perm[cn] = pv.p; iperm[pv.p] = cn; }
                } else if (bc + 1 < kLeafColGroups) {
                    update(w[bc + 1], pr[bc + 1], false);
                    fix_pivot(w[bc + 1], pr[bc + 1]);
                    const LeafPivot pv = leaf_argmax(w[bc + 1], used, ln, n);
#pragma unroll
                    for (int a = 0; a < kLeafRowGroups; ++a) {
                        const int r = ln + 32 * a;
                        if (r < n) fcol[buf ^ 1][r] = w[bc + 1][a];
                    }
                    if (ln == 0) { piv[buf ^ 1] = pv.p; pval[buf ^ 1] = pv.v; perm[cn] = pv.p; iperm[pv.p] = cn; }
                }
            }
#pragma unroll
            for (int b = 0; b < kLeafColGroups; ++b) {
                const bool done_early = next_here && ((cw + 1 < kLeafWarps) ? (b == bc) : (b == bc + 1));
                if (!done_early) update(w[b], pr[b], own && b == bc);
            }
            if (ln == pl) {
                switch (pa) {
#define XK_LEAF_FIX(A)                                                                           \
    case A:                                                                                      \
        _Pragma("unroll") for (int b = 0; b < kLeafColGroups; ++b) w[b][A] = pr[b];             \
        break;
                    XK_LEAF_FIX(0) XK_LEAF_FIX(1) XK_LEAF_FIX(2) XK_LEAF_FIX(3) XK_LEAF_FIX(4)
#undef XK_LEAF_FIX
                }
            }
            __syncthreads();
        }
    }
    // M^-1[k][p(c)] = W[p(k)][c]: row r = p(k) of W goes to row iperm[r] of the output
#pragma unroll
    for (int a = 0; a < kLeafRowGroups; ++a) {
        const int r = ln + 32 * a;
        if (r >= n) continue;
        float *o = t.out + (long long)iperm[r] * t.ldout;
#pragma unroll
        for (int b = 0; b < kLeafColGroups; ++b) {
            const int j = wv + kLeafWarps * b;
            if (j < n) o[perm[j]] = w[b][a];
        }
    }
}

// Level 0 (diagonal couplings), for each kept even layer i with eliminated neighbours l = i-1, r = i+1:
//   D_i -= diag(lo_i) INV_l diag(up_l) + diag(up_i) INV_r diag(lo_r)
//   CP(1, i/2) = [ -diag(lo_i) INV_l diag(lo_l) | -diag(up_i) INV_r diag(up_r) ]
__global__ void k_bcr_level0(float *D, const float *INV, float *CP, const float *lo, const float *up, const int *kept,
                             int L, int S, int Sp, const int *skip, const Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    const int i = kept[blockIdx.y];
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Sp * Sp) return;
    const int y = (int)(e / Sp), c = (int)(e - (long long)y * Sp);
    const long long blk = (long long)Sp * Sp;
    const bool hasl = i >= 1, hasr = i + 1 < L;
    const float loi = (hasl && y < S) ? lo[(long long)i * S + y] : 0.0f;
    const float upi = (hasr && y < S) ? up[(long long)i * S + y] : 0.0f;
    float upd = 0.0f;
    float *cp = CP + (long long)(i / 2) * Sp * 2 * Sp + (long long)y * 2 * Sp;
    if (hasl) {
        const float g = INV[(long long)(i - 1) * blk + e];
        upd += loi * g * (c < S ? up[(long long)(i - 1) * S + c] : 0.0f);
        if (i >= 2) cp[c] = -loi * g * (c < S ? lo[(long long)(i - 1) * S + c] : 0.0f);
    }
    if (hasr) {
        const float g = INV[(long long)(i + 1) * blk + e];
        upd += upi * g * (c < S ? lo[(long long)(i + 1) * S + c] : 0.0f);
        if (i + 2 <= L - 1) cp[Sp + c] = -upi * g * (c < S ? up[(long long)(i + 1) * S + c] : 0.0f);
    }
    D[(long long)i * blk + e] -= upd;
}

// Batched y = base + sign M v (one block per blockIdx.y, kMvRows rows per blockIdx.x).
__global__ void __launch_bounds__(kMvThreads) k_bcr_mv(const BcrMv *tasks, int S, int Sp, const int *skip, const Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    const BcrMv t = tasks[blockIdx.y];
    extern __shared__ float v[];
    for (int k = threadIdx.x; k < t.K; k += blockDim.x) {
        float val;
        if (k < Sp) {
            val = t.v0[k];
            if (k < S) {
                if (t.d0) val -= t.d0[k] * t.w0[k];
                if (t.d1) val -= t.d1[k] * t.w1[k];
            }
        } else {
            val = t.v1[k - Sp];
        }
        v[k] = val;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r1 = min(Sp, (int)(blockIdx.x + 1) * kMvRows);
    for (int r = blockIdx.x * kMvRows + warp; r < r1; r += kMvThreads / 32) {
        const float4 *row = (const float4 *)(t.M + (long long)r * t.ld);
        float acc = 0.0f;
        for (int q = lane; q < t.K / 4; q += 32) {
            const float4 m = row[q];
            acc += m.x * v[4 * q] + m.y * v[4 * q + 1] + m.z * v[4 * q + 2] + m.w * v[4 * q + 3];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) t.y[r] = (t.base ? t.base[r] : 0.0f) + t.sign * acc;
    }
}

__global__ void k_bcr_in(const double *b, const double *bscale, float *bw, int L, int S, int Sp, const int *skip,
                         const Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)L * Sp) return;
    const int k = (int)(e / Sp), y = (int)(e - (long long)k * Sp);
    float val = 0.0f;
    if (y < S) {
        const long long q = (long long)k * S + y;
        val = (float)(bscale ? b[q] * bscale[q] : b[q]);
    }
    bw[e] = val;
}

__global__ void k_bcr_out(const float *xw, const double *xscale, double *x, int L, int S, int Sp, const int *skip,
                          const Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)L * S) return;
    const int k = (int)(e / S), y = (int)(e - (long long)k * S);
    const double val = (double)xw[(long long)k * Sp + y];
    x[e] = xscale ? val * xscale[e] : val;
}

// Level-0 right-hand-side update of the kept even layers: b_i -= lo_i t_{i-1} + up_i t_{i+1}.
__global__ void k_bcr_fwd0(float *bw, const float *tw, const float *lo, const float *up, int L, int S, int Sp,
                           const int *skip, const Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nk = (L + 1) / 2;
    if (e >= (long long)nk * S) return;
    const int i = 2 * (int)(e / S), y = (int)(e % S);
    float acc = 0.0f;
    if (i >= 1) acc += lo[(long long)i * S + y] * tw[(long long)(i - 1) * Sp + y];
    if (i + 1 < L) acc += up[(long long)i * S + y] * tw[(long long)(i + 1) * Sp + y];
    bw[(long long)i * Sp + y] -= acc;
}

// The whole solve in one cooperative launch: the stages of the plan in order, each spread over
// the grid, separated by bounded grid barriers.  A skipped solve costs one early-exiting launch.
struct SolveArgs {
    const BcrStage *stages;
    const BcrMv *mv;
    const double *b, *bscale, *xscale;
    double *x;
    float *bw, *tw, *xw;
    const float *lo, *up;
    unsigned *bar;
    int nstages, L, S, Sp;
};

__global__ void __launch_bounds__(kMvThreads) k_bcr_solve_all(SolveArgs a, const int *skip, Ctl *ctl)
{
    if (stop(skip, ctl)) return;
    extern __shared__ float v[];
    const int S = a.S, Sp = a.Sp, L = a.L;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gstride = (long long)gridDim.x * blockDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int chunks = (Sp + kMvRows - 1) / kMvRows;
    for (int si = 0; si < a.nstages; ++si) {
        const BcrStage st = a.stages[si];
        if (st.kind == kBcrIn) {
            for (long long e = gtid; e < (long long)L * Sp; e += gstride) {
                const int k = (int)(e / Sp), y = (int)(e - (long long)k * Sp);
                float val = 0.0f;
                if (y < S) {
                    const long long q = (long long)k * S + y;
                    val = (float)(a.bscale ? a.b[q] * a.bscale[q] : a.b[q]);
                }
                a.bw[e] = val;
            }
        } else if (st.kind == kBcrFwd0) {
            const int nk = (L + 1) / 2;
            for (long long e = gtid; e < (long long)nk * S; e += gstride) {
                const int i = 2 * (int)(e / S), y = (int)(e % S);
                float acc = 0.0f;
                if (i >= 1) acc += a.lo[(long long)i * S + y] * a.tw[(long long)(i - 1) * Sp + y];
                if (i + 1 < L) acc += a.up[(long long)i * S + y] * a.tw[(long long)(i + 1) * Sp + y];
                a.bw[(long long)i * Sp + y] -= acc;
            }
        } else if (st.kind == kBcrOut) {
            for (long long e = gtid; e < (long long)L * S; e += gstride) {
                const int k = (int)(e / S), y = (int)(e - (long long)k * S);
                const double val = (double)a.xw[(long long)k * Sp + y];
                a.x[e] = a.xscale ? val * a.xscale[e] : val;
            }
        } else if (st.kind == kBcrMv) {
            const int items = st.count * chunks;
            for (int item = blockIdx.x; item < items; item += gridDim.x) {
                const BcrMv t = a.mv[st.off + item / chunks];
                const int chunk = item % chunks;
                __syncthreads();
                for (int k = threadIdx.x; k < t.K; k += blockDim.x) {
                    float val;
                    if (k < Sp) {
                        val = t.v0[k];
                        if (k < S) {
                            if (t.d0) val -= t.d0[k] * t.w0[k];
                            if (t.d1) val -= t.d1[k] * t.w1[k];
                        }
                    } else {
                        val = t.v1[k - Sp];
                    }
                    v[k] = val;
                }
                __syncthreads();
                const int r1 = min(Sp, (chunk + 1) * kMvRows);
                for (int r = chunk * kMvRows + warp; r < r1; r += kMvThreads / 32) {
                    const float4 *row = (const float4 *)(t.M + (long long)r * t.ld);
                    float acc = 0.0f;
                    for (int q = lane; q < t.K / 4; q += 32) {
                        const float4 m = row[q];
                        acc += m.x * v[4 * q] + m.y * v[4 * q + 1] + m.z * v[4 * q + 2] + m.w * v[4 * q + 3];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) t.y[r] = (t.base ? t.base[r] : 0.0f) + t.sign * acc;
                }
            }
        }
        if (si + 1 < a.nstages && !grid_barrier(a.bar, ctl)) return;
    }
}

__global__ void k_bcr_pad(float *D, int L, int S, int Sp)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int padr = Sp - S;
    if (padr <= 0 || e >= (long long)L * padr * Sp) return;
    const int k = (int)(e / ((long long)padr * Sp));
    const long long rem = e - (long long)k * padr * Sp;
    const int y = S + (int)(rem / Sp), c = (int)(rem % Sp);
    D[((long long)k * Sp + y) * Sp + c] = (c == y) ? 1.0f : 0.0f;
}

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Host: the plan (stages of task lists), built from the layer structure alone.
// ---------------------------------------------------------------------------
struct View {
    int arr, r0, c0;
};

struct Builder {
    BcrPlan &p;
    int L, S, Sp;
    std::vector<int> depth_col;

    int cols(int arr) const
    {
        switch (arr) {
        case kArrD: case kArrINV: return Sp;
        case kArrTMP: return p.Wt;
        default: return 2 * Sp;
        }
    }
    float *base(int arr) const
    {
        switch (arr) {
        case kArrD: return p.D;
        case kArrINV: return p.INV;
        case kArrTMP: return p.TMP;
        case kArrCP: return p.CP;
        default: return p.PQ;
        }
    }
    float *ptr(int arr, int z, int r, int c) const
    {
        float *b = base(arr);
        if (!b) return nullptr;
        return b + ((size_t)z * Sp + r) * (size_t)cols(arr) + c;
    }
    TcOut out(int arr, int z, int r, int c, float alpha, float beta, int n, bool accumulate) const
    {
        TcOut o;
        o.ptr = ptr(arr, z, r, c);
        o.src = accumulate ? o.ptr : nullptr;
        o.ld = o.lds = cols(arr);
        o.alpha = alpha;
        o.beta = accumulate ? beta : 0.0f;
        o.n = n;
        return o;
    }
    // one product task C = A B: A (m x k) at (ai, az, ar, ac), B (k x n) at (bi, bz, br, bc)
    static TcTask product(int m, int n, int k, View a, int az, View b, int bz, TcOut o)
    {
        TcTask t{};
        t.nseg = 1;
        t.seg[0] = TcSeg{a.arr, a.c0, a.r0, az, b.arr, b.c0, b.r0, bz, k};
        t.nout = 1;
        t.out[0] = o;
        t.m = m;
        t.n = n;
        return t;
    }
    void gemm_stage(std::vector<TcTask> &ts, int level)
    {
        if (ts.empty()) return;
        BcrStage s{kBcrGemm, (int)p.gemm.size(), (int)ts.size(), tc_number_tiles(ts.data(), (int)ts.size()), level};
        p.gemm.insert(p.gemm.end(), ts.begin(), ts.end());
        p.fac.push_back(s);
    }
    // Widths of the temporaries at each recursion depth: X (h x r), Y (r x h), Sc (r x r) side by side.
    void widths(int n, int d, std::vector<int> &w) const
    {
        if (n <= kBcrLeafMax) return;
        const int h = split_of(n), r = n - h;
        if ((int)w.size() <= d) w.resize(d + 1, 0);
        w[d] = std::max(w[d], 2 * r + h);
        widths(h, d + 1, w);
        widths(r, d + 1, w);
    }
    // Inverse of the n x n blocks in (layer zin[b]) into out (layer zout[b]); temporaries in TMP layer b.
    void inverse(int n, View in, const std::vector<int> &zin, View out, const std::vector<int> &zout, int d, int level)
    {
        const int B = (int)zin.size();
        if (n <= kBcrLeafMax) {
            BcrStage s{kBcrLeafStage, (int)p.leaf.size(), B, 0, level};
            for (int b = 0; b < B; ++b)
                p.leaf.push_back(BcrLeaf{ptr(in.arr, zin[b], in.r0, in.c0), ptr(out.arr, zout[b], out.r0, out.c0),
                                         cols(in.arr), cols(out.arr), n});
            p.fac.push_back(s);
            return;
        }
        const int h = split_of(n), r = n - h, cd = depth_col[d];
        const View A{in.arr, in.r0, in.c0}, Bv{in.arr, in.r0, in.c0 + h}, Cv{in.arr, in.r0 + h, in.c0},
            Dv{in.arr, in.r0 + h, in.c0 + h};
        const View TL{out.arr, out.r0, out.c0}, TR{out.arr, out.r0, out.c0 + h}, BL{out.arr, out.r0 + h, out.c0},
            BR{out.arr, out.r0 + h, out.c0 + h};
        const View X{kArrTMP, 0, cd}, Y{kArrTMP, 0, cd + r}, Sc{kArrTMP, 0, cd + r + h};
        std::vector<int> zt(B);
        for (int b = 0; b < B; ++b) zt[b] = b;
        // 1. A^-1 into TL
        inverse(h, A, zin, TL, zout, d + 1, level);
        std::vector<TcTask> ts;
        // 2. X = A^-1 B, Y = C A^-1
        for (int b = 0; b < B; ++b) {
            ts.push_back(product(h, r, h, TL, zout[b], Bv, zin[b], out_of(X, b, 1.0f, 0.0f, r, false)));
            ts.push_back(product(r, h, h, Cv, zin[b], TL, zout[b], out_of(Y, b, 1.0f, 0.0f, h, false)));
        }
        gemm_stage(ts, level);
        ts.clear();
        // 3. Sc = D - C X
        for (int b = 0; b < B; ++b) {
            TcTask t = product(r, r, h, Cv, zin[b], X, zt[b], out_of(Sc, b, -1.0f, 1.0f, r, false));
            t.out[0].src = ptr(Dv.arr, zin[b], Dv.r0, Dv.c0);
            t.out[0].lds = cols(Dv.arr);
            t.out[0].beta = 1.0f;
            ts.push_back(t);
        }
        gemm_stage(ts, level);
        ts.clear();
        // 4. Sc^-1 into BR
        inverse(r, Sc, zt, BR, zout, d + 1, level);
        // 5. TR = -X Sc^-1, BL = -Sc^-1 Y
        for (int b = 0; b < B; ++b) {
            ts.push_back(product(h, r, r, X, zt[b], BR, zout[b], out_view(TR, zout[b], -1.0f, r)));
            ts.push_back(product(r, h, r, BR, zout[b], Y, zt[b], out_view(BL, zout[b], -1.0f, h)));
        }
        gemm_stage(ts, level);
        ts.clear();
        // 6. TL = A^-1 - X BL
        for (int b = 0; b < B; ++b) {
            TcTask t = product(h, h, r, X, zt[b], BL, zout[b], out_view(TL, zout[b], -1.0f, h));
            t.out[0].src = t.out[0].ptr;
            t.out[0].beta = 1.0f;
            ts.push_back(t);
        }
        gemm_stage(ts, level);
    }
    TcOut out_of(View v, int z, float alpha, float beta, int n, bool acc) const
    {
        return out(v.arr, z, v.r0, v.c0, alpha, beta, n, acc);
    }
    TcOut out_view(View v, int z, float alpha, int n) const { return out(v.arr, z, v.r0, v.c0, alpha, 0.0f, n, false); }

    void mv_stage(std::vector<BcrMv> &ts, int level)
    {
        if (ts.empty()) return;
        BcrStage s{kBcrMv, (int)p.mv.size(), (int)ts.size(), 0, level};
        p.mv.insert(p.mv.end(), ts.begin(), ts.end());
        p.sol.push_back(s);
    }
    float *vec(float *a, int k) const { return a ? a + (size_t)k * Sp : nullptr; }
    const float *row(const float *a, int k) const { return a ? a + (size_t)k * S : nullptr; }

    void build()
    {
        std::vector<int> w;
        widths(Sp, 0, w);
        depth_col.assign(w.size() + 1, 0);
        for (size_t d = 0; d < w.size(); ++d) depth_col[d + 1] = depth_col[d] + w[d];
        p.Wt = std::max(32, (depth_col.back() + 31) / 32 * 32);
        // the levels of the reduction
        std::vector<std::vector<int>> lists{std::vector<int>(L)};
        for (int k = 0; k < L; ++k) lists[0][k] = k;
        while (lists.back().size() > 1) {
            const auto &a = lists.back();
            std::vector<int> kept;
            for (size_t q = 0; q < a.size(); q += 2) kept.push_back(a[q]);
            lists.push_back(kept);
        }
        p.levels = (int)lists.size() - 1;
        std::vector<int> cp_off(lists.size(), 0);
        int ncp = 0;
        for (size_t l = 1; l < lists.size(); ++l) {
            cp_off[l] = ncp;
            ncp += (int)lists[l].size();
        }
        p.Ncp = std::max(ncp, 1);
        int zt = 1;
        for (int l = 0; l < p.levels; ++l) zt = std::max(zt, (int)lists[l].size() / 2);
        p.Zt = zt;
        p.level0_kept.clear();
        for (int k = 0; k < L; k += 2) p.level0_kept.push_back(k);
        const View Dfull{kArrD, 0, 0}, Ifull{kArrINV, 0, 0};
        // factorization
        for (int l = 0; l < p.levels; ++l) {
            const auto &a = lists[l];
            std::vector<int> elim;
            for (size_t q = 1; q < a.size(); q += 2) elim.push_back(a[q]);
            inverse(Sp, Dfull, elim, Ifull, elim, 0, l);
            if (l == 0) {
                p.fac.push_back(BcrStage{kBcrLevel0, 0, (int)p.level0_kept.size(), 0, 0});
                continue;
            }
            std::vector<TcTask> ts;
            // [P_j | Q_j] = D_j^-1 [L_j | U_j]
            for (size_t q = 1; q < a.size(); q += 2) {
                const int j = a[q];
                const bool right = q + 1 < a.size();
                const int n = right ? 2 * Sp : Sp;
                ts.push_back(product(Sp, n, Sp, Ifull, j, View{kArrCP, 0, 0}, cp_off[l] + (int)q,
                                     out(kArrPQ, j, 0, 0, 1.0f, 0.0f, n, false)));
            }
            gemm_stage(ts, l);
            ts.clear();
            // Schur complements and the couplings of the next level
            for (size_t q = 0; q < a.size(); q += 2) {
                const int i = a[q];
                const int cpi = cp_off[l] + (int)q;
                const bool hl = q >= 1, hr = q + 1 < a.size();
                if (!hl && !hr) continue;
                TcTask t{};
                t.nseg = 0;
                if (hr) t.seg[t.nseg++] = TcSeg{kArrCP, Sp, 0, cpi, kArrPQ, 0, 0, a[q + 1], Sp};       // U_i P_r
                if (hl) t.seg[t.nseg++] = TcSeg{kArrCP, 0, 0, cpi, kArrPQ, Sp, 0, a[q - 1], Sp};       // L_i Q_l
                t.nout = 1;
                t.out[0] = out(kArrD, i, 0, 0, -1.0f, 1.0f, Sp, true);
                t.m = Sp;
                t.n = Sp;
                ts.push_back(t);
                const int cpn = cp_off[l + 1] + (int)(q / 2);
                if (hl && q >= 2)       // L_i <- -L_i P_l
                    ts.push_back(product(Sp, Sp, Sp, View{kArrCP, 0, 0}, cpi, View{kArrPQ, 0, 0}, a[q - 1],
                                         out(kArrCP, cpn, 0, 0, -1.0f, 0.0f, Sp, false)));
                if (hr && q + 2 < a.size())   // U_i <- -U_i Q_r
                    ts.push_back(product(Sp, Sp, Sp, View{kArrCP, 0, Sp}, cpi, View{kArrPQ, 0, Sp}, a[q + 1],
                                         out(kArrCP, cpn, 0, Sp, -1.0f, 0.0f, Sp, false)));
            }
            gemm_stage(ts, l);
        }
        const int root = lists.back()[0];
        inverse(Sp, Dfull, std::vector<int>{root}, Ifull, std::vector<int>{root}, 0, p.levels);
        // solve
        p.sol.push_back(BcrStage{kBcrIn, 0, 0, 0, 0});
        for (int l = 0; l < p.levels; ++l) {
            const auto &a = lists[l];
            std::vector<BcrMv> ts;
            for (size_t q = 1; q < a.size(); q += 2) {       // t_j = D_j^-1 b_j
                const int j = a[q];
                ts.push_back(BcrMv{ptr(kArrINV, j, 0, 0), vec(p.bw, j), nullptr, nullptr, nullptr, nullptr, nullptr,
                                   nullptr, vec(p.tw, j), Sp, Sp, 1.0f});
            }
            mv_stage(ts, l);
            ts.clear();
            if (l == 0) {
                p.sol.push_back(BcrStage{kBcrFwd0, 0, 0, 0, 0});
                continue;
            }
            for (size_t q = 0; q < a.size(); q += 2) {       // b_i -= L_i t_l + U_i t_r
                const int i = a[q];
                const int cpi = cp_off[l] + (int)q;
                const bool hl = q >= 1, hr = q + 1 < a.size();
                if (!hl && !hr) continue;
                BcrMv t{};
                t.ld = 2 * Sp;
                t.sign = -1.0f;
                t.base = vec(p.bw, i);
                t.y = vec(p.bw, i);
                if (hl && hr) {
                    t.M = ptr(kArrCP, cpi, 0, 0); t.K = 2 * Sp; t.v0 = vec(p.tw, a[q - 1]); t.v1 = vec(p.tw, a[q + 1]);
                } else if (hl) {
                    t.M = ptr(kArrCP, cpi, 0, 0); t.K = Sp; t.v0 = vec(p.tw, a[q - 1]);
                } else {
                    t.M = ptr(kArrCP, cpi, 0, Sp); t.K = Sp; t.v0 = vec(p.tw, a[q + 1]);
                }
                ts.push_back(t);
            }
            mv_stage(ts, l);
        }
        {
            std::vector<BcrMv> ts{BcrMv{ptr(kArrINV, root, 0, 0), vec(p.bw, root), nullptr, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, vec(p.xw, root), Sp, Sp, 1.0f}};
            mv_stage(ts, p.levels);
        }
        for (int l = p.levels - 1; l >= 0; --l) {
            const auto &a = lists[l];
            std::vector<BcrMv> ts;
            for (size_t q = 1; q < a.size(); q += 2) {
                const int j = a[q];
                const bool hr = q + 1 < a.size();
                BcrMv t{};
                t.ld = Sp;
                t.K = Sp;
                t.y = vec(p.xw, j);
                if (l == 0) {      // x_j = D_j^-1 (b_j - lo_j x_{j-1} - up_j x_{j+1})
                    t.M = ptr(kArrINV, j, 0, 0);
                    t.v0 = vec(p.bw, j);
                    t.d0 = row(p.lo, j); t.w0 = vec(p.xw, a[q - 1]);
                    if (hr) { t.d1 = row(p.up, j); t.w1 = vec(p.xw, a[q + 1]); }
                    t.sign = 1.0f;
                } else {           // x_j = t_j - [P_j | Q_j] [x_l; x_r]
                    t.M = ptr(kArrPQ, j, 0, 0);
                    t.ld = 2 * Sp;
                    t.K = hr ? 2 * Sp : Sp;
                    t.v0 = vec(p.xw, a[q - 1]);
                    t.v1 = hr ? vec(p.xw, a[q + 1]) : nullptr;
                    t.base = vec(p.tw, j);
                    t.sign = -1.0f;
                }
                ts.push_back(t);
            }
            mv_stage(ts, l);
        }
        p.sol.push_back(BcrStage{kBcrOut, 0, 0, 0, 0});
    }
};

}  // namespace

BcrSizes bcr_sizes(int L, int S)
{
    BcrPlan p;
    p.L = L;
    p.S = S;
    p.Sp = (S + 31) / 32 * 32;
    Builder b{p, L, S, p.Sp, {}};
    b.build();
    BcrSizes z;
    z.Sp = p.Sp;
    z.Wt = p.Wt;
    z.Zt = p.Zt;
    z.Ncp = p.Ncp;
    z.ngemm = (int)p.gemm.size();
    z.nleaf = (int)p.leaf.size();
    z.nmv = (int)p.mv.size();
    z.nsol = (int)p.sol.size();
    const size_t blk = (size_t)p.Sp * p.Sp;
    z.floats_D = (size_t)L * blk;
    z.floats_INV = (size_t)L * blk;
    z.floats_TMP = (size_t)p.Zt * p.Sp * p.Wt;
    z.floats_CP = (size_t)p.Ncp * 2 * blk;
    z.floats_PQ = (size_t)L * 2 * blk;
    z.floats_vec = (size_t)L * p.Sp;
    return z;
}

int bcr_build(BcrPlan &p, int L, int S, cudaStream_t st)
{
    p.L = L;
    p.S = S;
    p.Sp = (S + 31) / 32 * 32;
    p.gemm.clear(); p.leaf.clear(); p.mv.clear(); p.fac.clear(); p.sol.clear();
    Builder b{p, L, S, p.Sp, {}};
    b.build();
    // tensor maps of the five arrays
    const TcArray arrs[kArrays] = {{p.D, L, p.Sp, p.Sp}, {p.INV, L, p.Sp, p.Sp}, {p.TMP, p.Zt, p.Sp, p.Wt},
                                   {p.CP, p.Ncp, p.Sp, 2 * p.Sp}, {p.PQ, L, p.Sp, 2 * p.Sp}};
    p.maps.assign(2 * kArrays, CUtensorMap{});
    for (int a = 0; a < kArrays; ++a)
        if (tc_make_maps(arrs[a], &p.maps[2 * a], &p.maps[2 * a + 1]) != 0) return -1;
    if (!p.gemm.empty() && cudaMemcpyAsync(p.gemm_d, p.gemm.data(), p.gemm.size() * sizeof(TcTask), cudaMemcpyHostToDevice, st))
        return -1;
    if (!p.leaf.empty() && cudaMemcpyAsync(p.leaf_d, p.leaf.data(), p.leaf.size() * sizeof(BcrLeaf), cudaMemcpyHostToDevice, st))
        return -1;
    if (!p.mv.empty() && cudaMemcpyAsync(p.mv_d, p.mv.data(), p.mv.size() * sizeof(BcrMv), cudaMemcpyHostToDevice, st))
        return -1;
    if (cudaMemcpyAsync(p.maps_d, p.maps.data(), p.maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st))
        return -1;
    if (cudaMemcpyAsync(p.l0_d, p.level0_kept.data(), p.level0_kept.size() * sizeof(int), cudaMemcpyHostToDevice, st))
        return -1;
    if (cudaMemcpyAsync(p.sol_d, p.sol.data(), p.sol.size() * sizeof(BcrStage), cudaMemcpyHostToDevice, st)) return -1;
    // the host copies of the task lists must outlive the asynchronous copies
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    return 0;
}

void bcr_init_pad(const BcrPlan &p, cudaStream_t st)
{
    const long long n = (long long)p.L * (p.Sp - p.S) * p.Sp;
    if (n <= 0) return;
    count_launches(1);
    k_bcr_pad<<<nblk(n, 256), 256, 0, st>>>(p.D, p.L, p.S, p.Sp);
}

void bcr_work(const BcrPlan &p, double *mma_flops, double *leaf_flops)
{
    double m = 0.0, l = 0.0;
    for (const TcTask &t : p.gemm) {
        long long k = 0;
        for (int s = 0; s < t.nseg; ++s) k += t.seg[s].k;
        m += 2.0 * t.m * (double)t.n * (double)k;
    }
    for (const BcrLeaf &f : p.leaf) l += 2.0 * (double)f.n * f.n * f.n;
    if (mma_flops) *mma_flops = m;
    if (leaf_flops) *leaf_flops = l;
}

cudaError_t bcr_factor(const BcrPlan &p, const int *skip, Ctl *ctl, cudaStream_t st, BcrTimer *timer)
{
    for (const BcrStage &s : p.fac) {
        switch (s.kind) {
        case kBcrLeafStage:
            if (timer) timer->begin(s.kind);
            count_launches(1);
            k_leaf_inverse<kLeafWarpsUsed><<<s.count, kLeafWarpsUsed * 32, 0, st>>>(p.leaf_d + s.off, skip, ctl);
            if (timer) timer->end(s.kind);
            break;
        case kBcrGemm: {
            if (timer) timer->begin(s.kind);
            cudaError_t e = launch_tc_gemm(p.gemm_d + s.off, s.count, s.tiles, p.maps_d, skip, ctl, st);
            if (timer) timer->end(s.kind);
            if (e != cudaSuccess) return e;
            break;
        }
        case kBcrLevel0:
            count_launches(1);
            k_bcr_level0<<<dim3(nblk((long long)p.Sp * p.Sp, 256), s.count), 256, 0, st>>>(
                p.D, p.INV, p.CP, p.lo, p.up, p.l0_d, p.L, p.S, p.Sp, skip, ctl);
            break;
        default:
            break;
        }
    }
    return cudaGetLastError();
}

cudaError_t bcr_solve(const BcrPlan &p, const double *b, double *x, const double *bscale, const double *xscale,
                      const int *skip, Ctl *ctl, cudaStream_t st)
{
    static int fit = 0;
    const size_t smem = (size_t)2 * p.Sp * sizeof(float);
    if (!fit) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bcr_solve_all, kMvThreads, 2 * 1280 * sizeof(float)) !=
                cudaSuccess || per < 1)
            per = 1;
        fit = sms * std::min(per, 4);
    }
    int ctas = p.solve_ctas > 0 ? std::min(p.solve_ctas, fit) : fit;
    SolveArgs a;
    a.stages = p.sol_d; a.mv = p.mv_d; a.b = b; a.bscale = bscale; a.xscale = xscale; a.x = x;
    a.bw = p.bw; a.tw = p.tw; a.xw = p.xw; a.lo = p.lo; a.up = p.up; a.bar = p.bar;
    a.nstages = (int)p.sol.size(); a.L = p.L; a.S = p.S; a.Sp = p.Sp;
    void *args[] = {(void *)&a, (void *)&skip, (void *)&ctl};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void *)k_bcr_solve_all, dim3(ctas), dim3(kMvThreads), args, smem, st);
}

}  // namespace xk
