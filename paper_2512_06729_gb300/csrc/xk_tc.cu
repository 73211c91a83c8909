// Batched products C = A B on the tcgen05 tensor cores with FP32 accuracy.
//
// Each CTA computes one 128 x 128 tile of one task's output.  Warp 0 streams
// the operands into shared memory with TMA, three stages deep: A (row-major,
// i.e. K-major) straight into the 128-byte swizzled layout the tensor core
// reads; B (row-major, i.e. N-major) as a plain [32 k][128 n] tile, because the
// TF32 kind reads K-major operands only (a ring of two such tiles).  Warps 2-9
// split every staged FP32
// element x into a TF32 head h (x rounded to nearest at 10 explicit mantissa
// bits, exact in TF32) and tail l = x - h (exact in FP32, at most 2^-11 |x|),
// itself rounded to TF32: A in place, B while transposing
// it into the K-major swizzled layout (16-byte chunk c of row n stored at chunk
// c ^ (n mod 8)).  Warp 1 issues, per K step of 8,
// the three products A_h B_h + A_h B_l + A_l B_h into one FP32 accumulator in
// tensor memory (the 3xTF32 scheme: the rounding of the tails and the dropped
// A_l B_l term leave at most about 3 * 2^-22 of |a||b| per product, a dozen FP32
// units, far below TF32's 2^-11).  Warps 2-9 then read the accumulator back
// (tcgen05.ld) and apply alpha, beta and the column routing of the task.
//
// Every wait on an mbarrier is bounded; a wait that gives up records
// ctl->err_timeout, and the CTA still waits (bounded) for its own tensor-core
// work and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "xk_tc.cuh"

namespace xk {

namespace {

constexpr int kStages = 3;
constexpr int kSplitWarps = 8;                           // warps 2-9: head/tail split, then the epilogue
constexpr int kSplitThreads = 32 * kSplitWarps;
constexpr int kThreads = 64 + kSplitThreads;             // warp 0 TMA, warp 1 MMA
constexpr uint32_t kTileBytes = kTcTileM * kTcStageK * 4; // 16 KB: A tile (128 x 32) or B tile (32 x 128)
constexpr uint32_t kStageBytes = 4 * kTileBytes;          // A head (TMA lands here), A tail, B head, B tail
constexpr int kRawB = 2;                                  // B as loaded: a ring of two tiles
constexpr uint32_t kTmemCols = 128;
constexpr size_t kSmemBytes = kStages * kStageBytes + kRawB * kTileBytes + 1024 + 256;
constexpr unsigned long long kWaitPolls = 1ull << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase of the given parity; false (and the error flag) when it gives up
// or another thread of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, Ctl *ctl)
{
    for (unsigned long long i = 0; i < kWaitPolls; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    if (ctl) atomicExch(&ctl->err_timeout, 1);
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle: start, leading and stride byte offsets.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of the 5th-generation tensor core
    d |= (uint64_t)2 << 61;          // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4)                  // accumulator FP32
         | (2u << 7)                  // A: TF32
         | (2u << 10)                 // B: TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x rounded to the nearest TF32 value (ties away from zero), low 13 bits cleared: exact in TF32.
__device__ __forceinline__ float tf32_round(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm(const TcTask *__restrict__ tasks, int ntasks, const CUtensorMap *__restrict__ maps, const int *skip, Ctl *ctl)
{
    if ((ctl && (ctl->finished || ctl->err_timeout)) || (skip && *skip)) return;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    const uint32_t raw_u = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + (((raw_u + 1023u) & ~1023u) - raw_u);     // 1024-byte aligned stages
    const uint32_t sbase = smem_u32(smem);
    const uint32_t rawb = sbase + kStages * kStageBytes;               // B as loaded, ring slot it % kRawB
    const uint32_t bars = rawb + kRawB * kTileBytes;
    auto full = [&](int s) { return bars + 8u * s; };
    auto split = [&](int s) { return bars + 8u * (kStages + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kStages + s); };
    const uint32_t accf = bars + 8u * (3 * kStages);
    const uint32_t drain = bars + 8u * (3 * kStages + 1);

    // this CTA's task: the last one whose first tile is at or before blockIdx.x
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const TcTask &t = tasks[lo];
    const int local = (int)blockIdx.x - t.tile0;
    const int tm = local / t.tiles_n, tn = local - tm * t.tiles_n;
    const int nk0 = t.seg[0].k / kTcStageK;
    const int nk = nk0 + (t.nseg > 1 ? t.seg[1].k / kTcStageK : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &abort_sh;

    if (threadIdx.x == 0) {
        abort_sh = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(split(s), kSplitThreads);
            mbar_init(empty(s), 1);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    bool mma_issued = false;

    if (warp == 0) {
        if (lane == 0) {
            for (int it = 0; it < nk; ++it) {
                const int s = it % kStages;
                const uint32_t round = (uint32_t)(it / kStages);
                if (it >= kStages && !mbar_wait(empty(s), (round & 1u) ^ 1u, abort, ctl)) break;
                // the raw-B slot of this iteration was last read by the split of iteration it - kRawB
                if (it >= kRawB) {
                    const int q = it - kRawB;
                    if (!mbar_wait(split(q % kStages), (uint32_t)(q / kStages) & 1u, abort, ctl)) break;
                }
                const TcSeg &g = it < nk0 ? t.seg[0] : t.seg[1];
                const int kk = (it < nk0 ? it : it - nk0) * kTcStageK;
                const uint32_t st = sbase + s * kStageBytes;
                mbar_expect_tx(full(s), 2 * kTileBytes);
                tma_load_3d(st, maps + 2 * g.amap, g.ax + kk, g.ay + tm * kTcTileM, g.az, full(s));
                tma_load_3d(rawb + (it % kRawB) * kTileBytes, maps + 2 * g.bmap + 1, g.bx + tn * kTcTileN, g.by + kk,
                            g.bz, full(s));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tf32_idesc(kTcTileM, kTcTileN);
            for (int it = 0; it < nk; ++it) {
                const int s = it % kStages;
                const uint32_t round = (uint32_t)(it / kStages);
                if (!mbar_wait(split(s), round & 1u, abort, ctl)) break;
                tc_fence_after();
                const uint32_t st = sbase + s * kStageBytes;
#pragma unroll
                for (int ks = 0; ks < kTcStageK / 8; ++ks) {
                    // K-major: rows of 32 FP32 (128 B), 8-row groups 1024 B apart, K step of 8 = 32 B
                    const uint64_t ah = sw128_desc(st + ks * 32u, 16u, 1024u);
                    const uint64_t al = sw128_desc(st + kTileBytes + ks * 32u, 16u, 1024u);
                    const uint64_t bh = sw128_desc(st + 2 * kTileBytes + ks * 32u, 16u, 1024u);
                    const uint64_t bl = sw128_desc(st + 3 * kTileBytes + ks * 32u, 16u, 1024u);
                    mma_tf32(tmem, ah, bh, idesc, (it | ks) ? 1u : 0u);
                    mma_tf32(tmem, ah, bl, idesc, 1u);
                    mma_tf32(tmem, al, bh, idesc, 1u);
                }
                mma_issued = true;
                mma_commit(empty(s));
            }
            mma_commit(accf);
        }
    } else {
        // split the staged tiles into TF32 head and tail, in place
        const int ct = threadIdx.x - 64;
        for (int it = 0; it < nk; ++it) {
            const int s = it % kStages;
            const uint32_t round = (uint32_t)(it / kStages);
            if (!mbar_wait(full(s), round & 1u, abort, ctl)) break;
            uint8_t *st = smem + s * kStageBytes;
            {   // A: element-wise, the layout is already the tensor core's
                float4 *h = (float4 *)st;
                float4 *l = (float4 *)(st + kTileBytes);
#pragma unroll 4
                for (int i = ct; i < (int)(kTileBytes / 16); i += kSplitThreads) {
                    float4 v = h[i];
                    float4 a = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
                    h[i] = a;
                    l[i] = make_float4(tf32_round(v.x - a.x), tf32_round(v.y - a.y), tf32_round(v.z - a.z),
                                       tf32_round(v.w - a.w));
                }
            }
            {   // B: thread ct takes column n = ct mod 128 of the [32 k][128 n] tile, half of its chunks, and
                // writes row n of the K-major tiles, 16-byte chunk c (k = 4c .. 4c+3) at chunk c ^ (n mod 8)
                const float *b = (const float *)(smem + kStages * kStageBytes + (it % kRawB) * kTileBytes);
                uint8_t *bh = st + 2 * kTileBytes, *bl = st + 3 * kTileBytes;
                const int n = ct & (kTcTileN - 1);
                const int c0 = (ct / kTcTileN) * (8 * kTcTileN / kSplitThreads);
#pragma unroll
                for (int c = c0; c < c0 + 8 * kTcTileN / kSplitThreads; ++c) {
                    float4 v = make_float4(b[(4 * c) * kTcTileN + n], b[(4 * c + 1) * kTcTileN + n],
                                           b[(4 * c + 2) * kTcTileN + n], b[(4 * c + 3) * kTcTileN + n]);
                    float4 a = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
                    const uint32_t off = (uint32_t)n * 128u + (uint32_t)((c ^ (n & 7)) * 16);
                    *(float4 *)(bh + off) = a;
                    *(float4 *)(bl + off) = make_float4(tf32_round(v.x - a.x), tf32_round(v.y - a.y),
                                                        tf32_round(v.z - a.z), tf32_round(v.w - a.w));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(split(s));
        }
        // epilogue: TMEM lanes 32 (warp % 4) .. +31 hold this warp's rows; the warps sharing those lanes
        // take different column ranges
        const bool ok = mbar_wait(accf, 0u, abort, ctl);
        tc_fence_after();
        const int ew = warp & 3;
        const int cpart = (warp - 2) / 4;
        constexpr int kColsPerWarp = kTcTileN * 4 / kSplitWarps;
        const int row = tm * kTcTileM + ew * 32 + lane;
#pragma unroll 1
        for (int c0 = cpart * kColsPerWarp; c0 < (cpart + 1) * kColsPerWarp; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0, r);
            const int n = tn * kTcTileN + c0;
            if (!ok || row >= t.m || n >= t.n) continue;
            const int o = (t.nout > 1 && n >= t.out[0].n) ? 1 : 0;
            const TcOut &O = t.out[o];
            const int nn = o ? n - t.out[0].n : n;
            float *dst = O.ptr + (long long)row * O.ld + nn;
            const float *src = (O.beta != 0.0f && O.src) ? O.src + (long long)row * O.lds + nn : nullptr;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 v = make_float4(O.alpha * __uint_as_float(r[j]), O.alpha * __uint_as_float(r[j + 1]),
                                       O.alpha * __uint_as_float(r[j + 2]), O.alpha * __uint_as_float(r[j + 3]));
                if (src) {
                    float4 c = *(const float4 *)(src + j);
                    v.x += O.beta * c.x; v.y += O.beta * c.y; v.z += O.beta * c.z; v.w += O.beta * c.w;
                }
                *(float4 *)(dst + j) = v;
            }
        }
    }
    // an aborted CTA waits (bounded) for the tensor-core work it issued before freeing TMEM
    if (warp == 1 && lane == 0 && *abort && mma_issued) {
        mma_commit(drain);
        for (unsigned long long i = 0; i < kWaitPolls && !mbar_try(drain, 0u); ++i) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

int tc_make_maps(const TcArray &a, CUtensorMap *amap, CUtensorMap *bmap)
{
    EncodeTiled enc = encode_fn();
    if (!enc || !a.base || a.C % 32 || a.R <= 0 || a.Z <= 0 || ((uintptr_t)a.base & 255)) return -1;
    const cuuint64_t dims[3] = {(cuuint64_t)a.C, (cuuint64_t)a.R, (cuuint64_t)a.Z};
    const cuuint64_t strides[2] = {(cuuint64_t)a.C * 4, (cuuint64_t)a.C * a.R * 4};
    const cuuint32_t elem[3] = {1, 1, 1};
    const cuuint32_t box_a[3] = {32, (cuuint32_t)kTcTileM, 1};
    const cuuint32_t box_b[3] = {(cuuint32_t)kTcTileN, (cuuint32_t)kTcStageK, 1};
    if (enc(amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.base, dims, strides, box_a, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return -1;
    if (enc(bmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.base, dims, strides, box_b, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return -1;
    return 0;
}

int tc_number_tiles(TcTask *tasks, int ntasks)
{
    int total = 0;
    for (int i = 0; i < ntasks; ++i) {
        TcTask &t = tasks[i];
        t.tiles_n = (t.n + kTcTileN - 1) / kTcTileN;
        t.tiles = ((t.m + kTcTileM - 1) / kTcTileM) * t.tiles_n;
        t.tile0 = total;
        total += t.tiles;
    }
    return total;
}

cudaError_t launch_tc_gemm(const TcTask *tasks, int ntasks, int total_tiles, const CUtensorMap *maps, const int *skip,
                           Ctl *ctl, cudaStream_t st)
{
    if (ntasks <= 0 || total_tiles <= 0) return cudaSuccess;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    });
    if (attr != cudaSuccess) return attr;
    count_launches(1);
    k_tc_gemm<<<total_tiles, kThreads, kSmemBytes, st>>>(tasks, ntasks, maps, skip, ctl);
    return cudaGetLastError();
}

}  // namespace xk

// ---------------------------------------------------------------------------
// C-ABI: one product, to check the tensor-core contraction on its own.
// ---------------------------------------------------------------------------
namespace {
__device__ xk::TcTask g_tc_task;
__device__ CUtensorMap g_tc_maps[4];
std::mutex g_tc_mu;
}  // namespace

extern "C" int xk_tc_gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                          float alpha, float beta, void *stream)
{
    using namespace xk;
    if (M <= 0 || N <= 0 || K <= 0 || M % 32 || N % 32 || K % 32 || lda % 32 || ldb % 32 || ldc % 32 || lda < K ||
        ldb < N || ldc < N || !A || !B || !C)
        return XK_EINVAL;
    if (((uintptr_t)A & 255) || ((uintptr_t)B & 255) || ((uintptr_t)C & 15)) return XK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    TcArray aa{const_cast<float *>(A), 1, M, lda}, bb{const_cast<float *>(B), 1, K, ldb};
    CUtensorMap maps[4];
    if (tc_make_maps(aa, &maps[0], &maps[1]) || tc_make_maps(bb, &maps[2], &maps[3])) return XK_EINVAL;
    TcTask t{};
    t.nseg = 1;
    t.seg[0] = TcSeg{0, 0, 0, 0, 1, 0, 0, 0, K};
    t.nout = 1;
    t.out[0] = TcOut{C, C, ldc, ldc, alpha, beta, N};
    t.m = M;
    t.n = N;
    int tiles = tc_number_tiles(&t, 1);
    std::lock_guard<std::mutex> lock(g_tc_mu);
    void *dtask = nullptr, *dmaps = nullptr;
    if (cudaGetSymbolAddress(&dtask, g_tc_task) != cudaSuccess || cudaGetSymbolAddress(&dmaps, g_tc_maps) != cudaSuccess ||
        cudaMemcpyAsync(dtask, &t, sizeof t, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dmaps, maps, sizeof maps, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    cudaError_t e = launch_tc_gemm((const TcTask *)dtask, 1, tiles, (const CUtensorMap *)dmaps, nullptr, nullptr, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    return XK_OK;
}
