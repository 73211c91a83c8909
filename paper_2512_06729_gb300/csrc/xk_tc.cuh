// Batched FP32-accurate matrix products on the 5th-generation tensor cores
// (tcgen05, TF32 with a hi/lo split: three products per step), the contraction
// the mixed path's block-cyclic-reduction factorization is built from.
#pragma once

#include <cuda.h>

#include "xk_internal.cuh"

namespace xk {

constexpr int kTcTileM = 128;     // output rows per CTA (one TMEM lane each)
constexpr int kTcTileN = 128;     // output columns per CTA (TMEM columns)
constexpr int kTcStageK = 32;     // K per pipeline stage (one 128-byte swizzle atom of FP32)

// A 3-D row-major FP32 array [Z][R][C] (C a multiple of 32, base 256-byte aligned).
struct TcArray {
    float *base;
    int Z, R, C;
};

// One K segment of a product: A tile rows ay + [0, m), columns ax + [0, k) of layer az of
// array amap; B rows by + [0, k), columns bx + [0, n) of layer bz of array bmap.
struct TcSeg {
    int amap, ax, ay, az;
    int bmap, bx, by, bz;
    int k;
};

// Output columns [0, n) of one destination: ptr[r * ld + c] = alpha * (A B)[r][c] + beta * src[r * lds + c]
// (src may equal ptr; beta == 0 reads nothing).
struct TcOut {
    float *ptr;
    const float *src;
    long long ld, lds;
    float alpha, beta;
    int n;
};

// C = sum over segments of A_s B_s, its columns split over up to two destinations.  m, n, k and
// every offset are multiples of 32.
struct TcTask {
    TcSeg seg[2];
    TcOut out[2];
    int nseg, nout;
    int m, n;
    int tile0, tiles_n, tiles;    // filled by tc_number_tiles
};

// Host: tensor maps of an array in its A role (box 32 x 128, 128-byte swizzle) and B role (box
// 128 x 32, unswizzled); 0 or -1.
int tc_make_maps(const TcArray &a, CUtensorMap *amap, CUtensorMap *bmap);
// Host: number the output tiles of a task list; returns the total.
int tc_number_tiles(TcTask *tasks, int ntasks);
// Launch one kernel over all tiles of the task list (tasks and maps in device memory, maps as
// [array][role]).  Exits at once when *skip != 0 or the control block reports a finished step
// or a timed-out wait; a wait of its own that gives up sets ctl->err_timeout.
cudaError_t launch_tc_gemm(const TcTask *tasks, int ntasks, int total_tiles, const CUtensorMap *maps,
                           const int *skip, Ctl *ctl, cudaStream_t st);

}  // namespace xk
