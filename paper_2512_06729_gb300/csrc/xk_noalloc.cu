// Block-tridiagonal solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator hooks, plugins whose host forbids
// device allocations, or code that must not allocate while other work is
// being captured.  For them xk_block_solve_noalloc runs the same FP64
// factorization and solve kernels as xk_block_solve, with all scratch (the
// working copy of the blocks, pivot indices, sweep vector, barrier words and
// control flags) in one file-scope device array of fixed size.  The array is
// part of the loaded library: every GPU that loads it holds the array until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "xk_internal.cuh"

namespace xk {
namespace {

// Fixed scratch for xk_block_solve_noalloc (see XK_NOALLOC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_noalloc_scratch[XK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Whether p is device (or managed) memory that the current device dev can address.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
// A cached address that no longer belongs to the current device's context (the
// device was reset and the library's module loaded again) is looked up anew.
int scratch_on_current_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return XK_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_dev_ptr[dev] && !on_device(g_dev_ptr[dev], dev)) g_dev_ptr[dev] = nullptr;
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return XK_ECUDA;
        }
        g_dev_ptr[dev] = (unsigned char *)p;
    }
    *out = g_dev_ptr[dev];
    return XK_OK;
}

}  // namespace
}  // namespace xk

using namespace xk;

extern "C" int xk_block_solve_noalloc(int L, int S, const double *A, const double *lo, const double *up,
                                      const double *f, double *x, void *stream)
{
    if (L <= 0 || S <= 0 || S > 65535 || !A || !lo || !up || !f || !x) return XK_EINVAL;
    const size_t ld = (size_t)(S + 31) / 32 * 32;
    const size_t LS = (size_t)L * S;
    // scratch layout: control block | barrier words | panel info | pivot rows | pivot columns | sweep vector | blocks
    const size_t o_ctl = 0;
    const size_t o_bar = up256(o_ctl + sizeof(Ctl));
    const size_t o_pinfo = up256(o_bar + 8 * sizeof(unsigned));
    const size_t o_ridx = up256(o_pinfo + (1 + 4 * 64) * sizeof(int));
    const size_t o_sig = up256(o_ridx + LS * sizeof(int));
    const size_t o_g = up256(o_sig + LS * sizeof(int));
    const size_t o_D = up256(o_g + LS * sizeof(double));
    const size_t need = o_D + LS * ld * sizeof(double);
    if (need > (size_t)XK_NOALLOC_SCRATCH_BYTES) return XK_ENOMEM;

    FactorPlan plan;
    if (factor_plan(S, 8, 0, 0, &plan) != 0) return XK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    // every array the kernels touch must be memory of this device (a host pointer would fault)
    if (!on_device(A, dev) || !on_device(lo, dev) || !on_device(up, dev) || !on_device(f, dev) || !on_device(x, dev))
        return XK_EINVAL;
    unsigned char *base = nullptr;
    int rc = scratch_on_current_device(dev, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Ctl *ctl = (Ctl *)(base + o_ctl);
    BlockSys<double> sys;
    sys.D = (double *)(base + o_D);
    sys.lo = lo;
    sys.up = up;
    sys.perm = (int *)(base + o_ridx);
    sys.iperm = (int *)(base + o_sig);
    sys.pinfo = (int *)(base + o_pinfo);
    sys.bar = (unsigned *)(base + o_bar);
    sys.L = L;
    sys.S = S;
    sys.ld = (int)ld;
    // the array keeps the previous call's contents: flags and barrier words start at zero
    // a refused clear or copy would leave the previous call's flags or blocks in place: no launch then
    if (cudaMemsetAsync(base, 0, o_pinfo, st) != cudaSuccess ||
        cudaMemcpy2DAsync(sys.D, ld * sizeof(double), A, (size_t)S * sizeof(double), (size_t)S * sizeof(double), LS,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    cudaError_t e = launch_factor<double>(sys, plan, ctl, st);
    if (e == cudaSuccess) e = launch_solve<double>(sys, plan, f, x, (double *)(base + o_g), ctl, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    Ctl h;
    if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    if (h.err_timeout) return XK_ETIMEOUT;
    if (h.err_singular) return XK_ESINGULAR;
    return XK_OK;
}
