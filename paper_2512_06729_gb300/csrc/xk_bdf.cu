// Kernels of the variable-order BDF integrator (the DLSODES family of Sec. 2.1): the predictor and
// the corrector's history terms, the checks and local-error estimates of a step attempt, and the
// acceptance.  The step's linear system is the backward-Euler system with dt = 1/c0 and the history
// terms subtracted from the right-hand side; the step controller runs on the host.
#include <cuda_runtime.h>

#include <cmath>

#include "xk_internal.cuh"

namespace xk {
namespace {

constexpr int kBdfThreads = 256;

__device__ __forceinline__ double combo(const double *Y, long long N, const BdfCombo &b, long long i)
{
    double v = 0.0;
    for (int j = 0; j < b.m; ++j) v += b.w[j] * Y[(long long)b.slot[j] * N + i];
    return v;
}

__global__ void k_bdf_predict(long long N, const double *Y, BdfStepArgs a, double *yhat, double *g)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double yh = combo(Y, N, a.pred, i);
        yhat[i] = yh;
        g[i] = a.c0 * yh + combo(Y, N, a.hist, i);
    }
}

__device__ __forceinline__ unsigned long long bits(double v) { return (unsigned long long)__double_as_longlong(v); }

__global__ void k_bdf_check(Col c, const double *Y, BdfStepArgs a, const double *yhat, const double *delta,
                            double *ynew, BdfResult *res)
{
    const long long N = (long long)c.L * c.S;
    unsigned long long e = 0, elo = 0, ehi = 0, rc = 0;
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / c.S);
        const double y = yhat[i] + delta[i];
        ynew[i] = y;
        const double ng = c.ngas[k];
        if (!isfinite(y) || y < -a.neg_tol * ng) bad = 1;
        if (y > a.f_floor * ng) {
            e = max(e, bits(fabs(y - yhat[i]) / (a.K * a.rtol * y)));
            if (a.lo.m) elo = max(elo, bits(fabs(y - combo(Y, N, a.lo, i)) / (a.Klo * a.rtol * y)));
            if (a.hi.m) ehi = max(ehi, bits(fabs(y - combo(Y, N, a.hi, i)) / (a.Khi * a.rtol * y)));
            rc = max(rc, bits(fabs(y - Y[(long long)a.newest * N + i]) / y));
        }
    }
    for (int o = 16; o; o >>= 1) {
        e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        elo = max(elo, __shfl_xor_sync(0xffffffffu, elo, o));
        ehi = max(ehi, __shfl_xor_sync(0xffffffffu, ehi, o));
        rc = max(rc, __shfl_xor_sync(0xffffffffu, rc, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (e) atomicMax(&res->err, e);
        if (elo) atomicMax(&res->err_lo, elo);
        if (ehi) atomicMax(&res->err_hi, ehi);
        if (rc) atomicMax(&res->relc, rc);
        if (bad) atomicExch(&res->bad, 1);
    }
}

__global__ void k_bdf_accept(long long N, const double *ynew, double *Yslot, double *n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double v = ynew[i] < 0.0 ? 0.0 : ynew[i];
        Yslot[i] = v;
        n[i] = v;
    }
}

int grid_for(long long N)
{
    long long b = (N + kBdfThreads - 1) / kBdfThreads;
    if (b > 152LL * 8) b = 152LL * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_bdf_predict(long long N, const double *Y, const BdfStepArgs &a, double *yhat, double *g, cudaStream_t st)
{
    k_bdf_predict<<<grid_for(N), kBdfThreads, 0, st>>>(N, Y, a, yhat, g);
    count_launches(1);
}

void launch_bdf_check(const Col &c, const double *Y, const BdfStepArgs &a, const double *yhat, const double *delta,
                      double *ynew, BdfResult *res, cudaStream_t st)
{
    k_bdf_check<<<grid_for((long long)c.L * c.S), kBdfThreads, 0, st>>>(c, Y, a, yhat, delta, ynew, res);
    count_launches(1);
}

void launch_bdf_accept(long long N, const double *ynew, double *Yslot, double *n, cudaStream_t st)
{
    k_bdf_accept<<<grid_for(N), kBdfThreads, 0, st>>>(N, ynew, Yslot, n);
    count_launches(1);
}

}  // namespace xk
