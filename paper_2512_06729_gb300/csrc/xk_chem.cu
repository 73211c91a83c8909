// Chemistry and transport rows of the implicit step: grid, thermochemistry,
// rate coefficients, photolysis, reaction rates and their derivatives,
// residual F(n) (Eq. 1 with the flux of Eq. 2), Jacobian blocks, the
// matrix-free Jacobian-vector product, and device-side step control.
#include <math.h>

#include <algorithm>

#include <atomic>

#include "xk_internal.cuh"

namespace xk {

namespace {

constexpr int kThreads = 256;

inline int nblocks(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }
// Grid of a kernel that a device flag may skip: a grid-stride loop over at most a few waves, so
// that a skipped launch (an FGMRES slot past convergence, an FP64 route not taken) schedules a
// few thousand threads, not one per element.
constexpr int kGatedBlocks = 152 * 8;
inline int gated_blocks(long long n, int t = kThreads) { return (int)std::min<long long>((n + t - 1) / t, kGatedBlocks); }

// ---------------------------------------------------------------------------
// grid (Sec. 2.1): n_gas = P / (k_B T); hydrostatic altitudes; layer widths
// ---------------------------------------------------------------------------
__global__ void k_grid(Col c)
{
    int L = c.L;
    for (int k = threadIdx.x; k < L; k += blockDim.x)
        c.ngas[k] = c.P[k] * kBarToCgs / (kBoltz * c.T[k]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double z = 0.0;
        c.z[0] = 0.0;
        for (int k = 0; k + 1 < L; ++k) {
            double Th = 0.5 * (c.T[k] + c.T[k + 1]);
            double H = kBoltz * Th / (c.mbar * kAmu * c.g);
            z = z + H * log(c.P[k] / c.P[k + 1]);
            c.z[k + 1] = z;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        if (k + 1 < L) c.dzi[k] = c.z[k + 1] - c.z[k];
        double w;
        if (L == 1) w = 1.0;
        else if (k == 0) w = c.z[1] - c.z[0];
        else if (k == L - 1) w = c.z[L - 1] - c.z[L - 2];
        else w = 0.5 * (c.z[k + 1] - c.z[k - 1]);
        c.dz[k] = w;
    }
}

// Eq. 2 at interface k+1/2: phi = u n_k - v n_{k+1}; eddy part in mixing-ratio
// form -K n_gas d(n/n_gas)/dz, molecular part -D (dn/dz + n (1/H_y + (1+alpha_T) T'/T)).
__global__ void k_transport(Col c)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int S = c.S;
    if (idx >= (long long)(c.L - 1) * S) return;
    int k = (int)(idx / S), y = (int)(idx % S);
    double Th = 0.5 * (c.T[k] + c.T[k + 1]);
    double nh = 0.5 * (c.ngas[k] + c.ngas[k + 1]);
    double Kh = 0.5 * (c.Kzz[k] + c.Kzz[k + 1]);
    double h = c.dzi[k];
    double dTdz = (c.T[k + 1] - c.T[k]) / h;
    double D = c.dcoef[y] * pow(Th, 0.75) / nh;
    double Hy = kBoltz * Th / (c.mass[y] * kAmu * c.g);
    double a = 1.0 / Hy + (1.0 + c.alpha_T) * dTdz / Th;
    c.u[idx] = Kh * nh / (h * c.ngas[k]) + D * (1.0 / h - 0.5 * a);
    c.v[idx] = Kh * nh / (h * c.ngas[k + 1]) + D * (1.0 / h + 0.5 * a);
}

// ---------------------------------------------------------------------------
// thermochemistry (Appendix A) and rate coefficients (Sec. 2.3)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double gibbs_rt(const double *nasa15, double T)
{
    const double *a = (T < nasa15[0]) ? nasa15 + 1 : nasa15 + 8;
    return a[0] * (1.0 - log(T)) - a[1] * T / 2.0 - a[2] * T * T / 6.0
         - a[3] * T * T * T / 12.0 - a[4] * T * T * T * T / 20.0 + a[5] / T - a[6];
}

__global__ void k_gibbs(Col c)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.S) return;
    int k = (int)(idx / c.S), y = (int)(idx % c.S);
    c.grt[idx] = gibbs_rt(c.nasa + 15 * y, c.T[k]);
}

__device__ __forceinline__ double arrh(double al, double be, double ga, double T, int form)
{
    double Tb = (form == 0) ? T / 300.0 : T;
    return al * pow(Tb, be) * exp(-ga / T);
}

__device__ __forceinline__ double troe_f(const double *tr, double T, double Pr)
{
    if (tr[0] == 0.0 || Pr <= 0.0) return 1.0;
    double Fc = (1.0 - tr[0]) * exp(-T / tr[1]) + tr[0] * exp(-T / tr[2]);
    if (tr[3] != 0.0) Fc += exp(-tr[3] / T);
    double lFc = log10(Fc);
    double cc = -0.4 - 0.67 * lFc;
    double N = 0.75 - 1.27 * lFc;
    double x = log10(Pr) + cc;
    double q = x / (N - 0.14 * x);
    return pow(10.0, lFc / (1.0 + q * q));
}

// k_f, k_r and ln K_c per (layer, reaction); ln K_c = -sum nu G/RT + dnu ln(p0 / k_B T).
__global__ void k_rates(Col c)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.R) return;
    int k = (int)(idx / c.R), r = (int)(idx % c.R);
    double T = c.T[k];
    int t = c.rtype[r];
    const double *grt = c.grt + (long long)k * c.S;
    double dG = 0.0;
    int dnu = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        int i = c.reac[3 * r + s];
        if (i >= 0) { dG -= grt[i]; dnu -= 1; }
        int j = c.prod[3 * r + s];
        if (j >= 0) { dG += grt[j]; dnu += 1; }
    }
    double lnk = (t == XK_RX_PHOTO) ? 0.0 : -dG + dnu * log(kP0 / (kBoltz * T));
    const double *a = c.arr + 9 * r;
    double f = 0.0, b = 0.0;
    if (t == XK_RX_TWO_BODY) {
        f = arrh(a[0], a[1], a[2], T, c.form[r]);
    } else if (t == XK_RX_THREE_BODY) {
        double k0 = arrh(a[3], a[4], a[5], T, c.form[r]);
        double ki = arrh(a[6], a[7], a[8], T, c.form[r]);
        double M = c.ngas[k];
        double Pr = k0 * M / ki;
        f = k0 * M / (1.0 + k0 * M / ki) * troe_f(c.troe + 4 * r, T, Pr);
    }
    if (t != XK_RX_PHOTO) b = f / exp(lnk);
    c.kf[idx] = f;
    c.kr[idx] = b;
    if (c.lnkc) c.lnkc[idx] = lnk;
}

// ---------------------------------------------------------------------------
// photolysis (Sec. 2.3.3): extinction by absorption and Rayleigh scattering, direct beam with the
// optical depth to the layer midpoint, and optionally the diffuse field J_diff = (J_up + J_down) / 2
// ---------------------------------------------------------------------------
constexpr int kExtLayers = 4;   // layers per thread of the extinction sums (sigma loaded once for them)

// alpha (absorption) and alpha_s (scattering) per (layer, wavelength): one thread per wavelength and
// kExtLayers consecutive layers, reading each cross section once for all of them (coalesced in w)
__global__ void k_photo_alpha(Col c, const double *n)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int k0 = blockIdx.y * kExtLayers;
    if (w >= c.W) return;
    const int nk = min(kExtLayers, c.L - k0);
    double sa[kExtLayers], ss[kExtLayers];
#pragma unroll
    for (int j = 0; j < kExtLayers; ++j) sa[j] = ss[j] = 0.0;
    for (int i = 0; i < c.Sabs; ++i) {
        const double sg = c.sig_abs[(long long)i * c.W + w];
        const int y = c.abs_sp[i];
#pragma unroll
        for (int j = 0; j < kExtLayers; ++j)
            if (j < nk) sa[j] += sg * n[(long long)(k0 + j) * c.S + y];
    }
    for (int i = 0; i < c.Ssca; ++i) {
        const double sg = c.sig_sca[(long long)i * c.W + w];
        const int y = c.sca_sp[i];
#pragma unroll
        for (int j = 0; j < kExtLayers; ++j)
            if (j < nk) ss[j] += sg * n[(long long)(k0 + j) * c.S + y];
    }
#pragma unroll
    for (int j = 0; j < kExtLayers; ++j)
        if (j < nk) {
            c.alpha[(long long)(k0 + j) * c.W + w] = sa[j];
            c.alpha_s[(long long)(k0 + j) * c.W + w] = ss[j];
        }
}

// One thread per wavelength.  Top-down: optical depth, direct beam into Jw and, with the diffuse
// field, the two-stream recursion.  In layer k the diffuse fluxes leaving it, D_k down through its
// bottom and U_k up through its top, obey
//     D_k = T_k D_{k+1} + r_k U_{k-1} + P_k / 2,   U_k = T_k U_{k-1} + r_k D_{k+1} + P_k / 2,
// with D_L = 0 and U_{-1} = albedo (D_0 + beam at the bottom); r_k = (1 - t) omega / 2,
// T_k = t + (1 - t) omega / 2, t = exp(-2 dtau_k), omega_k = dtau_s / dtau, and P_k = omega_k mu J0
// (e^{-tau_top/mu} - e^{-tau_bot/mu}) the beam photons the layer scatters.  Going down, each layer's
// fluxes are written in terms of the flux entering from below: D_k = p_k U_{k-1} + h0_k,
// U_k = q_k U_{k-1} + h1_k (p_k is the reflectance of the layers from k up, as in the adding
// method); going up, U_{-1} is found from the boundary and the fluxes follow layer by layer.
__global__ void k_photo_J(Col c)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= c.W) return;
    const long long LW = (long long)c.L * c.W;
    const double J0 = c.J0[w], mu = c.mu;
    double above = 0.0, pn = 0.0, h0n = 0.0;
    for (int k = c.L - 1; k >= 0; --k) {
        const long long i = (long long)k * c.W + w;
        const double ta = c.alpha[i] * c.dz[k], ts = c.alpha_s[i] * c.dz[k];
        const double dt = ta + ts;
        c.Jw[i] = J0 * exp(-(above + 0.5 * dt) / mu);
        if (c.diffuse) {
            const double om = dt > 0.0 ? ts / dt : 0.0;
            const double t = exp(-dt / 0.5);
            const double r = (1.0 - t) * om / 2.0, T = t + (1.0 - t) * om / 2.0;
            const double P = om * mu * J0 * (exp(-above / mu) - exp(-(above + dt) / mu));
            const double den = 1.0 - r * pn;
            const double q = T / den, h1 = (r * h0n + P / 2.0) / den;
            const double p = r + T * pn * q;
            const double h0 = T * pn * h1 + T * h0n + P / 2.0;
            c.rt[i] = p;
            c.rt[LW + i] = q;
            c.rt[2 * LW + i] = h0;
            c.rt[3 * LW + i] = h1;
            pn = p;
            h0n = h0;
        }
        above += dt;
    }
    if (!c.diffuse) return;
    const double A = c.albedo;
    const double bottom = mu * J0 * exp(-above / mu);
    // U_{-1} = A (D_0 + bottom), D_0 = p_0 U_{-1} + h0_0
    double Ub = A * (c.rt[2 * LW + w] + bottom) / (1.0 - A * c.rt[w]);
    for (int k = 0; k < c.L; ++k) {
        const long long i = (long long)k * c.W + w;
        const double Dk = c.rt[i] * Ub + c.rt[2 * LW + i];
        const double Uk = c.rt[LW + i] * Ub + c.rt[3 * LW + i];
        double Dn = 0.0;
        if (k + 1 < c.L) Dn = c.rt[i + c.W] * Uk + c.rt[2 * LW + i + c.W];
        const double up = 0.5 * (Ub + Uk), dn = 0.5 * (Dk + Dn);
        c.Jw[i] += 0.5 * (up + dn);
        Ub = Uk;
    }
}

// Direct beam only: one warp per wavelength.  Lane l takes a run of consecutive layers counted
// from the top, sums their optical thicknesses, and a warp scan gives the optical depth above its
// run; the lane then walks its run (32x the parallelism of a thread per wavelength, which left
// 1,000 bins on 8 SMs).
__global__ void k_photo_J_direct(Col c)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    const int per = (c.L + 31) / 32;
    const int i0 = lane * per, i1 = min(c.L, i0 + per);   // positions from the top: layer L-1-i
    double run = 0.0;
    for (int i = i0; i < i1; ++i) {
        const int k = c.L - 1 - i;
        const long long idx = (long long)k * c.W + w;
        run += (c.alpha[idx] + c.alpha_s[idx]) * c.dz[k];
    }
    double incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    double above = __shfl_up_sync(0xffffffffu, incl, 1);   // sum over the runs above this one
    if (lane == 0) above = 0.0;
    const double J0 = c.J0[w], mu = c.mu;
    for (int i = i0; i < i1; ++i) {
        const int k = c.L - 1 - i;
        const long long idx = (long long)k * c.W + w;
        const double dt = (c.alpha[idx] + c.alpha_s[idx]) * c.dz[k];
        c.Jw[idx] = J0 * exp(-(above + 0.5 * dt) / mu);
        above += dt;
    }
}

// k_ph = t_f sum_w J(k, w) sigma(w) dlambda(w); one warp per (layer, reaction), lanes striding
// the wavelengths (coalesced), partial sums added in lane order
__global__ void k_photo_k(Col c)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= c.L * c.Rph) return;
    int k = warp / c.Rph, q = warp % c.Rph;
    const double *J = c.Jw + (long long)k * c.W;
    const double *sg = c.sigma + (long long)q * c.W;
    double s = 0.0;
    for (int w = lane; w < c.W; w += 32)
        s += J[w] * sg[w] * c.dlam[w];
    double tot = 0.0;
    for (int l = 0; l < 32; ++l) {
        double v = __shfl_sync(0xffffffffu, s, l);
        tot += v;
    }
    if (lane == 0) c.kph[(long long)k * c.Rph + q] = c.tf * tot;
}

// ---------------------------------------------------------------------------
// reaction rates w = k_f prod n_reac - k_r prod n_prod and partial derivatives
// d[slot] = d(k_f prod n_reac)/d n_reac[slot] (slots 0-2) and
//           -d(k_r prod n_prod)/d n_prod[slot] (slots 3-5)
// ---------------------------------------------------------------------------
__global__ void k_reaction_terms(Col c, const double *n)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.R) return;
    int k = (int)(idx / c.R), r = (int)(idx % c.R);
    reaction_terms_at(c, k, r, n + (long long)k * c.S, c.w + idx, c.d + idx * 6);
}

// F = sum_r nu w_r - (phi_{k+1/2} - phi_{k-1/2}) / dz_k; also the solve scaling
// s = max(n, f_floor n_gas) and the scaled right-hand side b = F / s.
__global__ void k_residual(Col c, const double *n, double *F, const Ctl *ctl, double f_floor)
{
    if (ctl && ctl->finished) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int S = c.S, L = c.L;
    if (idx >= (long long)L * S) return;
    int k = (int)(idx / S), y = (int)(idx % S);
    const double *wk = c.w + (long long)k * c.R;
    double f = 0.0;
    for (int e = c.yp[y]; e < c.yp[y + 1]; ++e) {
        int code = c.yent[e];
        int r = code >> 4;
        int nu = (code & 15) - 8;
        if (nu < 0) f -= wk[r];
        else f += wk[r];
    }
    double nk = n[idx];
    double upf = 0.0, dnf = 0.0;
    if (k + 1 < L) upf = c.u[(long long)k * S + y] * nk - c.v[(long long)k * S + y] * n[idx + S];
    if (k > 0) dnf = c.u[(long long)(k - 1) * S + y] * n[idx - S] - c.v[(long long)(k - 1) * S + y] * nk;
    f += -(upf - dnf) / c.dz[k];
    if (c.fshift) f -= c.fshift[idx];
    F[idx] = f;
    if (c.s) {
        double sc = fmax(nk, f_floor * c.ngas[k]);
        c.s[idx] = sc;
        c.b[idx] = f / sc;
        if (c.rs) c.rs[idx] = 1.0 / sc;
    }
}

// Dense diagonal blocks A_k = I/dt - dF_k/dn_k, couplings lo/up; one warp per row.
// Contributions are summed in a fixed order (deterministic).  scaled != 0 writes
// diag(1/s) A diag(s) and the matching couplings.
template <typename T>
__global__ void k_jacobian(Col c, const double *n, const Ctl *ctl, double dt_override, int scaled,
                           T *A, T *lo, T *up, double *dout, const int *skip, long long lstride)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    extern __shared__ double sh[];
    const int S = c.S, L = c.L;
    const int wpb = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *rowbuf = sh + (long long)warp * (S + 64);
    const double dt = dt_override > 0.0 ? dt_override : ctl->dt;
    for (long long row = (long long)blockIdx.x * wpb + warp; row < (long long)L * S; row += (long long)gridDim.x * wpb) {
        const int k = (int)(row / S), i = (int)(row % S);
        __syncwarp();
        for (int j = lane; j < S; j += 32) rowbuf[j] = 0.0;
        __syncwarp();
        const double *dk = c.d + (long long)k * c.R * 6;
        // each lane owns whole column entries and sums their terms in a fixed order (deterministic)
        for (int q = c.jp[i] + lane; q < c.jp[i + 1]; q += 32) {
            double acc = 0.0;
            for (int t = c.jtp[q]; t < c.jtp[q + 1]; ++t) {
                const int code = c.jrs[t];
                const int rs = code >> 1;
                const double dv = dk[(long long)(rs >> 3) * 6 + (rs & 7)];
                acc += (code & 1) ? dv : -dv;
            }
            rowbuf[c.jcol[q]] = acc;
        }
        __syncwarp();
        const double *sk = c.s + (long long)k * S;
        if (lane == 0) {
            rowbuf[i] += 1.0 / dt + c.tdg[row];
            if (dout) dout[row] = fmax(fabs(rowbuf[i]), 1.0 / dt);
            double lov = c.tlo[row];
            double upv = c.tup[row];
            if (scaled) {
                if (k > 0) lov *= c.s[(long long)(k - 1) * S + i] / sk[i];
                if (k + 1 < L) upv *= c.s[(long long)(k + 1) * S + i] / sk[i];
            }
            lo[row] = (T)lov;
            up[row] = (T)upv;
        }
        __syncwarp();
        T *Ar = A + (long long)k * (lstride > 0 ? lstride : (long long)S * c.ld) + (long long)i * c.ld;
        if (scaled) {
            double inv = 1.0 / sk[i];
            for (int j = lane; j < S; j += 32) Ar[j] = (T)(rowbuf[j] * sk[j] * inv);
        } else {
            for (int j = lane; j < S; j += 32) Ar[j] = (T)rowbuf[j];
        }
        for (int j = S + lane; j < c.ld; j += 32) Ar[j] = (T)0;
    }
}

// y = diag(1/s) (I/dt - J) diag(s) x, matrix-free from the reaction derivatives (FP64), in two
// passes.  First the directional derivative of every rate along v = s x:
//   dw[k][r] = sum over the reaction's slots of d[k][r][slot] v[k][species(slot)]
// (d holds d(k_f prod n_reac)/dn and -d(k_r prod n_prod)/dn, so dw is the change of w_r);
// then per species (J v)_i = sum_r nu_ir dw_r through the species-major stoichiometry, a warp
// per row, plus the transport terms.
// ---------------------------------------------------------------------------
// photolysis rates in the Jacobian (cfg.photo_jacobian): the change of k_ph along the physical
// direction v = s x of J v.  The direct beam J = J0 exp(-tau/mu) changes by -J dtau/mu, with dtau
// the optical depth of the extinction change sum_i sigma_i v_i above the layer (half the layer's
// own), so dk_ph = t_f sum_w dJ sigma dlambda; the rate w = k_ph n_A then changes by dk_ph n_A.
// ---------------------------------------------------------------------------
__global__ void k_photo_beta(Col c, const Ctl *ctl, const double *x, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int k0 = blockIdx.y * kExtLayers;
    if (w >= c.W) return;
    const int nk = min(kExtLayers, c.L - k0);
    double sb[kExtLayers];
#pragma unroll
    for (int j = 0; j < kExtLayers; ++j) sb[j] = 0.0;
    for (int i = 0; i < c.Sabs; ++i) {
        const double sg = c.sig_abs[(long long)i * c.W + w];
        const int y = c.abs_sp[i];
#pragma unroll
        for (int j = 0; j < kExtLayers; ++j)
            if (j < nk) {
                const long long e = (long long)(k0 + j) * c.S + y;
                sb[j] += sg * c.s[e] * x[e];
            }
    }
    for (int i = 0; i < c.Ssca; ++i) {
        const double sg = c.sig_sca[(long long)i * c.W + w];
        const int y = c.sca_sp[i];
#pragma unroll
        for (int j = 0; j < kExtLayers; ++j)
            if (j < nk) {
                const long long e = (long long)(k0 + j) * c.S + y;
                sb[j] += sg * c.s[e] * x[e];
            }
    }
#pragma unroll
    for (int j = 0; j < kExtLayers; ++j)
        if (j < nk) c.pbeta[(long long)(k0 + j) * c.W + w] = sb[j];
}

// one warp per wavelength, the same run-and-scan layout as the direct beam
__global__ void k_photo_dJ(Col c, const Ctl *ctl, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    const int per = (c.L + 31) / 32;
    const int i0 = lane * per, i1 = min(c.L, i0 + per);
    double run = 0.0;
    for (int i = i0; i < i1; ++i) {
        const int k = c.L - 1 - i;
        run += c.pbeta[(long long)k * c.W + w] * c.dz[k];
    }
    double incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    double above = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) above = 0.0;
    for (int i = i0; i < i1; ++i) {
        const int k = c.L - 1 - i;
        const long long idx = (long long)k * c.W + w;
        const double db = c.pbeta[idx] * c.dz[k];
        c.pdJ[idx] = -c.Jw[idx] * (above + 0.5 * db) / c.mu;
        above += db;
    }
}

// dk_ph = t_f sum_w dJ sigma dlambda; one warp per (layer, reaction)
__global__ void k_photo_dk(Col c, const Ctl *ctl, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= c.L * c.Rph) return;
    const int k = warp / c.Rph, q = warp % c.Rph;
    const double *dJ = c.pdJ + (long long)k * c.W;
    const double *sg = c.sigma + (long long)q * c.W;
    double s = 0.0;
    for (int w = lane; w < c.W; w += 32) s += dJ[w] * sg[w] * c.dlam[w];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) c.pdk[(long long)k * c.Rph + q] = c.tf * s;
}

// the photolysis rate's extra change along v (0 unless photo_jacobian): dk_ph n_A
__device__ __forceinline__ double photo_jv_term(const Col &c, int k, int r)
{
    if (!c.photo_jac || c.rtype[r] != XK_RX_PHOTO) return 0.0;
    return c.pdk[(long long)k * c.Rph + c.prow[r]] * c.n[(long long)k * c.S + c.reac[3 * r]];
}

__global__ void k_jv_rates(Col c, const Ctl *ctl, const double *x, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)c.L * c.R;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / c.R), r = (int)(idx % c.R);
        const double *d = c.d + idx * 6;
        const double *sk = c.s + (long long)k * c.S, *xk = x + (long long)k * c.S;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int i = c.reac[3 * r + q];
            if (i >= 0) acc += d[q] * sk[i] * xk[i];
            const int j = c.prod[3 * r + q];
            if (j >= 0) acc += d[3 + q] * sk[j] * xk[j];
        }
        c.dw[idx] = acc + photo_jv_term(c, k, r);
    }
}

__device__ __forceinline__ void jv_row(const Col &c, const Ctl *ctl, const double *x, double *y, const double *rowdiv,
                                       int warp, int lane);
__device__ __forceinline__ void jv_finish(const Col &c, const Ctl *ctl, const double *x, double *y,
                                          const double *rowdiv, int k, int i, double acc);

// The same J v in one launch with one CTA per layer: the layer's R directional rate derivatives are
// formed in shared memory, then each species sums its stoichiometric entries from there (the
// gathers hit shared memory instead of L1).  For networks whose R doubles fit shared memory.
__global__ void k_jv_layer(Col c, const Ctl *ctl, const double *x, double *y, const double *rowdiv, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    extern __shared__ double dws[];
    const int S = c.S, R = c.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = blockIdx.x; k < c.L; k += gridDim.x) {
        const double *sk = c.s + (long long)k * S, *xk = x + (long long)k * S;
        const double *dk = c.d + (long long)k * R * 6;
        __syncthreads();
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            const double *d = dk + (long long)r * 6;
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int a = c.reac[3 * r + q];
                if (a >= 0) acc += d[q] * sk[a] * xk[a];
                const int b = c.prod[3 * r + q];
                if (b >= 0) acc += d[3 + q] * sk[b] * xk[b];
            }
            dws[r] = acc + photo_jv_term(c, k, r);
        }
        __syncthreads();
        for (int i = warp; i < S; i += nw) {
            double acc = 0.0;
            for (int e = c.yp[i] + lane; e < c.yp[i + 1]; e += 32) {
                const int code = c.yent[e];
                const double v = dws[code >> 4];
                acc += ((code & 15) - 8 < 0) ? v : -v;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) jv_finish(c, ctl, x, y, rowdiv, k, i, acc);
        }
    }
}

__global__ void k_jv(Col c, const Ctl *ctl, const double *x, double *y, const double *rowdiv, const int *skip)
{
    if ((ctl && ctl->finished) || (skip && *skip)) return;
    const int S = c.S, L = c.L;
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); warp < L * S; warp += nwarps)
        jv_row(c, ctl, x, y, rowdiv, warp, lane);
}

__device__ __forceinline__ void jv_row(const Col &c, const Ctl *ctl, const double *x, double *y, const double *rowdiv,
                                       int warp, int lane)
{
    const int S = c.S, L = c.L;
    int k = warp / S, i = warp % S;
    const double *dwk = c.dw + (long long)k * c.R;
    const double *sk = c.s + (long long)k * S;
    const double *xk = x + (long long)k * S;
    double acc = 0.0;
    for (int e = c.yp[i] + lane; e < c.yp[i + 1]; e += 32) {
        const int code = c.yent[e];
        const double v = dwk[code >> 4];
        acc += ((code & 15) - 8 < 0) ? v : -v;       // -(nu) dw: reactant rows +, product rows -
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) jv_finish(c, ctl, x, y, rowdiv, k, i, acc);
    (void)sk;
    (void)xk;
}

// Row (k, i) of y from the chemistry sum acc = -(J diag(s) x)_i: scaling, I/dt and transport.
__device__ __forceinline__ void jv_finish(const Col &c, const Ctl *ctl, const double *x, double *y,
                                          const double *rowdiv, int k, int i, double acc)
{
    const int S = c.S, L = c.L;
    const long long q = (long long)k * S + i;
    const double ri = c.rs[q];
    double r = acc * ri + (1.0 / ctl->dt + c.tdg[q]) * x[q];
    if (k > 0) r += c.tlo[q] * c.s[q - S] * ri * x[q - S];
    if (k + 1 < L) r += c.tup[q] * c.s[q + S] * ri * x[q + S];
    if (rowdiv) r /= rowdiv[q];
    y[q] = r;
}

// y = x / d (row equilibration of a right-hand side)
__global__ void k_rowdiv(long long N, const double *x, const double *d, double *y)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < N) y[idx] = x[idx] / d[idx];
}

__global__ void k_unscale(Col c, const double *xs, double *delta)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.S) return;
    delta[idx] = xs[idx] * c.s[idx];
}

// ---------------------------------------------------------------------------
// step control on the device
// ---------------------------------------------------------------------------
__global__ void k_check(Col c, Ctl *ctl, Policy pol)
{
    if (ctl->finished) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int S = c.S;
    double rel = 0.0;
    int bad = 0, neg = 0;
    if (idx < (long long)c.L * S) {
        int k = (int)(idx / S);
        double nv = c.n[idx], dv = c.delta[idx];
        double nn = nv + dv;
        double ng = c.ngas[k];
        if (!isfinite(nn)) bad = 1;
        else {
            if (nn < -pol.neg_tol * ng) bad = 1;
            if (nn < 0.0) neg = 1;
            if (nv > pol.f_floor * ng) rel = fabs(dv) / nv;
        }
    }
    // warp-level combine, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rel = fmax(rel, __shfl_xor_sync(0xffffffffu, rel, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        neg += __shfl_xor_sync(0xffffffffu, neg, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (rel > 0.0) atomicMax(&ctl->max_rel_bits, (unsigned long long)__double_as_longlong(rel));
        if (bad) atomicOr(&ctl->bad, 1);
        if (neg) atomicAdd(&ctl->n_neg, neg);
    }
}

// Mixed precision routing at the start of a step: steps at dt at or above the
// smallest dt where the FP32-preconditioned solve failed go straight to FP64.
__global__ void k_route(Ctl *ctl)
{
    ctl->skip32 = ctl->dt >= ctl->dt_fp64 ? 1 : 0;
    const int reuse = ctl->skip32 && ctl->have64 && ctl->reuse_enabled;
    ctl->skip_reuse = reuse ? 0 : 1;
    ctl->skip64 = (ctl->skip32 && !reuse) ? 0 : 1;
    ctl->used_fp64 = ctl->skip32;
}

// Diagonal of I/dt - dF/dn per (layer, species), from the reaction derivatives and transport.
__global__ void k_diag(Col c, const Ctl *ctl, double *diag)
{
    if (ctl->finished) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int S = c.S, L = c.L;
    if (idx >= (long long)L * S) return;
    int k = (int)(idx / S), i = (int)(idx % S);
    const double *dk = c.d + (long long)k * c.R * 6;
    double acc = 0.0;
    const int q = c.jdq[i];
    if (q >= 0)
        for (int t = c.jtp[q]; t < c.jtp[q + 1]; ++t) {
            const int code = c.jrs[t];
            const int rs = code >> 1;
            const double dv = dk[(long long)(rs >> 3) * 6 + (rs & 7)];
            acc += (code & 1) ? dv : -dv;
        }
    double dg = 1.0 / ctl->dt + acc;
    if (k + 1 < L) dg += c.u[(long long)k * S + i] / c.dz[k];
    if (k > 0) dg += c.v[(long long)(k - 1) * S + i] / c.dz[k];
    diag[idx] = fmax(fabs(dg), 1.0 / ctl->dt);
}

// Scalings of the reused FP64 factorization: input rowd * s / s64, output s64 / s.
__global__ void k_reuse_scales(long long N, const double *rowd, const double *s, const double *s64, double *pin,
                               double *pout, const Ctl *ctl)
{
    if (ctl->finished || ctl->skip_reuse) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    pin[idx] = rowd[idx] * s[idx] / s64[idx];
    pout[idx] = s64[idx] / s[idx];
}

// After an FP64 factorization: remember its scaling, mark the factors valid.
__global__ void k_after_refactor(long long N, const double *s, double *s64, Ctl *ctl)
{
    if (ctl->finished || ctl->skip64) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < N) s64[idx] = s[idx];
    if (idx == 0) {
        ctl->have64 = 1;
        ctl->refactors += 1;
    }
}

__global__ void k_begin(Ctl *ctl)
{
    if (ctl->finished) {
        ctl->accepted = 0;
        return;
    }
    ctl->max_rel_bits = 0ull;
    ctl->solver_iters = 0;
    ctl->solver_resid = 0.0;
    ctl->bad = 0;
    ctl->n_neg = 0;
    ctl->accepted = 0;
    ctl->converged = 0;
}

__global__ void k_decide(Ctl *ctl, Policy pol)
{
    if (ctl->finished) return;
    double dt = ctl->dt;
    double maxrel = __longlong_as_double((long long)ctl->max_rel_bits);
    int ok = !ctl->bad && !ctl->err_singular && !ctl->err_timeout;
    if (ok && maxrel > pol.rel_reject) ok = 0;
    ctl->max_rel = maxrel;
    ctl->last_dt = dt;
    ctl->steps += 1;
    if (ctl->used_fp64) ctl->fp64_steps += 1;
    if (ok) {
        double fac = (maxrel > 0.0) ? pol.rel_target / maxrel : pol.grow_max;
        if (fac > pol.grow_max) fac = pol.grow_max;
        if (fac < pol.shrink_min) fac = pol.shrink_min;
        double dn = dt * fac;
        ctl->dt_next = (dn > pol.dt_max) ? pol.dt_max : dn;
        ctl->accepted = 1;
        ctl->n_acc += 1;
        ctl->t += dt;
        if (dt >= pol.ss_dt && maxrel < pol.ss_tol) {
            ctl->converged = 1;
            ctl->finished = 1;
        }
    } else {
        ctl->dt_next = 0.5 * dt;
        ctl->accepted = 0;
        ctl->n_neg = 0;
        ctl->n_rej += 1;
        if (ctl->err_timeout) { ctl->status = XK_ETIMEOUT; ctl->finished = 1; }
        else if (ctl->dt_next < pol.dt_min) { ctl->status = XK_ENEG; ctl->finished = 1; }
    }
    ctl->dt = ctl->dt_next;
}

// n <- max(n + delta, 0) on an accepted step (reads the decision of this step).
__global__ void k_apply(Col c, Ctl *ctl)
{
    if (!ctl->accepted) return;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.S) return;
    double nn = c.n[idx] + c.delta[idx];
    c.n[idx] = nn < 0.0 ? 0.0 : nn;
}

__global__ void k_set_mixing(Col c, const double *f, double *n)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.L * c.S) return;
    n[idx] = f[idx] * c.ngas[idx / c.S];
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

__global__ void k_convert32(const double *src, size_t lds, float *dst, size_t ldd, size_t rows, size_t cols)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(rows * cols)) return;
    size_t r = idx / cols, j = idx - r * cols;
    dst[r * ldd + j] = (float)src[r * lds + j];
}

void launch_convert32(const double *src, size_t lds, float *dst, size_t ldd, size_t rows, size_t cols, cudaStream_t st)
{
    if (rows * cols == 0) return;
    count_launches(1);
    k_convert32<<<nblocks((long long)(rows * cols)), kThreads, 0, st>>>(src, lds, dst, ldd, rows, cols);
}

void launch_set_mixing(const Col &c, const double *f, double *n, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_set_mixing<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, f, n); }
}

// ---------------------------------------------------------------------------
// Transport terms of the rows of I/dt - dF/dn (the same quotients k_jacobian forms per row).
__global__ void k_transport_rows(Col c)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int S = c.S, L = c.L;
    if (idx >= (long long)L * S) return;
    const int k = (int)(idx / S), i = (int)(idx % S);
    double dg = 0.0;
    if (k + 1 < L) dg += c.u[(long long)k * S + i] / c.dz[k];
    if (k > 0) dg += c.v[(long long)(k - 1) * S + i] / c.dz[k];
    c.tdg[idx] = dg;
    c.tlo[idx] = (k > 0) ? -c.u[(long long)(k - 1) * S + i] / c.dz[k] : 0.0;
    c.tup[idx] = (k + 1 < L) ? -c.v[(long long)k * S + i] / c.dz[k] : 0.0;
}

void launch_transport_coeffs(const Col &c, const double *Kzz, double *u, double *v, cudaStream_t st)
{
    if (c.L < 2) return;
    Col t = c;
    t.Kzz = Kzz;
    t.u = u;
    t.v = v;
    count_launches(1);
    k_transport<<<nblocks((long long)(c.L - 1) * c.S), kThreads, 0, st>>>(t);
}

void launch_grid(const Col &c, cudaStream_t st)
{
    count_launches(1); k_grid<<<1, 256, 0, st>>>(c);
    if (c.L > 1) { count_launches(1); k_transport<<<nblocks((long long)(c.L - 1) * c.S), kThreads, 0, st>>>(c); }
    if ((long long)c.L * c.S > 0) { count_launches(1); k_transport_rows<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c); }
}

void launch_thermo(const Col &c, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_gibbs<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c); }
}

void launch_rates(const Col &c, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_gibbs<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c); }
    if (((long long)c.L * c.R) > 0) { count_launches(1); k_rates<<<nblocks((long long)c.L * c.R), kThreads, 0, st>>>(c); }
}

void launch_photolysis(const Col &c, const double *n, cudaStream_t st)
{
    if (c.Rph == 0) return;
    if (c.W > 0) {
        if (c.L > 0) {
            count_launches(1);
            dim3 grid(nblocks(c.W, 128), (c.L + kExtLayers - 1) / kExtLayers);
            k_photo_alpha<<<grid, 128, 0, st>>>(c, n);
        }
        count_launches(1);
        if (c.diffuse) k_photo_J<<<nblocks(c.W, 64), 64, 0, st>>>(c);   // 10,000 bins: 157 CTAs, every SM
        else k_photo_J_direct<<<nblocks((long long)c.W * 32, 128), 128, 0, st>>>(c);
    }
    if (((long long)c.L * c.Rph * 32) > 0) { count_launches(1); k_photo_k<<<nblocks((long long)c.L * c.Rph * 32), kThreads, 0, st>>>(c); }
}

void launch_reaction_terms(const Col &c, const double *n, cudaStream_t st)
{
    if (((long long)c.L * c.R) > 0) { count_launches(1); k_reaction_terms<<<nblocks((long long)c.L * c.R), kThreads, 0, st>>>(c, n); }
}

void launch_residual(const Col &c, const double *n, double *F, const Ctl *ctl, double f_floor, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_residual<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, n, F, ctl, f_floor); }
}

static size_t jac_smem(const Col &c, int wpb)
{
    return (size_t)wpb * ((size_t)(c.S + 64) * sizeof(double));
}

void launch_jacobian64(const Col &c, const double *n, const Ctl *ctl, double dt_override, int scaled,
                       double *A, double *lo, double *up, cudaStream_t st, const int *skip)
{
    const int wpb = 4;
    size_t sm = jac_smem(c, wpb);
    cudaFuncSetAttribute(k_jacobian<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_jacobian<double><<<skip ? gated_blocks((long long)c.L * c.S, wpb) : nblocks((long long)c.L * c.S, wpb), wpb * 32, sm, st>>>(c, n, ctl, dt_override, scaled, A, lo, up, nullptr, skip, 0); }
}

void launch_jacobian32(const Col &c, const double *n, const Ctl *ctl, float *A, float *lo, float *up, double *diag,
                       cudaStream_t st, const int *skip, long long lstride)
{
    const int wpb = 4;
    size_t sm = jac_smem(c, wpb);
    cudaFuncSetAttribute(k_jacobian<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_jacobian<float><<<skip ? gated_blocks((long long)c.L * c.S, wpb) : nblocks((long long)c.L * c.S, wpb), wpb * 32, sm, st>>>(c, n, ctl, 0.0, 1, A, lo, up, diag, skip, lstride); }
}

void launch_jv(const Col &c, const Ctl *ctl, const double *xs, double *ys, const double *rowdiv, const int *skip,
               cudaStream_t st)
{
    if ((long long)c.L * c.S <= 0) return;
    if (c.photo_jac) {
        count_launches(3);
        dim3 grid(nblocks(c.W, 128), (c.L + kExtLayers - 1) / kExtLayers);
        k_photo_beta<<<grid, 128, 0, st>>>(c, ctl, xs, skip);
        k_photo_dJ<<<nblocks((long long)c.W * 32, 128), 128, 0, st>>>(c, ctl, skip);
        k_photo_dk<<<nblocks((long long)c.L * c.Rph * 32), kThreads, 0, st>>>(c, ctl, skip);
    }
    const size_t sm = (size_t)std::max(c.R, 1) * sizeof(double);
    if (sm <= 160 * 1024) {
        static size_t attr = 0;
        if (sm > attr) {
            cudaFuncSetAttribute(k_jv_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(160 * 1024));
            attr = 160 * 1024;
        }
        count_launches(1);
        k_jv_layer<<<std::min(c.L, kGatedBlocks), 512, sm, st>>>(c, ctl, xs, ys, rowdiv, skip);
        return;
    }
    if (((long long)c.L * c.R) > 0) { count_launches(1); k_jv_rates<<<gated_blocks((long long)c.L * c.R), kThreads, 0, st>>>(c, ctl, xs, skip); }
    count_launches(1);
    k_jv<<<gated_blocks((long long)c.L * c.S * 32), kThreads, 0, st>>>(c, ctl, xs, ys, rowdiv, skip);
}

void launch_rowdiv(long long N, const double *x, const double *d, double *y, cudaStream_t st)
{
    if (N > 0) { count_launches(1); k_rowdiv<<<nblocks(N), kThreads, 0, st>>>(N, x, d, y); }
}

void launch_unscale(const Col &c, const double *xs, double *delta, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_unscale<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, xs, delta); }
}

void launch_check(const Col &c, Ctl *ctl, const Policy &pol, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_check<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, ctl, pol); }
}

void launch_decide(const Col &c, Ctl *ctl, const Policy &pol, cudaStream_t st)
{
    (void)c;
    count_launches(1); k_decide<<<1, 1, 0, st>>>(ctl, pol);
}

void launch_apply(const Col &c, Ctl *ctl, cudaStream_t st)
{
    if (((long long)c.L * c.S) > 0) { count_launches(1); k_apply<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, ctl); }
}

void launch_diag(const Col &c, const Ctl *ctl, double *diag, cudaStream_t st)
{
    count_launches(1);
    k_diag<<<nblocks((long long)c.L * c.S), kThreads, 0, st>>>(c, ctl, diag);
}

void launch_reuse_scales(long long N, const double *rowd, const double *s, const double *s64, double *pin, double *pout,
                         const Ctl *ctl, cudaStream_t st)
{
    count_launches(1);
    k_reuse_scales<<<nblocks(N), kThreads, 0, st>>>(N, rowd, s, s64, pin, pout, ctl);
}

void launch_after_refactor(long long N, const double *s, double *s64, Ctl *ctl, cudaStream_t st)
{
    count_launches(1);
    k_after_refactor<<<nblocks(N), kThreads, 0, st>>>(N, s, s64, ctl);
}

void launch_route(Ctl *ctl, cudaStream_t st)
{
    count_launches(1);
    k_route<<<1, 1, 0, st>>>(ctl);
}

void launch_begin(Ctl *ctl, cudaStream_t st)
{
    count_launches(1);
    k_begin<<<1, 1, 0, st>>>(ctl);
}

}  // namespace xk
