/*
 * Plain FP64 CPU oracle of the implicit photochemical-kinetics step
 * (Ghosh et al., XODIAC; Sec. 2.1 continuity and transport, Sec. 2.3 rate
 * coefficients, Sec. 2.5 boundaries, Appendix A thermochemistry).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  Straight loops in
 * the order the paper states the method, no blocking, no fusion.
 *
 * Readings where the paper is silent or garbled (each one also in the design
 * notes):
 *  - Eulerian backward-Euler discretisation of Eq. 1 with the flux of Eq. 2 in
 *    conservative form on a hydrostatic grid; interface values are arithmetic
 *    means (the "k +- 1/2" convention stated with Eq. 3); the eddy term is
 *    written in mixing-ratio form, which is what the n_gas ratios of Eq. 3 are.
 *  - molecular diffusion D_y = b_y T^0.75 / n_gas (binary-mixture form; the
 *    coefficients are inputs).
 *  - K_c from the Gibbs energy of reaction in concentration units:
 *    ln K_c = -sum nu G/RT + dnu ln(p0 / (k_B T)), p0 = 1 bar (Sec. 2.3.4).
 *  - three-body fall-off: Lindemann (Sec. 2.3.2) times the Troe broadening
 *    factor when a Troe set is given; [M] = n_gas.
 *  - photolysis: the direct beam, optical depth (absorption plus Rayleigh
 *    scattering) to the layer midpoint, plus optionally the diffuse field of a
 *    layer-by-layer two-stream photon budget (ora_two_stream); rates lagged
 *    (evaluated at the start of a step, not differentiated); photolysis is
 *    irreversible.
 *  - zero-flux top and bottom boundaries (Sec. 2.5).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_KB 1.380649e-16        /* erg / K */
#define ORA_AMU 1.66053906660e-24  /* g */
#define ORA_P0 1.0e6               /* 1 bar in dyn / cm^2 */
/* FP64 iterative-refinement sweeps of the step's linear solve: the step is the
 * solution of (I/dt - J) delta = F, and block Thomas without pivoting across
 * layers leaves a componentwise backward error up to ~1e-8 on the largest
 * columns; each sweep (FP64 residual, correction with the stored factors)
 * brings it back to a few ulp. */
#define ORA_REFINE_SWEEPS 4

/* ------------------------------------------------------------------ grid */

void ora_grid(const ora_problem *p, double *ngas, double *z, double *dz, double *dzi)
{
    int L = p->L;
    for (int k = 0; k < L; ++k)
        ngas[k] = p->P_bar[k] * 1.0e6 / (ORA_KB * p->T[k]);
    /* hydrostatic balance: dz = H ln(P_k / P_{k+1}), H = k_B T / (mbar g) at the interface */
    z[0] = 0.0;
    for (int k = 0; k + 1 < L; ++k) {
        double Th = 0.5 * (p->T[k] + p->T[k + 1]);
        double H = ORA_KB * Th / (p->mbar * ORA_AMU * p->g);
        z[k + 1] = z[k] + H * log(p->P_bar[k] / p->P_bar[k + 1]);
    }
    for (int k = 0; k + 1 < L; ++k)
        dzi[k] = z[k + 1] - z[k];
    if (L == 1) {
        dz[0] = 1.0;
        return;
    }
    dz[0] = z[1] - z[0];
    dz[L - 1] = z[L - 1] - z[L - 2];
    for (int k = 1; k + 1 < L; ++k)
        dz[k] = 0.5 * (z[k + 1] - z[k - 1]);
}

/* ------------------------------------------------------------ thermo */

static const double *nasa_set(const double *nasa15, double T)
{
    /* low set below T_mid, high set at and above it */
    return (T < nasa15[0]) ? nasa15 + 1 : nasa15 + 8;
}

double ora_gibbs_rt(const double *nasa15, double T)
{
    const double *a = nasa_set(nasa15, T);
    return a[0] * (1.0 - log(T)) - a[1] * T / 2.0 - a[2] * T * T / 6.0
         - a[3] * T * T * T / 12.0 - a[4] * T * T * T * T / 20.0 + a[5] / T - a[6];
}

double ora_cp_r(const double *nasa15, double T)
{
    const double *a = nasa_set(nasa15, T);
    return a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
}

static double ln_kc(const ora_problem *p, int r, double T, const double *grt)
{
    double dG = 0.0;
    int dnu = 0;
    for (int s = 0; s < 3; ++s) {
        int i = p->reac[3 * r + s];
        if (i >= 0) { dG -= grt[i]; dnu -= 1; }
        int j = p->prod[3 * r + s];
        if (j >= 0) { dG += grt[j]; dnu += 1; }
    }
    return -dG + dnu * log(ORA_P0 / (ORA_KB * T));
}

void ora_thermo(const ora_problem *p, double *grt, double *lnkc)
{
    for (int k = 0; k < p->L; ++k) {
        double T = p->T[k];
        for (int y = 0; y < p->S; ++y)
            grt[(size_t)k * p->S + y] = ora_gibbs_rt(p->nasa + 15 * y, T);
        for (int r = 0; r < p->R; ++r)
            lnkc[(size_t)k * p->R + r] = (p->rtype[r] == 2) ? 0.0
                                       : ln_kc(p, r, T, grt + (size_t)k * p->S);
    }
}

/* -------------------------------------------------------------- rates */

static double arrhenius(double alpha, double beta, double gamma, double T, int form)
{
    double Tb = (form == 0) ? T / 300.0 : T;
    return alpha * pow(Tb, beta) * exp(-gamma / T);
}

static double troe_factor(const double *tr, double T, double Pr)
{
    if (tr[0] == 0.0 || Pr <= 0.0)
        return 1.0;
    double Fc = (1.0 - tr[0]) * exp(-T / tr[1]) + tr[0] * exp(-T / tr[2]);
    if (tr[3] != 0.0)
        Fc += exp(-tr[3] / T);
    double lFc = log10(Fc);
    double c = -0.4 - 0.67 * lFc;
    double N = 0.75 - 1.27 * lFc;
    double x = log10(Pr) + c;
    double q = x / (N - 0.14 * x);
    return pow(10.0, lFc / (1.0 + q * q));
}

void ora_rate_coefficients(const ora_problem *p, double *kf, double *kr)
{
    int L = p->L, R = p->R, S = p->S;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    double *grt = malloc(sizeof(double) * S);
    for (int k = 0; k < L; ++k) {
        double T = p->T[k];
        for (int y = 0; y < S; ++y)
            grt[y] = ora_gibbs_rt(p->nasa + 15 * y, T);
        for (int r = 0; r < R; ++r) {
            const double *a = p->arr + 9 * r;
            double f = 0.0, b = 0.0;
            if (p->rtype[r] == 0) {
                f = arrhenius(a[0], a[1], a[2], T, p->form[r]);
            } else if (p->rtype[r] == 1) {
                double k0 = arrhenius(a[3], a[4], a[5], T, p->form[r]);
                double ki = arrhenius(a[6], a[7], a[8], T, p->form[r]);
                double M = ngas[k];
                double Pr = k0 * M / ki;
                f = k0 * M / (1.0 + k0 * M / ki) * troe_factor(p->troe + 4 * r, T, Pr);
            }
            if (p->rtype[r] != 2)
                b = f / exp(ln_kc(p, r, T, grt));
            kf[(size_t)k * R + r] = f;
            kr[(size_t)k * R + r] = b;
        }
    }
    free(grt);
    free(ngas);
}

/*
 * Sec. 2.3.3 diffuse field, where the paper gives J_diff = (J_up + J_down) / 2 but not how the two
 * fluxes are found.  Reading: a two-stream photon budget layer by layer.  The beam loses
 * mu F0 (e^{-tau_top/mu} - e^{-tau_bot/mu}) photons per unit horizontal area in layer k; the
 * scattered fraction omega_k = dtau_s / (dtau_a + dtau_s) of them is shared equally between the
 * two hemispheres (isotropic, as Rayleigh scattering is in the mean).  A diffuse flux crossing the
 * layer goes through with probability t = exp(-dtau / mubar), mubar = 1/2 (the hemispheric mean
 * path 2 dtau); otherwise it interacts, and is scattered (half back, half on) with probability
 * omega or absorbed.  So layer k reflects r = (1 - t) omega / 2 and transmits T = t + (1 - t) omega / 2
 * of each diffuse flux.  The lower boundary reflects the fraction `albedo` of what reaches it
 * (diffuse and beam); nothing diffuse enters at the top.  Unknowns: U_i, D_i at the L + 1
 * interfaces (D_L = 0), solved as one banded system
 *     D_k     - T_k D_{k+1} - r_k U_k = P_k / 2,
 *     U_{k+1} - T_k U_k - r_k D_{k+1} = P_k / 2,
 *     U_0     - albedo D_0            = albedo B_bottom,
 * by Gaussian elimination without pivoting (each row is diagonally dominant: T + r <= 1).
 */
int ora_two_stream(int L, const double *dtau_a, const double *dtau_s, double F0, double mu, double albedo,
                   double *U, double *D, double *Jdiff)
{
    /* unknowns v[2i] = U_i (i = 0..L), v[2i+1] = D_i (i = 0..L-1); band a[row][col - row + 2] */
    int n = 2 * L + 1;
    double *a = calloc((size_t)n * 5, sizeof(double)), *rhs = calloc((size_t)n, sizeof(double));
    double *r = malloc(sizeof(double) * L * 3), *T = r + L, *P = T + L;
    if (!a || !rhs || !r) { free(a); free(rhs); free(r); return -1; }
    double tau_top = 0.0;
    for (int k = L - 1; k >= 0; --k) {
        double dt = dtau_a[k] + dtau_s[k];
        double om = dt > 0.0 ? dtau_s[k] / dt : 0.0;
        double t = exp(-dt / 0.5);
        r[k] = (1.0 - t) * om / 2.0;
        T[k] = t + (1.0 - t) * om / 2.0;
        P[k] = om * mu * F0 * (exp(-tau_top / mu) - exp(-(tau_top + dt) / mu));
        tau_top += dt;
    }
    double Bbot = mu * F0 * exp(-tau_top / mu);
#define BAND(i, j) a[(size_t)(i) * 5 + (j) - (i) + 2]
    /* bottom boundary, row 0 (U_0) */
    BAND(0, 0) = 1.0;
    BAND(0, 1) = -albedo;
    rhs[0] = albedo * Bbot;
    for (int k = 0; k < L; ++k) {
        int rd = 2 * k + 1, ru = 2 * k + 2;            /* rows of D_k and U_{k+1} */
        BAND(rd, rd) = 1.0;
        if (k + 1 < L) BAND(rd, 2 * k + 3) = -T[k];   /* D_{k+1} */
        BAND(rd, 2 * k) = -r[k];                       /* U_k */
        rhs[rd] = P[k] / 2.0;
        BAND(ru, ru) = 1.0;
        BAND(ru, 2 * k) = -T[k];                       /* U_k */
        if (k + 1 < L) BAND(ru, 2 * k + 3) = -r[k];   /* D_{k+1} */
        rhs[ru] = P[k] / 2.0;
    }
    /* elimination below the diagonal (lower bandwidth 2, upper bandwidth 2, no fill outside) */
    int rc = 0;
    for (int c = 0; c < n; ++c) {
        double piv = BAND(c, c);
        if (piv == 0.0) { rc = -1; break; }
        for (int i = c + 1; i <= c + 2 && i < n; ++i) {
            double l = BAND(i, c) / piv;
            if (l == 0.0) continue;
            for (int j = c; j <= c + 2 && j < n; ++j)
                BAND(i, j) -= l * BAND(c, j);
            rhs[i] -= l * rhs[c];
        }
    }
    if (rc == 0)
        for (int i = n - 1; i >= 0; --i) {
            double s = rhs[i];
            for (int j = i + 1; j <= i + 2 && j < n; ++j)
                s -= BAND(i, j) * rhs[j];
            rhs[i] = s / BAND(i, i);
        }
#undef BAND
    if (rc == 0) {
        for (int i = 0; i <= L; ++i) {
            U[i] = rhs[2 * i];
            D[i] = i < L ? rhs[2 * i + 1] : 0.0;
        }
        for (int k = 0; k < L; ++k) {
            double up = 0.5 * (U[k] + U[k + 1]), dn = 0.5 * (D[k] + D[k + 1]);
            Jdiff[k] = 0.5 * (up + dn);
        }
    }
    free(a);
    free(rhs);
    free(r);
    return rc;
}

void ora_photolysis(const ora_problem *p, const double *n, double *kph)
{
    int L = p->L, S = p->S, W = p->W, R = p->R, Rph = p->Rph;
    if (Rph == 0)
        return;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    double *alpha = malloc(sizeof(double) * L * 2), *alpha_s = alpha + L;
    double *J = malloc(sizeof(double) * L * W);
    double *ta = malloc(sizeof(double) * (L * 3 + 2 * (L + 1))), *ts = ta + L, *Jd = ts + L;
    double *U = Jd + L, *D = U + L + 1;
    for (int w = 0; w < W; ++w) {
        /* absorption and Rayleigh-scattering coefficients per layer: sum_i sigma_i n_i */
        for (int k = 0; k < L; ++k) {
            double s = 0.0, sc = 0.0;
            for (int i = 0; i < S; ++i) {
                s += p->sigma_abs[(size_t)i * W + w] * n[(size_t)k * S + i];
                if (p->sigma_s) sc += p->sigma_s[(size_t)i * W + w] * n[(size_t)k * S + i];
            }
            alpha[k] = s;
            alpha_s[k] = sc;
        }
        /* total optical depth (absorption plus scattering) from the top down to the layer midpoint */
        double above = 0.0;
        for (int k = L - 1; k >= 0; --k) {
            double ext = alpha[k] + alpha_s[k];
            double tau = above + 0.5 * ext * dz[k];
            J[(size_t)k * W + w] = p->J0[w] * exp(-tau / p->mu);
            above += ext * dz[k];
        }
        if (p->diffuse) {
            for (int k = 0; k < L; ++k) {
                ta[k] = alpha[k] * dz[k];
                ts[k] = alpha_s[k] * dz[k];
            }
            if (ora_two_stream(L, ta, ts, p->J0[w], p->mu, p->albedo, U, D, Jd) == 0)
                for (int k = 0; k < L; ++k)
                    J[(size_t)k * W + w] += Jd[k];
        }
    }
    for (int k = 0; k < L; ++k)
        for (int q = 0; q < Rph; ++q) {
            double s = 0.0;
            for (int w = 0; w < W; ++w)
                s += J[(size_t)k * W + w] * p->sigma[(size_t)q * W + w] * p->dlam[w];
            kph[(size_t)k * Rph + q] = p->tf * s;
        }
    (void)R;
    free(ta);
    free(J);
    free(alpha);
    free(ngas);
}

/* ---------------------------------------------------------- transport */

void ora_transport(const ora_problem *p, double *u, double *v)
{
    int L = p->L, S = p->S;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    for (int k = 0; k + 1 < L; ++k) {
        double Th = 0.5 * (p->T[k] + p->T[k + 1]);
        double nh = 0.5 * (ngas[k] + ngas[k + 1]);
        double Kh = 0.5 * (p->Kzz[k] + p->Kzz[k + 1]);
        double h = dzi[k];
        double dTdz = (p->T[k + 1] - p->T[k]) / h;
        for (int y = 0; y < S; ++y) {
            double D = p->dcoef[y] * pow(Th, 0.75) / nh;
            double Hy = ORA_KB * Th / (p->mass[y] * ORA_AMU * p->g);
            double a = 1.0 / Hy + (1.0 + p->alpha_T) * dTdz / Th;
            /* eddy: -K n_gas d(n/n_gas)/dz; molecular: -D (dn/dz + n a) */
            u[(size_t)k * S + y] = Kh * nh / (h * ngas[k]) + D * (1.0 / h - 0.5 * a);
            v[(size_t)k * S + y] = Kh * nh / (h * ngas[k + 1]) + D * (1.0 / h + 0.5 * a);
        }
    }
    free(ngas);
}

/* ----------------------------------------------------------- residual */

static void layer_rates(const ora_problem *p, int k, const double *kf, const double *kr,
                        const double *kph, double *kf_k, double *kr_k)
{
    for (int r = 0; r < p->R; ++r) {
        if (p->rtype[r] == 2) {
            kf_k[r] = kph[(size_t)k * p->Rph + p->prow[r]];
            kr_k[r] = 0.0;
        } else {
            kf_k[r] = kf[(size_t)k * p->R + r];
            kr_k[r] = kr[(size_t)k * p->R + r];
        }
    }
}

void ora_residual(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                  const double *n, double *F)
{
    int L = p->L, S = p->S, R = p->R;
    double *kf_k = malloc(sizeof(double) * R * 2), *kr_k = kf_k + R;
    double *u = malloc(sizeof(double) * (L > 1 ? (L - 1) : 1) * S * 2);
    double *v = u + (size_t)(L > 1 ? (L - 1) : 1) * S;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    ora_transport(p, u, v);
    for (int k = 0; k < L; ++k) {
        const double *nk = n + (size_t)k * S;
        double *Fk = F + (size_t)k * S;
        for (int y = 0; y < S; ++y)
            Fk[y] = 0.0;
        layer_rates(p, k, kf, kr, kph, kf_k, kr_k);
        /* chemistry: production minus loss, mass action */
        for (int r = 0; r < R; ++r) {
            double wf = kf_k[r], wb = kr_k[r];
            for (int s = 0; s < 3; ++s) {
                if (p->reac[3 * r + s] >= 0) wf *= nk[p->reac[3 * r + s]];
                if (p->prod[3 * r + s] >= 0) wb *= nk[p->prod[3 * r + s]];
            }
            double w = wf - wb;
            for (int s = 0; s < 3; ++s) {
                if (p->reac[3 * r + s] >= 0) Fk[p->reac[3 * r + s]] -= w;
                if (p->prod[3 * r + s] >= 0) Fk[p->prod[3 * r + s]] += w;
            }
        }
        /* transport: -(phi_{k+1/2} - phi_{k-1/2}) / dz_k, zero flux at both ends */
        for (int y = 0; y < S; ++y) {
            double up = 0.0, dn = 0.0;
            if (k + 1 < L)
                up = u[(size_t)k * S + y] * nk[y] - v[(size_t)k * S + y] * n[(size_t)(k + 1) * S + y];
            if (k > 0)
                dn = u[(size_t)(k - 1) * S + y] * n[(size_t)(k - 1) * S + y] - v[(size_t)(k - 1) * S + y] * nk[y];
            Fk[y] += -(up - dn) / dz[k];
        }
    }
    free(ngas);
    free(u);
    free(kf_k);
}

/* ----------------------------------------------------------- jacobian */

void ora_jacobian(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                  const double *n, double dt, double *A, double *lo, double *up)
{
    int L = p->L, S = p->S, R = p->R;
    double *kf_k = malloc(sizeof(double) * R * 2), *kr_k = kf_k + R;
    double *u = malloc(sizeof(double) * (L > 1 ? (L - 1) : 1) * S * 2);
    double *v = u + (size_t)(L > 1 ? (L - 1) : 1) * S;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    ora_transport(p, u, v);
    for (int k = 0; k < L; ++k) {
        const double *nk = n + (size_t)k * S;
        double *Ak = A + (size_t)k * S * S;
        memset(Ak, 0, sizeof(double) * S * S);
        layer_rates(p, k, kf, kr, kph, kf_k, kr_k);
        /* dF_i/dn_j = sum_r nu_ir dw_r/dn_j; A = I/dt - dF/dn */
        for (int r = 0; r < R; ++r) {
            for (int side = 0; side < 2; ++side) {
                const int *sp = (side == 0) ? p->reac + 3 * r : p->prod + 3 * r;
                double kk = (side == 0) ? kf_k[r] : -kr_k[r];
                for (int s = 0; s < 3; ++s) {
                    int j = sp[s];
                    if (j < 0)
                        continue;
                    double d = kk;                  /* derivative of k prod n w.r.t. the s-th factor */
                    for (int t = 0; t < 3; ++t)
                        if (t != s && sp[t] >= 0)
                            d *= nk[sp[t]];
                    for (int q = 0; q < 3; ++q) {
                        if (p->reac[3 * r + q] >= 0) Ak[(size_t)p->reac[3 * r + q] * S + j] += d;  /* -(-d) */
                        if (p->prod[3 * r + q] >= 0) Ak[(size_t)p->prod[3 * r + q] * S + j] -= d;  /* -(+d) */
                    }
                }
            }
        }
        for (int y = 0; y < S; ++y) {
            double diag = 1.0 / dt;
            if (k + 1 < L) diag += u[(size_t)k * S + y] / dz[k];
            if (k > 0) diag += v[(size_t)(k - 1) * S + y] / dz[k];
            Ak[(size_t)y * S + y] += diag;
            lo[(size_t)k * S + y] = (k > 0) ? -u[(size_t)(k - 1) * S + y] / dz[k] : 0.0;
            up[(size_t)k * S + y] = (k + 1 < L) ? -v[(size_t)k * S + y] / dz[k] : 0.0;
        }
    }
    free(ngas);
    free(u);
    free(kf_k);
}

/* ------------------------------------------------------ block solve */

/* Gaussian elimination with partial pivoting: a (S x S) becomes L\U, piv the row order. */
static int lu_factor(int S, double *a, int *piv)
{
    for (int i = 0; i < S; ++i)
        piv[i] = i;
    for (int c = 0; c < S; ++c) {
        int best = c;
        double bv = fabs(a[(size_t)c * S + c]);
        for (int i = c + 1; i < S; ++i) {
            double v = fabs(a[(size_t)i * S + c]);
            if (v > bv) { bv = v; best = i; }
        }
        if (bv == 0.0)
            return -1;
        if (best != c) {
            for (int j = 0; j < S; ++j) {
                double t = a[(size_t)c * S + j];
                a[(size_t)c * S + j] = a[(size_t)best * S + j];
                a[(size_t)best * S + j] = t;
            }
            int t = piv[c]; piv[c] = piv[best]; piv[best] = t;
        }
        double inv = 1.0 / a[(size_t)c * S + c];
        for (int i = c + 1; i < S; ++i) {
            double l = a[(size_t)i * S + c] * inv;
            a[(size_t)i * S + c] = l;
            for (int j = c + 1; j < S; ++j)
                a[(size_t)i * S + j] -= l * a[(size_t)c * S + j];
        }
    }
    return 0;
}

/* Solve (L U) X = P B for m right-hand-side columns stored row-major in B (S x m). */
static void lu_solve(int S, const double *a, const int *piv, const double *B, double *X, int m)
{
    for (int i = 0; i < S; ++i)
        memcpy(X + (size_t)i * m, B + (size_t)piv[i] * m, sizeof(double) * m);
    for (int i = 0; i < S; ++i)
        for (int c = 0; c < i; ++c) {
            double l = a[(size_t)i * S + c];
            for (int j = 0; j < m; ++j)
                X[(size_t)i * m + j] -= l * X[(size_t)c * m + j];
        }
    for (int i = S - 1; i >= 0; --i) {
        for (int c = i + 1; c < S; ++c) {
            double uu = a[(size_t)i * S + c];
            for (int j = 0; j < m; ++j)
                X[(size_t)i * m + j] -= uu * X[(size_t)c * m + j];
        }
        double inv = 1.0 / a[(size_t)i * S + i];
        for (int j = 0; j < m; ++j)
            X[(size_t)i * m + j] *= inv;
    }
}

/* Block Thomas, elimination: D'_k = A_k - diag(lo_k) D'^-1_{k-1} diag(up_{k-1}), each D'_k
 * overwritten by its LU factors (row order in piv). */
static int block_factor(int L, int S, double *A, const double *lo, const double *up, int *piv)
{
    double *B = malloc(sizeof(double) * (size_t)S * S);
    double *X = malloc(sizeof(double) * (size_t)S * S);
    int rc = 0;
    for (int k = 0; k < L && rc == 0; ++k) {
        double *Ak = A + (size_t)k * S * S;
        if (k > 0) {
            double *Ap = A + (size_t)(k - 1) * S * S;
            memset(B, 0, sizeof(double) * S * S);
            for (int y = 0; y < S; ++y)
                B[(size_t)y * S + y] = up[(size_t)(k - 1) * S + y];
            lu_solve(S, Ap, piv + (size_t)(k - 1) * S, B, X, S);
            for (int i = 0; i < S; ++i)
                for (int j = 0; j < S; ++j)
                    Ak[(size_t)i * S + j] -= lo[(size_t)k * S + i] * X[(size_t)i * S + j];
        }
        if (lu_factor(S, Ak, piv + (size_t)k * S) != 0)
            rc = -1;
    }
    free(X); free(B);
    return rc;
}

/* Block Thomas, substitution with the factors of block_factor: g_k = f_k - diag(lo_k) D'^-1_{k-1} g_{k-1},
 * then x_k = D'^-1_k (g_k - diag(up_k) x_{k+1}). */
static void block_apply(int L, int S, const double *LU, const int *piv, const double *lo, const double *up,
                        const double *f, double *x)
{
    double *g = malloc(sizeof(double) * (size_t)L * S);
    double *t = malloc(sizeof(double) * S);
    memcpy(g, f, sizeof(double) * (size_t)L * S);
    for (int k = 1; k < L; ++k) {
        lu_solve(S, LU + (size_t)(k - 1) * S * S, piv + (size_t)(k - 1) * S, g + (size_t)(k - 1) * S, t, 1);
        for (int i = 0; i < S; ++i)
            g[(size_t)k * S + i] -= lo[(size_t)k * S + i] * t[i];
    }
    for (int k = L - 1; k >= 0; --k) {
        for (int i = 0; i < S; ++i)
            t[i] = g[(size_t)k * S + i] - ((k + 1 < L) ? up[(size_t)k * S + i] * x[(size_t)(k + 1) * S + i] : 0.0);
        lu_solve(S, LU + (size_t)k * S * S, piv + (size_t)k * S, t, x + (size_t)k * S, 1);
    }
    free(t); free(g);
}

int ora_block_solve(int L, int S, double *A, const double *lo, const double *up,
                    const double *f, double *x)
{
    int *piv = malloc(sizeof(int) * (size_t)L * S);
    int rc = block_factor(L, S, A, lo, up, piv);
    if (rc == 0)
        block_apply(L, S, A, piv, lo, up, f, x);
    free(piv);
    return rc;
}

/* r = f - M x for the block-tridiagonal M = (A, lo, up), in FP64. */
static void block_residual(int L, int S, const double *A, const double *lo, const double *up,
                           const double *f, const double *x, double *r)
{
    for (int k = 0; k < L; ++k)
        for (int i = 0; i < S; ++i) {
            const double *Ar = A + ((size_t)k * S + i) * S;
            double acc = f[(size_t)k * S + i];
            for (int j = 0; j < S; ++j)
                acc -= Ar[j] * x[(size_t)k * S + j];
            if (k > 0) acc -= lo[(size_t)k * S + i] * x[(size_t)(k - 1) * S + i];
            if (k + 1 < L) acc -= up[(size_t)k * S + i] * x[(size_t)(k + 1) * S + i];
            r[(size_t)k * S + i] = acc;
        }
}

int ora_block_solve_refined(int L, int S, const double *A, const double *lo, const double *up,
                            const double *f, double *x, int sweeps)
{
    size_t LS = (size_t)L * S;
    double *W = malloc(sizeof(double) * LS * S);
    int *piv = malloc(sizeof(int) * LS);
    double *r = malloc(sizeof(double) * LS * 2), *d = r + LS;
    memcpy(W, A, sizeof(double) * LS * S);
    int rc = block_factor(L, S, W, lo, up, piv);
    if (rc == 0) {
        block_apply(L, S, W, piv, lo, up, f, x);
        for (int it = 0; it < sweeps; ++it) {
            block_residual(L, S, A, lo, up, f, x, r);
            block_apply(L, S, W, piv, lo, up, r, d);
            for (size_t i = 0; i < LS; ++i)
                x[i] += d[i];
        }
    }
    free(r); free(piv); free(W);
    return rc;
}

/* ---------------------------------------------------------- stepping */

int ora_step_delta(const ora_problem *p, const double *n, double dt, double *delta)
{
    int L = p->L, S = p->S, R = p->R;
    size_t LS = (size_t)L * S;
    double *kf = malloc(sizeof(double) * (size_t)L * R * 2), *kr = kf + (size_t)L * R;
    double *kph = malloc(sizeof(double) * (size_t)L * (p->Rph > 0 ? p->Rph : 1));
    double *F = malloc(sizeof(double) * LS * 3), *lo = F + LS, *up = lo + LS;
    double *A = malloc(sizeof(double) * LS * S);
    ora_rate_coefficients(p, kf, kr);
    ora_photolysis(p, n, kph);
    ora_residual(p, kf, kr, kph, n, F);
    ora_jacobian(p, kf, kr, kph, n, dt, A, lo, up);
    int rc = ora_block_solve_refined(L, S, A, lo, up, F, delta, ORA_REFINE_SWEEPS);
    free(A); free(F); free(kph); free(kf);
    return rc;
}

int ora_step(const ora_problem *p, const ora_policy *pol, double *n, double dt, ora_step_info *info)
{
    int L = p->L, S = p->S;
    size_t LS = (size_t)L * S;
    double *delta = malloc(sizeof(double) * LS);
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    int rc = ora_step_delta(p, n, dt, delta);
    int ok = (rc == 0);
    double maxrel = 0.0;
    int nneg = 0;
    for (int k = 0; k < L && ok; ++k)
        for (int y = 0; y < S; ++y) {
            double d = delta[(size_t)k * S + y], nv = n[(size_t)k * S + y];
            double nn = nv + d;
            if (!isfinite(nn)) { ok = 0; break; }
            if (nn < -pol->neg_tol * ngas[k]) ok = 0;
            if (nv > pol->f_floor * ngas[k]) {
                double rel = fabs(d) / nv;
                if (rel > maxrel) maxrel = rel;
            }
        }
    if (ok && maxrel > pol->rel_reject)
        ok = 0;
    info->dt_used = dt;
    info->max_rel = maxrel;
    info->n_neg = 0;
    if (ok) {
        for (size_t i = 0; i < LS; ++i) {
            double nn = n[i] + delta[i];
            if (nn < 0.0) { nn = 0.0; ++nneg; }
            n[i] = nn;
        }
        double fac = (maxrel > 0.0) ? pol->rel_target / maxrel : pol->grow_max;
        if (fac > pol->grow_max) fac = pol->grow_max;
        if (fac < pol->shrink_min) fac = pol->shrink_min;
        double dn = dt * fac;
        info->dt_next = (dn > pol->dt_max) ? pol->dt_max : dn;
        info->accepted = 1;
        info->n_neg = nneg;
    } else {
        info->dt_next = 0.5 * dt;
        info->accepted = 0;
    }
    free(ngas);
    free(delta);
    return 0;
}

int ora_run_to_steady(const ora_problem *p, const ora_policy *pol, double *n, double dt0,
                      int max_steps, ora_run_info *info)
{
    double dt = dt0, t = 0.0;
    int steps = 0, acc = 0, rej = 0, conv = 0;
    ora_step_info si;
    si.max_rel = 0.0;
    while (steps < max_steps) {
        ora_step(p, pol, n, dt, &si);
        ++steps;
        if (si.accepted) {
            ++acc;
            t += dt;
            if (dt >= pol->ss_dt && si.max_rel < pol->ss_tol) { conv = 1; dt = si.dt_next; break; }
        } else {
            ++rej;
        }
        dt = si.dt_next;
        if (dt < pol->dt_min)
            break;
    }
    info->converged = conv;
    info->steps = steps;
    info->accepted = acc;
    info->rejected = rej;
    info->t = t;
    info->dt = dt;
    info->max_rel = si.max_rel;
    return conv ? 0 : -1;
}

/* ------------------------------------------------ Lagrangian parcel */

/* The paper's own driver (Sec. 2, Fig. 1 and Fig. 2): an air parcel is carried
 * from the bottom of the atmosphere to the top and back; in each layer it evolves
 * under that layer's chemistry, and molecular diffusion acts on it as a pair of
 * pseudo-reactions (Sec. 2.1, after Eq. 4): the parcel loses a species to the
 * neighbouring layers and gains it back from their stored densities.  Eddy
 * diffusion has no term of its own: it is the parcel's motion.  A global
 * iteration is one such round trip; the run has converged when two successive
 * iterations change no mixing ratio by 0.1 % or more (Sec. 2).
 *
 * Readings where the paper is silent:
 *  - visits: layers 0, 1, ..., L-1, then L-2, ..., 0 (2L - 1 visits; the top
 *    layer once); each visit stores the parcel's densities as that layer's;
 *  - the parcel keeps its mixing ratios as it moves: entering layer k its
 *    densities are f * n_gas,k;
 *  - residence time in layer k: the eddy mixing time tau_k = dz_k^2 / K_zz,k;
 *  - time integration within a visit, in place of the paper's DLSODES:
 *    linearly implicit Euler steps over [0, tau_k] under the step controller
 *    of the Eulerian path (ora_step): a step is rejected and halved when a
 *    density would fall below -neg_tol n_gas or change by more than rel_reject
 *    (relative, over species above f_floor); an accepted step clips negatives
 *    to 0 and scales the next one by rel_target / max change, within
 *    [shrink_min, grow_max]; a step never crosses the end of the visit, and
 *    the trial step is carried from visit to visit (a step cut short by the
 *    end of a visit does not shrink it);
 *  - molecular diffusion: the molecular part of Eq. 2's flux (eddy K = 0)
 *    between the parcel and the stored densities of layers k - 1 and k + 1
 *    as they stand at the visit (zero flux at both ends);
 *  - photolysis rates from the stored profile at the start of the iteration;
 *  - the convergence measure: the largest |N_new - N_old| / N_new over
 *    entries above f_floor mixing ratio (same layer, so mixing ratios and
 *    densities give the same ratio). */

#define ORA_PARCEL_REFINE 2

/* Chemistry of one layer at composition nk: Fk = sum_r nu_r w_r and the dense Jacobian
 * Jk = dFk/dnk (S x S, row-major), mass action as in ora_residual / ora_jacobian. */
static void layer_chemistry(const ora_problem *p, const double *kf_k, const double *kr_k, const double *nk,
                            double *Fk, double *Jk)
{
    int S = p->S, R = p->R;
    memset(Fk, 0, sizeof(double) * S);
    memset(Jk, 0, sizeof(double) * S * S);
    for (int r = 0; r < R; ++r) {
        const int *ra = p->reac + 3 * r, *pa = p->prod + 3 * r;
        double wf = kf_k[r], wb = kr_k[r];
        for (int s = 0; s < 3; ++s) {
            if (ra[s] >= 0) wf *= nk[ra[s]];
            if (pa[s] >= 0) wb *= nk[pa[s]];
        }
        double w = wf - wb;
        for (int s = 0; s < 3; ++s) {
            if (ra[s] >= 0) Fk[ra[s]] -= w;
            if (pa[s] >= 0) Fk[pa[s]] += w;
        }
        /* dw/dn_j, then dF_i/dn_j = nu_i dw/dn_j */
        for (int side = 0; side < 2; ++side) {
            const int *sp = side == 0 ? ra : pa;
            double kk = side == 0 ? kf_k[r] : -kr_k[r];
            for (int s = 0; s < 3; ++s) {
                int j = sp[s];
                if (j < 0)
                    continue;
                double d = kk;
                for (int t = 0; t < 3; ++t)
                    if (t != s && sp[t] >= 0)
                        d *= nk[sp[t]];
                for (int q = 0; q < 3; ++q) {
                    if (ra[q] >= 0) Jk[(size_t)ra[q] * S + j] -= d;
                    if (pa[q] >= 0) Jk[(size_t)pa[q] * S + j] += d;
                }
            }
        }
    }
}

/* Everything a visit needs that does not change within an iteration. */
typedef struct {
    double *ngas, *z, *dz, *dzi;
    double *kf, *kr, *kph;
    double *um, *vm;          /* molecular part of Eq. 2's u, v per interface */
} parcel_fields;

static void parcel_fields_make(const ora_problem *p, const double *N, parcel_fields *f)
{
    int L = p->L, S = p->S, R = p->R;
    size_t m = (size_t)(L > 1 ? L - 1 : 1) * S;
    f->ngas = malloc(sizeof(double) * L * 4);
    f->z = f->ngas + L; f->dz = f->z + L; f->dzi = f->dz + L;
    ora_grid(p, f->ngas, f->z, f->dz, f->dzi);
    f->kf = malloc(sizeof(double) * (size_t)L * R * 2);
    f->kr = f->kf + (size_t)L * R;
    ora_rate_coefficients(p, f->kf, f->kr);
    f->kph = malloc(sizeof(double) * (size_t)L * (p->Rph > 0 ? p->Rph : 1));
    ora_photolysis(p, N, f->kph);
    f->um = malloc(sizeof(double) * m * 2);
    f->vm = f->um + m;
    double *zero = calloc((size_t)L, sizeof(double));
    ora_problem q = *p;
    q.Kzz = zero;
    ora_transport(&q, f->um, f->vm);
    free(zero);
}

static void parcel_fields_free(parcel_fields *f)
{
    free(f->ngas); free(f->kf); free(f->kph); free(f->um);
}

/* F and A = I/h - dF/dpk of the parcel with densities pk in layer k. */
static void parcel_system(const ora_problem *p, const parcel_fields *f, const double *N, int k,
                          const double *pk, double h, double *F, double *A)
{
    int L = p->L, S = p->S, R = p->R;
    double *kf_k = malloc(sizeof(double) * R * 2 + sizeof(double)), *kr_k = kf_k + R;
    layer_rates(p, k, f->kf, f->kr, f->kph, kf_k, kr_k);
    layer_chemistry(p, kf_k, kr_k, pk, F, A);
    /* A = -J so far: negate, then add I/h */
    for (size_t i = 0; i < (size_t)S * S; ++i)
        A[i] = -A[i];
    for (int y = 0; y < S; ++y) {
        /* molecular diffusion: loss of the parcel's own density, gain from the neighbours' */
        double loss = 0.0, gain = 0.0;
        if (k + 1 < L) {
            loss += f->um[(size_t)k * S + y];
            gain += f->vm[(size_t)k * S + y] * N[(size_t)(k + 1) * S + y];
        }
        if (k > 0) {
            loss += f->vm[(size_t)(k - 1) * S + y];
            gain += f->um[(size_t)(k - 1) * S + y] * N[(size_t)(k - 1) * S + y];
        }
        F[y] += (gain - loss * pk[y]) / f->dz[k];
        A[(size_t)y * S + y] += 1.0 / h + loss / f->dz[k];
    }
    free(kf_k);
}

int ora_parcel_system(const ora_problem *p, const double *N, int k, const double *pk, double h,
                      double *F, double *A)
{
    if (k < 0 || k >= p->L || !(h > 0.0))
        return -1;
    parcel_fields f;
    parcel_fields_make(p, N, &f);
    parcel_system(p, &f, N, k, pk, h, F, A);
    parcel_fields_free(&f);
    return 0;
}

/* delta solves A delta = F: partial-pivot LU plus ORA_PARCEL_REFINE refinement sweeps. */
static int dense_solve(int S, const double *A, const double *F, double *delta)
{
    double *LU = malloc(sizeof(double) * ((size_t)S * S + 2 * S));
    double *r = LU + (size_t)S * S, *c = r + S;
    int *piv = malloc(sizeof(int) * S);
    memcpy(LU, A, sizeof(double) * S * S);
    int rc = lu_factor(S, LU, piv);
    if (rc == 0) {
        lu_solve(S, LU, piv, F, delta, 1);
        for (int sweep = 0; sweep < ORA_PARCEL_REFINE; ++sweep) {
            for (int i = 0; i < S; ++i) {
                double acc = F[i];
                for (int j = 0; j < S; ++j)
                    acc -= A[(size_t)i * S + j] * delta[j];
                r[i] = acc;
            }
            lu_solve(S, LU, piv, r, c, 1);
            for (int i = 0; i < S; ++i)
                delta[i] += c[i];
        }
    }
    free(piv);
    free(LU);
    return rc;
}

/* Integrate the parcel x over one visit of layer k (tau_k); *h is the trial step, carried. */
static int parcel_visit(const ora_problem *p, const ora_policy *pol, const parcel_fields *f, const double *N, int k,
                        int max_steps, double *x, double *h, double *A, double *F, double *delta, ora_parcel_info *info)
{
    int S = p->S;
    double tau = f->dz[k] * f->dz[k] / p->Kzz[k];
    double t = 0.0;
    int steps = 0;
    while (t < tau) {
        double rest = tau - t;
        double hs = *h < rest ? *h : rest;
        if (hs > pol->dt_max) hs = pol->dt_max;
        int last = hs >= rest;
        parcel_system(p, f, N, k, x, hs, F, A);
        if (dense_solve(S, A, F, delta) != 0)
            return -1;
        int ok = 1;
        double maxrel = 0.0;
        for (int y = 0; y < S; ++y) {
            double nn = x[y] + delta[y];
            if (!isfinite(nn) || nn < -pol->neg_tol * f->ngas[k]) { ok = 0; break; }
            if (x[y] > pol->f_floor * f->ngas[k]) {
                double rel = fabs(delta[y]) / x[y];
                if (rel > maxrel) maxrel = rel;
            }
        }
        if (ok && maxrel > pol->rel_reject)
            ok = 0;
        if (ok) {
            for (int y = 0; y < S; ++y) {
                double nn = x[y] + delta[y];
                x[y] = nn < 0.0 ? 0.0 : nn;
            }
            t = last ? tau : t + hs;
            double fac = maxrel > 0.0 ? pol->rel_target / maxrel : pol->grow_max;
            if (fac > pol->grow_max) fac = pol->grow_max;
            if (fac < pol->shrink_min) fac = pol->shrink_min;
            double next = hs * fac;
            if (hs < *h && fac >= 1.0 && next < *h)
                next = *h;                 /* cut short by the end of the visit: keep the trial step */
            *h = next;
            ++info->steps;
        } else {
            *h = 0.5 * hs;
            ++info->rejected;
            if (*h < pol->dt_min)
                return -2;
        }
        if (++steps > max_steps)
            return -3;
    }
    return 0;
}

int ora_parcel_iteration(const ora_problem *p, const ora_policy *pol, int max_visit_steps, double *N,
                         ora_parcel_info *info)
{
    int L = p->L, S = p->S;
    size_t LS = (size_t)L * S;
    parcel_fields f;
    parcel_fields_make(p, N, &f);
    double *old = malloc(sizeof(double) * LS);
    double *x = malloc(sizeof(double) * ((size_t)S * S + 4 * S));
    double *A = x + S, *F = A + (size_t)S * S, *delta = F + S, *vmr = delta + S;
    memcpy(old, N, sizeof(double) * LS);
    for (int y = 0; y < S; ++y)
        vmr[y] = N[y] / f.ngas[0];
    info->steps = 0;
    info->rejected = 0;
    int rc = 0;
    for (int v = 0; v < 2 * L - 1 && rc == 0; ++v) {
        int k = v < L ? v : 2 * L - 2 - v;
        for (int y = 0; y < S; ++y)
            x[y] = vmr[y] * f.ngas[k];
        rc = parcel_visit(p, pol, &f, N, k, max_visit_steps, x, &info->h, A, F, delta, info);
        for (int y = 0; y < S; ++y) {
            N[(size_t)k * S + y] = x[y];
            vmr[y] = x[y] / f.ngas[k];
        }
    }
    double change = 0.0;
    for (int k = 0; k < L; ++k)
        for (int y = 0; y < S; ++y) {
            double nv = N[(size_t)k * S + y];
            if (nv > pol->f_floor * f.ngas[k]) {
                double c = fabs(nv - old[(size_t)k * S + y]) / nv;
                if (c > change) change = c;
            }
        }
    info->max_change = change;
    free(x);
    free(old);
    parcel_fields_free(&f);
    return rc;
}

int ora_parcel_run(const ora_problem *p, const ora_policy *pol, int max_visit_steps, int max_iter, double tol,
                   double *N, ora_parcel_info *info, int *iterations)
{
    int it = 0, rc = 0;
    int steps = 0, rejected = 0;
    while (it < max_iter) {
        rc = ora_parcel_iteration(p, pol, max_visit_steps, N, info);
        ++it;
        steps += info->steps;
        rejected += info->rejected;
        if (rc != 0 || info->max_change < tol)
            break;
    }
    info->steps = steps;
    info->rejected = rejected;
    *iterations = it;
    if (rc != 0)
        return rc;
    return info->max_change < tol ? 0 : 1;
}

/* ------------------------------------------- equilibrium initial state */
/*
 * Sec. 2.5, option (i): the initial composition in chemical equilibrium.  Per layer,
 * at the layer's T and P, the ideal-gas mixture of minimum Gibbs energy
 *     G/RT = sum_y N_y (g_y + ln(P/p0) + ln(N_y / N)),   N = sum_y N_y,
 * subject to the element totals sum_y a_ey N_y = b_e, with g_y = G_y/RT from the NASA-7
 * sets (Appendix A).  At the minimum every species satisfies
 *     g_y + ln(P/p0) + ln x_y = sum_e pi_e a_ey
 * with element potentials pi_e.  Solved by Newton iterations on that condition,
 * linearised in ln N_y, ln N and pi (the reduced Gibbs iteration of the NASA
 * equilibrium program, Gordon & McBride 1994): each iteration solves one
 * (E+1) x (E+1) system for pi and d ln N, then sets
 *     d ln N_y = -(g_y + ln(P/p0) + ln N_y - ln N) + sum_e pi_e a_ey + d ln N,
 * with the step limited so that no major species' ln N_y moves by more than 2 and
 * no trace species rises above about 1e-4 of N in one step.  Start: every species
 * 1/S_active, N = 1, b normalised to sum 1.  At convergence the mole fractions are
 * taken from the potentials, x_y = exp(sum_e pi_e a_ey - g_y - ln(P/p0)), normalised,
 * which keeps trace species exact in relative terms.  An element with b_e <= 0 is
 * absent: its potential is not solved for and every species containing it has x = 0.
 */
int ora_equilibrium(const ora_problem *p, const double *b, double *x, int max_iter, double tol, int *iters)
{
    int S = p->S, E = p->E, M = p->E + 1;
    double *lnN = malloc(sizeof(double) * S * 3), *nj = lnN + S, *mu = nj + S;
    double *A = malloc(sizeof(double) * M * (M + 1)), *sol = malloc(sizeof(double) * M);
    int *act = malloc(sizeof(int) * (S + E)), *eact = act + S;
    int worst = 0, rc = 0, notconv = 0;
    for (int k = 0; k < p->L && rc == 0; ++k) {
        const double *bk = b + (size_t)k * E;
        double *xk = x + (size_t)k * S;
        double T = p->T[k], lnP = log(p->P_bar[k]);
        double bsum = 0.0;
        for (int e = 0; e < E; ++e) {
            eact[e] = bk[e] > 0.0;
            if (eact[e]) bsum += bk[e];
        }
        int nact = 0;
        for (int y = 0; y < S; ++y) {
            act[y] = 1;
            for (int e = 0; e < E; ++e)
                if (p->elem[y * E + e] > 0 && !eact[e]) act[y] = 0;
            nact += act[y];
        }
        if (nact == 0 || bsum <= 0.0) { rc = -1; break; }
        for (int y = 0; y < S; ++y)
            lnN[y] = act[y] ? log(1.0 / nact) : 0.0;
        double lntot = 0.0;
        int it, done = 0;
        for (it = 0; it < max_iter; ++it) {
            double ntot = exp(lntot);
            for (int y = 0; y < S; ++y) {
                if (!act[y]) { nj[y] = 0.0; mu[y] = 0.0; continue; }
                nj[y] = exp(lnN[y]);
                mu[y] = ora_gibbs_rt(p->nasa + 15 * y, T) + lnP + lnN[y] - lntot;
            }
            /* the (E+1) x (E+1) system, augmented with its right-hand side in column M */
            for (int i = 0; i < M * (M + 1); ++i)
                A[i] = 0.0;
            for (int i = 0; i < E; ++i) {
                if (!eact[i]) { A[i * (M + 1) + i] = 1.0; continue; }
                for (int j = 0; j < E; ++j) {
                    if (!eact[j]) continue;
                    double s = 0.0;
                    for (int y = 0; y < S; ++y)
                        s += (double)p->elem[y * E + i] * p->elem[y * E + j] * nj[y];
                    A[i * (M + 1) + j] = s;
                }
                double c = 0.0, d = 0.0;
                for (int y = 0; y < S; ++y) {
                    c += p->elem[y * E + i] * nj[y];
                    d += p->elem[y * E + i] * nj[y] * mu[y];
                }
                A[i * (M + 1) + E] = c;
                A[E * (M + 1) + i] = c;
                A[i * (M + 1) + M] = bk[i] / bsum - c + d;
            }
            double sn = 0.0, snm = 0.0;
            for (int y = 0; y < S; ++y) {
                sn += nj[y];
                snm += nj[y] * mu[y];
            }
            A[E * (M + 1) + E] = sn - ntot;
            A[E * (M + 1) + M] = ntot - sn + snm;
            /* Gaussian elimination with partial pivoting */
            for (int c = 0; c < M && rc == 0; ++c) {
                int best = c;
                for (int i = c + 1; i < M; ++i)
                    if (fabs(A[i * (M + 1) + c]) > fabs(A[best * (M + 1) + c])) best = i;
                if (A[best * (M + 1) + c] == 0.0) { rc = -1; break; }
                if (best != c)
                    for (int j = 0; j <= M; ++j) {
                        double t = A[c * (M + 1) + j];
                        A[c * (M + 1) + j] = A[best * (M + 1) + j];
                        A[best * (M + 1) + j] = t;
                    }
                for (int i = c + 1; i < M; ++i) {
                    double l = A[i * (M + 1) + c] / A[c * (M + 1) + c];
                    for (int j = c; j <= M; ++j)
                        A[i * (M + 1) + j] -= l * A[c * (M + 1) + j];
                }
            }
            if (rc) break;
            for (int i = M - 1; i >= 0; --i) {
                double s = A[i * (M + 1) + M];
                for (int j = i + 1; j < M; ++j)
                    s -= A[i * (M + 1) + j] * sol[j];
                sol[i] = s / A[i * (M + 1) + i];
            }
            double dlntot = sol[E];
            /* step limit and convergence measure */
            double big = 5.0 * fabs(dlntot), lam2 = 1.0, conv = 0.0;
            for (int y = 0; y < S; ++y) {
                if (!act[y]) continue;
                double d = -mu[y] + dlntot;
                for (int e = 0; e < E; ++e)
                    if (eact[e]) d += sol[e] * p->elem[y * E + e];
                mu[y] = d;   /* now d ln N_y */
                double lx = lnN[y] - lntot;
                if (lx > log(1e-8)) {
                    if (fabs(d) > big) big = fabs(d);
                } else if (d - dlntot > 0.0) {
                    double v = fabs((-lx - 9.2103) / (d - dlntot));
                    if (v < lam2) lam2 = v;
                }
                conv += nj[y] * fabs(d);
            }
            conv /= sn;
            double lam = 1.0;
            if (big > 2.0) lam = 2.0 / big;
            if (lam2 < lam) lam = lam2;
            for (int y = 0; y < S; ++y)
                if (act[y]) lnN[y] += lam * mu[y];
            lntot += lam * dlntot;
            if (conv < tol && fabs(dlntot) < tol) { done = 1; break; }
        }
        if (rc) break;
        if (it + 1 > worst) worst = it + 1;
        if (!done) { notconv = 1; worst = max_iter; }
        /* mole fractions from the potentials of the last solve, normalised */
        double amax = -INFINITY;
        for (int y = 0; y < S; ++y) {
            if (!act[y]) continue;
            double a = -ora_gibbs_rt(p->nasa + 15 * y, T) - lnP;
            for (int e = 0; e < E; ++e)
                if (eact[e]) a += sol[e] * p->elem[y * E + e];
            xk[y] = a;
            if (a > amax) amax = a;
        }
        double z = 0.0;
        for (int y = 0; y < S; ++y)
            if (act[y]) z += exp(xk[y] - amax);
        for (int y = 0; y < S; ++y)
            xk[y] = act[y] ? exp(xk[y] - amax - log(z)) : 0.0;
    }
    if (iters) *iters = worst;
    free(lnN);
    free(A);
    free(sol);
    free(act);
    return rc ? rc : notconv;
}

/* ------------------------------------------------ reaction pathways */
/*
 * Sec. 4, the reaction-pathway analyser: the kinetically fastest route between two
 * species is the path of least total inverse rate, found with Dijkstra's algorithm.
 * Graph of one layer: each reaction direction with a positive rate q (molecules
 * cm^-3 s^-1; forward q = k_f prod n_reac, reverse q = k_r prod n_prod, photolysis
 * forward only) gives an edge from each species it consumes to each species it
 * produces (other than itself), of weight 1/q.  Edge code = 2 r + direction
 * (0 forward, 1 reverse).  The rate-limiting step of a path is its edge of largest
 * weight (the slowest reaction).
 */
void ora_fluxes(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                const double *n, double *q)
{
    int L = p->L, S = p->S, R = p->R;
    double *kf_k = malloc(sizeof(double) * R * 2), *kr_k = kf_k + R;
    for (int k = 0; k < L; ++k) {
        const double *nk = n + (size_t)k * S;
        layer_rates(p, k, kf, kr, kph, kf_k, kr_k);
        for (int r = 0; r < R; ++r) {
            double wf = kf_k[r], wb = kr_k[r];
            for (int s = 0; s < 3; ++s) {
                if (p->reac[3 * r + s] >= 0) wf *= nk[p->reac[3 * r + s]];
                if (p->prod[3 * r + s] >= 0) wb *= nk[p->prod[3 * r + s]];
            }
            q[((size_t)k * R + r) * 2 + 0] = wf;
            q[((size_t)k * R + r) * 2 + 1] = wb;
        }
    }
    free(kf_k);
}

static int side_has(const int *side3, int y)
{
    return side3[0] == y || side3[1] == y || side3[2] == y;
}

/* Dijkstra from src on the graph of one layer (q: R x 2 rates).  The unfinished species
 * of least distance is taken next (the lower index on ties); an edge replaces a
 * predecessor only when it makes the distance strictly smaller, edges scanned in
 * increasing edge code.  dist = +inf and pred = -1 where unreachable. */
void ora_pathways(const ora_problem *p, const double *q, int src, double *dist, int *pred_sp,
                  int *pred_edge, int *lim_edge, double *lim_w)
{
    int S = p->S, R = p->R;
    int *done = malloc(sizeof(int) * S * 2), *order = done + S;
    for (int y = 0; y < S; ++y) {
        dist[y] = INFINITY;
        pred_sp[y] = -1;
        pred_edge[y] = -1;
        lim_edge[y] = -1;
        lim_w[y] = 0.0;
        done[y] = 0;
    }
    dist[src] = 0.0;
    int nord = 0;
    for (;;) {
        int u = -1;
        for (int y = 0; y < S; ++y)
            if (!done[y] && dist[y] < INFINITY && (u < 0 || dist[y] < dist[u])) u = y;
        if (u < 0) break;
        done[u] = 1;
        order[nord++] = u;
        for (int r = 0; r < R; ++r)
            for (int dir = 0; dir < 2; ++dir) {
                const int *from = dir == 0 ? p->reac + 3 * r : p->prod + 3 * r;
                const int *to = dir == 0 ? p->prod + 3 * r : p->reac + 3 * r;
                double rate = q[(size_t)r * 2 + dir];
                if (!(rate > 0.0) || !side_has(from, u)) continue;
                double w = 1.0 / rate;
                for (int s = 0; s < 3; ++s) {
                    int v = to[s];
                    if (v < 0 || v == u) continue;
                    double cand = dist[u] + w;
                    if (cand < dist[v]) {
                        dist[v] = cand;
                        pred_sp[v] = u;
                        pred_edge[v] = 2 * r + dir;
                    }
                }
            }
    }
    /* slowest step along each path, in the order the species were finished */
    for (int i = 0; i < nord; ++i) {
        int v = order[i], u = pred_sp[v];
        if (u < 0) continue;
        int e = pred_edge[v];
        double w = 1.0 / q[e];
        if (u == src || w > lim_w[u]) {
            lim_edge[v] = e;
            lim_w[v] = w;
        } else {
            lim_edge[v] = lim_edge[u];
            lim_w[v] = lim_w[u];
        }
    }
    free(done);
}

/* ------------------------------------------------------------ BDF integrator */
/*
 * Variable-order, variable-step backward differentiation formulas, the family of the paper's
 * DLSODES (Sec. 2.1, "Commonly used methods"), applied to Eq. 1 on the Eulerian grid.  Order q uses
 * the accepted states at tau_1 > ... > tau_q and asks that the interpolating polynomial through them
 * and the new state at tau_0 = t + h have the derivative F at tau_0:
 *     c_0 y_new + sum_{j>=1} c_j y(tau_j) = F(y_new),   c_j = l_j'(tau_0)  (Lagrange basis).
 * Linearly implicit: F is linearised once about the predictor y_hat (the polynomial through the
 * last q+1 states, fewer at the start, evaluated at tau_0), so each step solves
 *     (c_0 I - J(y_hat)) delta = F(y_hat) - c_0 y_hat - sum_{j>=1} c_j y(tau_j),   y_new = y_hat + delta
 * with the same block-tridiagonal solve as the backward-Euler step (q = 1 with y_hat = y_n is that
 * step exactly).
 * Error control: the local error of order q is estimated as (y_new - y_hat) / (q + 1) and measured
 * relative to y_new over species above f_floor mixing ratio, in units of rtol (err <= 1 accepts).
 * A step is also rejected when y_new is non-finite or below -neg_tol n_gas.  On rejection h shrinks
 * by max(0.2, min(0.9, 0.9 err^{-1/(q+1)})) (0.25 for a bad state) and, after two rejections in a
 * row, the order drops by one.  On acceptance negatives are clipped to zero, and after q + 1 steps
 * at one order the next order is chosen among q - 1, q, q + 1 by the largest step factor
 * eta = err_q'^{-1/(q'+1)} (divided by 1.3, 1.2, 1.4 respectively, favouring the current order),
 * err_q' being the same estimate with the predictor of degree q'; otherwise eta = eta_q / 1.2.  The
 * next step is h * clamp(eta, 0.2, grow), at most dt_max and no further than t_end.
 */
void ora_bdf_coeffs(int q, const double *tau, double *c)
{
    double c0 = 0.0;
    for (int m = 1; m <= q; ++m)
        c0 += 1.0 / (tau[0] - tau[m]);
    c[0] = c0;
    for (int j = 1; j <= q; ++j) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m <= q; ++m) {
            if (m == j) continue;
            if (m != 0) num *= tau[0] - tau[m];
            den *= tau[j] - tau[m];
        }
        c[j] = num / den;
    }
}

void ora_bdf_extrap(int m, const double *tau, double t, double *w)
{
    for (int j = 0; j < m; ++j) {
        double v = 1.0;
        for (int i = 0; i < m; ++i)
            if (i != j) v *= (t - tau[i]) / (tau[j] - tau[i]);
        w[j] = v;
    }
}

#define ORA_BDF_QMAX 5

/* max over entries with y > floor n_gas of |y - yp| / (K rtol y) */
static double bdf_err(const ora_problem *p, const double *ngas, double f_floor, const double *y,
                      const double *yp, double K, double rtol)
{
    double e = 0.0;
    for (int k = 0; k < p->L; ++k)
        for (int s = 0; s < p->S; ++s) {
            size_t i = (size_t)k * p->S + s;
            if (y[i] > f_floor * ngas[k]) {
                double v = fabs(y[i] - yp[i]) / (K * rtol * y[i]);
                if (v > e) e = v;
            }
        }
    return e;
}

int ora_bdf_run(const ora_problem *p, const ora_policy *pol, const ora_bdf_config *cfg, double *n,
                double h0, double t_end, int stop_at_steady, int max_steps, ora_bdf_info *info)
{
    int L = p->L, S = p->S, R = p->R;
    size_t LS = (size_t)L * S;
    int qmax = cfg->qmax < 1 ? 1 : (cfg->qmax > ORA_BDF_QMAX ? ORA_BDF_QMAX : cfg->qmax);
    int HMAX = qmax + 2;                          /* states kept: enough for the order q+1 predictor */
    double *Y = malloc(sizeof(double) * LS * HMAX), th[ORA_BDF_QMAX + 2];
    double *yhat = malloc(sizeof(double) * LS * 6), *g = yhat + LS, *rhs = g + LS, *delta = rhs + LS;
    double *ynew = delta + LS, *yalt = ynew + LS;
    double *kf = malloc(sizeof(double) * (size_t)L * R * 2), *kr = kf + (size_t)L * R;
    double *kph = malloc(sizeof(double) * (size_t)L * (p->Rph > 0 ? p->Rph : 1));
    double *F = malloc(sizeof(double) * LS * 3), *lo = F + LS, *up = lo + LS;
    double *A = malloc(sizeof(double) * LS * S);
    double *ngas = malloc(sizeof(double) * L * 4);
    ora_grid(p, ngas, ngas + L, ngas + 2 * L, ngas + 3 * L);
    ora_rate_coefficients(p, kf, kr);
    memset(info, 0, sizeof(*info));
    memcpy(Y, n, sizeof(double) * LS);
    th[0] = 0.0;
    int hist = 1, q = 1, nq = 0, nrej = 0, rc = 1;
    double t = 0.0, h = h0;
    if (h > t_end - t) h = t_end - t;
    while (info->steps < max_steps) {
        info->steps++;
        int qe = q < hist ? q : hist;
        double tau[ORA_BDF_QMAX + 2], c[ORA_BDF_QMAX + 1], w[ORA_BDF_QMAX + 2];
        tau[0] = t + h;
        for (int j = 1; j <= qe; ++j) tau[j] = th[j - 1];
        ora_bdf_coeffs(qe, tau, c);
        int m = qe + 1 < hist ? qe + 1 : hist;
        ora_bdf_extrap(m, th, t + h, w);
        for (size_t i = 0; i < LS; ++i) {
            double v = 0.0;
            for (int j = 0; j < m; ++j) v += w[j] * Y[(size_t)j * LS + i];
            yhat[i] = v;
        }
        for (size_t i = 0; i < LS; ++i) {
            double v = c[0] * yhat[i];
            for (int j = 1; j <= qe; ++j) v += c[j] * Y[(size_t)(j - 1) * LS + i];
            g[i] = v;
        }
        ora_photolysis(p, yhat, kph);
        ora_residual(p, kf, kr, kph, yhat, F);
        for (size_t i = 0; i < LS; ++i) rhs[i] = F[i] - g[i];
        ora_jacobian(p, kf, kr, kph, yhat, 1.0 / c[0], A, lo, up);
        if (ora_block_solve_refined(L, S, A, lo, up, rhs, delta, ORA_REFINE_SWEEPS) != 0) { rc = -1; break; }
        int bad = 0;
        for (int k = 0; k < L; ++k)
            for (int s = 0; s < S; ++s) {
                size_t i = (size_t)k * S + s;
                ynew[i] = yhat[i] + delta[i];
                if (!isfinite(ynew[i]) || ynew[i] < -pol->neg_tol * ngas[k]) bad = 1;
            }
        double err = bad ? INFINITY : bdf_err(p, ngas, pol->f_floor, ynew, yhat, qe + 1.0, cfg->rtol);
        info->err = err;
        if (cfg->fixed_step) {
            if (bad) { rc = -2; break; }
            err = 0.0;
        }
        if (bad || err > 1.0) {
            info->rejected++;
            nrej++;
            double f = bad ? 0.25 : 0.9 * pow(err, -1.0 / (qe + 1));
            if (!bad) { if (f > 0.9) f = 0.9; if (f < 0.2) f = 0.2; }
            h *= f;
            if (nrej >= 2 && q > 1) { q--; nq = 0; }
            if (h < pol->dt_min) { rc = -2; break; }
            continue;
        }
        /* accepted */
        double relc = 0.0;
        for (int k = 0; k < L; ++k)
            for (int s = 0; s < S; ++s) {
                size_t i = (size_t)k * S + s;
                if (ynew[i] > pol->f_floor * ngas[k]) {
                    double v = fabs(ynew[i] - Y[i]) / ynew[i];
                    if (v > relc) relc = v;
                }
            }
        /* order choice (needs the old history for the other predictors) */
        double eta = pow(err > 1e-10 ? err : 1e-10, -1.0 / (qe + 1)) / 1.2;
        int qnew = q;
        nq++;
        if (!cfg->fixed_order && nq >= qe + 1) {
            if (qe > 1) {
                ora_bdf_extrap(qe, th, t + h, w);
                for (size_t i = 0; i < LS; ++i) {
                    double v = 0.0;
                    for (int j = 0; j < qe; ++j) v += w[j] * Y[(size_t)j * LS + i];
                    yalt[i] = v;
                }
                double e1 = bdf_err(p, ngas, pol->f_floor, ynew, yalt, (double)qe, cfg->rtol);
                double eta1 = pow(e1 > 1e-10 ? e1 : 1e-10, -1.0 / qe) / 1.3;
                if (eta1 > eta) { eta = eta1; qnew = qe - 1; }
            }
            if (qe < qmax && hist >= qe + 2) {
                ora_bdf_extrap(qe + 2, th, t + h, w);
                for (size_t i = 0; i < LS; ++i) {
                    double v = 0.0;
                    for (int j = 0; j < qe + 2; ++j) v += w[j] * Y[(size_t)j * LS + i];
                    yalt[i] = v;
                }
                double e2 = bdf_err(p, ngas, pol->f_floor, ynew, yalt, qe + 2.0, cfg->rtol);
                double eta2 = pow(e2 > 1e-10 ? e2 : 1e-10, -1.0 / (qe + 2)) / 1.4;
                if (eta2 > eta) { eta = eta2; qnew = qe + 1; }
            }
            if (qnew != q) nq = 0;
        }
        if (cfg->fixed_order > 0) qnew = cfg->fixed_order > qmax ? qmax : cfg->fixed_order;
        /* push the state (negatives clipped) */
        for (int j = HMAX - 1; j > 0; --j) {
            memcpy(Y + (size_t)j * LS, Y + (size_t)(j - 1) * LS, sizeof(double) * LS);
            th[j] = th[j - 1];
        }
        for (size_t i = 0; i < LS; ++i) Y[i] = ynew[i] < 0.0 ? 0.0 : ynew[i];
        th[0] = t + h;
        if (hist < HMAX) hist++;
        info->accepted++;
        info->order_steps[qe]++;
        nrej = 0;
        double hused = h;
        t += h;
        q = qnew;
        if (!cfg->fixed_step) {
            if (eta < 0.2) eta = 0.2;
            if (eta > cfg->grow) eta = cfg->grow;
            h *= eta;
            if (h > pol->dt_max) h = pol->dt_max;
        }
        info->max_rel = relc;
        if (stop_at_steady && hused >= pol->ss_dt && relc < pol->ss_tol) { info->converged = 1; rc = 0; break; }
        if (t >= t_end * (1.0 - 1e-12)) { rc = 0; break; }
        if (h > t_end - t) h = t_end - t;
    }
    info->t = t;
    info->h = h;
    info->q = q;
    memcpy(n, Y, sizeof(double) * LS);
    free(Y); free(yhat); free(kf); free(kph); free(F); free(A); free(ngas);
    return rc;
}

/* ------------------------------------- photolysis rates in the Jacobian */
/*
 * dk_ph / dn of the direct beam (Sec. 2.3.3): k_ph,q,k = t_f sum_w J_kw sigma_qw dlambda_w with
 * J_kw = J0_w exp(-tau_kw / mu) and tau_kw = sum_{j>k} e_jw dz_j + e_kw dz_k / 2, e_jw =
 * sum_i (sigma_a,iw + sigma_s,iw) n_ji.  So dk_ph,q,k / dn_ji = -(t_f / mu) sum_w J_kw sigma_qw
 * dlambda_w (sigma_a,iw + sigma_s,iw) c_kj dz_j, with c_kj = 1 above k, 1/2 at k, 0 below: a
 * species absorbs for every layer beneath it.  Written out for every (k, q) and (j, i):
 * dk [(k Rph + q)][(j S + i)].  The diffuse field's derivative is not included.
 */
void ora_photolysis_dn(const ora_problem *p, const double *n, double *dk)
{
    int L = p->L, S = p->S, W = p->W, Rph = p->Rph;
    size_t LS = (size_t)L * S;
    memset(dk, 0, sizeof(double) * (size_t)L * Rph * LS);
    if (Rph == 0 || W == 0)
        return;
    double *ngas = malloc(sizeof(double) * L * 4);
    double *z = ngas + L, *dz = z + L, *dzi = dz + L;
    ora_grid(p, ngas, z, dz, dzi);
    double *J = malloc(sizeof(double) * (size_t)L * W), *ext = malloc(sizeof(double) * L);
    for (int w = 0; w < W; ++w) {
        for (int k = 0; k < L; ++k) {
            double s = 0.0;
            for (int i = 0; i < S; ++i) {
                double sg = p->sigma_abs[(size_t)i * W + w] + (p->sigma_s ? p->sigma_s[(size_t)i * W + w] : 0.0);
                s += sg * n[(size_t)k * S + i];
            }
            ext[k] = s;
        }
        double above = 0.0;
        for (int k = L - 1; k >= 0; --k) {
            double tau = above + 0.5 * ext[k] * dz[k];
            J[(size_t)k * W + w] = p->J0[w] * exp(-tau / p->mu);
            above += ext[k] * dz[k];
        }
    }
    for (int k = 0; k < L; ++k)
        for (int q = 0; q < Rph; ++q) {
            double *row = dk + ((size_t)k * Rph + q) * LS;
            for (int j = k; j < L; ++j) {
                double c = (j == k) ? 0.5 : 1.0;
                for (int i = 0; i < S; ++i) {
                    double s = 0.0;
                    for (int w = 0; w < W; ++w) {
                        double sg = p->sigma_abs[(size_t)i * W + w] + (p->sigma_s ? p->sigma_s[(size_t)i * W + w] : 0.0);
                        if (sg == 0.0) continue;
                        s += J[(size_t)k * W + w] * p->sigma[(size_t)q * W + w] * p->dlam[w] * sg;
                    }
                    row[(size_t)j * S + i] = -(p->tf / p->mu) * s * c * dz[j];
                }
            }
        }
    free(ext);
    free(J);
    free(ngas);
}

/* The linearly implicit step with the photolysis rates differentiated as well: (I/dt - J_full) delta
 * = F(n), J_full = the block-tridiagonal Jacobian plus, for every photolysis reaction r (A -> ...)
 * in layer k, nu_yr n_A,k dk_ph,r,k / dn (a coupling to every layer at and above k), solved as one
 * dense system by Gaussian elimination with partial pivoting and FP64 iterative refinement.
 * Returns 0, or -1 on a singular matrix. */
int ora_step_delta_coupled(const ora_problem *p, const double *n, double dt, double *delta)
{
    int L = p->L, S = p->S, R = p->R, Rph = p->Rph;
    size_t LS = (size_t)L * S;
    double *kf = malloc(sizeof(double) * (size_t)L * R * 2), *kr = kf + (size_t)L * R;
    double *kph = malloc(sizeof(double) * (size_t)L * (Rph > 0 ? Rph : 1));
    double *F = malloc(sizeof(double) * LS * 3), *lo = F + LS, *up = lo + LS;
    double *A = malloc(sizeof(double) * LS * S);
    double *M = malloc(sizeof(double) * LS * LS), *LU = malloc(sizeof(double) * LS * LS);
    double *dk = malloc(sizeof(double) * (size_t)L * (Rph > 0 ? Rph : 1) * LS);
    double *r = malloc(sizeof(double) * LS * 2), *c = r + LS;
    int *piv = malloc(sizeof(int) * LS);
    ora_rate_coefficients(p, kf, kr);
    ora_photolysis(p, n, kph);
    ora_residual(p, kf, kr, kph, n, F);
    ora_jacobian(p, kf, kr, kph, n, dt, A, lo, up);
    ora_photolysis_dn(p, n, dk);
    memset(M, 0, sizeof(double) * LS * LS);
    for (int k = 0; k < L; ++k)
        for (int y = 0; y < S; ++y) {
            size_t row = (size_t)k * S + y;
            for (int x = 0; x < S; ++x)
                M[row * LS + (size_t)k * S + x] = A[((size_t)k * S + y) * S + x];
            if (k > 0) M[row * LS + (size_t)(k - 1) * S + y] = lo[row];
            if (k + 1 < L) M[row * LS + (size_t)(k + 1) * S + y] = up[row];
        }
    /* minus d(photolysis production - loss)/dn through the rates */
    for (int rr = 0; rr < R; ++rr) {
        if (p->rtype[rr] != 2) continue;
        int q = p->prow[rr], a = p->reac[3 * rr];
        for (int k = 0; k < L; ++k) {
            const double *drow = dk + ((size_t)k * Rph + q) * LS;
            double na = n[(size_t)k * S + a];
            for (int s = 0; s < 3; ++s) {
                int yr = p->reac[3 * rr + s], yp = p->prod[3 * rr + s];
                for (size_t col = 0; col < LS; ++col) {
                    double v = na * drow[col];
                    if (v == 0.0) continue;
                    if (yr >= 0) M[((size_t)k * S + yr) * LS + col] += v;   /* loss: -(-v) */
                    if (yp >= 0) M[((size_t)k * S + yp) * LS + col] -= v;   /* production */
                }
            }
        }
    }
    memcpy(LU, M, sizeof(double) * LS * LS);
    int rc = lu_factor((int)LS, LU, piv);
    if (rc == 0) {
        lu_solve((int)LS, LU, piv, F, delta, 1);
        for (int sweep = 0; sweep < ORA_REFINE_SWEEPS; ++sweep) {
            for (size_t i = 0; i < LS; ++i) {
                double s = F[i];
                for (size_t j = 0; j < LS; ++j)
                    s -= M[i * LS + j] * delta[j];
                r[i] = s;
            }
            lu_solve((int)LS, LU, piv, r, c, 1);
            for (size_t i = 0; i < LS; ++i)
                delta[i] += c[i];
        }
    }
    free(piv); free(r); free(dk); free(LU); free(M); free(A); free(F); free(kph); free(kf);
    return rc;
}
