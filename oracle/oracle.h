/*
 * Plain FP64 CPU oracle of the implicit photochemical-kinetics step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA path; both start from the same raw inputs
 * (element vectors, reaction lists, rate parameters, NASA-7 sets, cross
 * sections, profiles) and compute everything else on their own.
 *
 * Every quantity is FP64.  Layout is row-major; layer 0 is the bottom of the
 * atmosphere.  Units: cgs, pressure input in bar, wavelength in Angstrom.
 */
#ifndef XK_ORACLE_H
#define XK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int S, E, R, L, W, Rph;
    const int *elem;        /* S x E */
    const double *mass;     /* S (u) */
    const int *rtype;       /* R: 0 two-body, 1 three-body, 2 photolysis */
    const int *reac;        /* R x 3, -1 pad */
    const int *prod;        /* R x 3, -1 pad */
    const double *arr;      /* R x 9 */
    const double *troe;     /* R x 4: a, T***, T*, T**; a == 0 -> Lindemann */
    const int *form;        /* R: 0 Kooij, 1 modified Arrhenius */
    const double *nasa;     /* S x 15: Tmid, low a1..a7, high a1..a7 */
    const int *prow;        /* R: sigma row of a photolysis reaction, else -1 */
    const double *lam, *dlam, *J0;   /* W */
    const double *sigma;    /* Rph x W */
    const double *sigma_abs;/* S x W */
    double mu, tf;
    const double *P_bar, *T, *Kzz;   /* L */
    const double *dcoef;    /* S */
    double g, mbar, alpha_T;
    /* Sec. 2.3.3 extinction and diffuse field (optional): sigma_s S x W Rayleigh scattering cross
     * sections (NULL: none), albedo of the lower boundary, diffuse = 1 adds J_diff to the beam */
    const double *sigma_s;
    double albedo;
    int diffuse;
} ora_problem;

typedef struct {
    double dt_max;      /* largest step (s) */
    double rel_reject;  /* reject when max relative change exceeds this */
    double rel_target;  /* step-size controller target relative change */
    double grow_max, shrink_min;
    double neg_tol;     /* reject when n < -neg_tol * n_gas */
    double f_floor;     /* relative change measured over species with f > f_floor */
    double dt_min;      /* give up below this step */
    double ss_dt;       /* steady state needs dt >= ss_dt ... */
    double ss_tol;      /* ... and max relative change < ss_tol */
} ora_policy;

typedef struct {
    int accepted;       /* 1 accepted, 0 rejected */
    double dt_used, dt_next, max_rel;
    int n_neg;          /* entries clipped to zero on acceptance */
} ora_step_info;

typedef struct {
    int converged, steps, accepted, rejected;
    double t, dt, max_rel;
} ora_run_info;

/* Sec. 2.1: n_gas = P / (k_B T); hydrostatic altitudes; layer and interface widths. */
void ora_grid(const ora_problem *p, double *ngas, double *z, double *dz, double *dzi);
/* Appendix A: G/RT and Cp/R of one NASA-7 set at temperature T. */
double ora_gibbs_rt(const double *nasa15, double T);
double ora_cp_r(const double *nasa15, double T);
/* Sec. 2.3.4: G/RT per layer and species, ln K_c per layer and reaction. */
void ora_thermo(const ora_problem *p, double *grt, double *lnkc);
/* Sec. 2.3.1-2.3.4: thermal k_f and k_r per layer and reaction (photolysis rows 0). */
void ora_rate_coefficients(const ora_problem *p, double *kf, double *kr);
/* Sec. 2.3.3: photolysis rate constants per layer and photolysis reaction. */
void ora_photolysis(const ora_problem *p, const double *n, double *kph);
/* Sec. 2.3.3 diffuse field of one wavelength on L layers: dtau_a, dtau_s [L] absorption and
 * scattering optical thickness of each layer (layer 0 at the bottom), beam photon flux F0 at the top
 * with cos(zenith) mu, lower-boundary albedo.  U, D [L+1]: upward and downward diffuse fluxes
 * (photons per unit horizontal area) crossing interface i (0 bottom, L top); Jdiff [L] =
 * (J_up + J_down) / 2 per layer, each the mean of the layer's two interfaces.  Returns 0 or -1. */
int ora_two_stream(int L, const double *dtau_a, const double *dtau_s, double F0, double mu, double albedo,
                   double *U, double *D, double *Jdiff);
/* Eq. 2: interface flux phi_{k+1/2} = u n_k - v n_{k+1}, per interface and species. */
void ora_transport(const ora_problem *p, double *u, double *v);
/* Eq. 1: F = P - L - d(phi)/dz at state n (kf/kr/kph supplied). */
void ora_residual(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                  const double *n, double *F);
/* Block-tridiagonal matrix I/dt - dF/dn: dense diagonal blocks A[L][S][S],
 * diagonal couplings lo[L][S] (to layer k-1) and up[L][S] (to layer k+1). */
void ora_jacobian(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                  const double *n, double dt, double *A, double *lo, double *up);
/* Block Thomas with partial-pivot LU per block; A is overwritten.  Returns 0 or -1 (singular). */
int ora_block_solve(int L, int S, double *A, const double *lo, const double *up,
                    const double *f, double *x);
/* The same solve followed by `sweeps` rounds of FP64 iterative refinement with the
 * stored factors (A, lo, up unchanged). */
int ora_block_solve_refined(int L, int S, const double *A, const double *lo, const double *up,
                            const double *f, double *x, int sweeps);
/* One linearly implicit backward-Euler step of size dt: delta solves (I/dt - J) delta = F
 * (block Thomas plus FP64 iterative refinement). */
int ora_step_delta(const ora_problem *p, const double *n, double dt, double *delta);
/* One controlled step: accept/reject, clip, next dt.  n is updated when accepted. */
int ora_step(const ora_problem *p, const ora_policy *pol, double *n, double dt, ora_step_info *info);
/* Steps from dt0 until steady state or max_steps. */
int ora_run_to_steady(const ora_problem *p, const ora_policy *pol, double *n, double dt0,
                      int max_steps, ora_run_info *info);

/* Lagrangian parcel scheme (Sec. 2, Fig. 2).  The parcel's system in layer k with densities
 * pk: F = chemistry of layer k at pk plus the molecular-diffusion exchange with the stored
 * densities N of layers k -+ 1, and A = I/h - dF/dpk (S x S row-major).  0 or -1. */
int ora_parcel_system(const ora_problem *p, const double *N, int k, const double *pk, double h,
                      double *F, double *A);
typedef struct {
    double h;           /* in: the first trial step (s); out: the trial step after the last visit */
    int steps;          /* accepted implicit steps (of the iteration; of the run for ora_parcel_run) */
    int rejected;       /* rejected trial steps */
    double max_change;  /* largest |N_new - N_old| / N_new over entries above f_floor mixing ratio */
} ora_parcel_info;
/* One global iteration (bottom to top and back) on the stored profile N [L][S], updated in
 * place; each visit integrated under the step controller of pol.  0; -1 singular visit
 * system; -2 step below dt_min; -3 more than max_visit_steps steps in one visit. */
int ora_parcel_iteration(const ora_problem *p, const ora_policy *pol, int max_visit_steps, double *N,
                         ora_parcel_info *info);
/* Global iterations until info->max_change < tol (returns 0) or max_iter (returns 1); a
 * negative return as ora_parcel_iteration.  info->h is the first trial step. */
int ora_parcel_run(const ora_problem *p, const ora_policy *pol, int max_visit_steps, int max_iter, double tol,
                   double *N, ora_parcel_info *info, int *iterations);

/* Sec. 2.5 option (i): chemical-equilibrium composition per layer at the layer's T and P, the
 * ideal-gas mixture of minimum Gibbs energy with element totals b [L][E] (any common unit; an
 * element with b <= 0 is absent).  x [L][S] receives mole fractions (sum 1).  Returns 0, 1 when a
 * layer did not converge within max_iter (tol on the Newton update of ln N_y and ln N), -1 on a
 * singular system.  *iters: the most iterations any layer took. */
int ora_equilibrium(const ora_problem *p, const double *b, double *x, int max_iter, double tol, int *iters);
/* Forward and reverse rate of every reaction in every layer at state n: q [L][R][2] (molecules
 * cm^-3 s^-1; photolysis forward only). */
void ora_fluxes(const ora_problem *p, const double *kf, const double *kr, const double *kph,
                const double *n, double *q);
/* Sec. 4 reaction-pathway analyser on one layer (q: that layer's [R][2] rates): Dijkstra from src
 * with edge weights 1/q from each consumed to each produced species.  dist [S] (+inf unreachable),
 * pred_sp [S] predecessor species, pred_edge [S] edge code 2 r + direction (0 forward, 1 reverse),
 * lim_edge / lim_w [S] the slowest step of the path and its weight; -1 where there is none. */
void ora_pathways(const ora_problem *p, const double *q, int src, double *dist, int *pred_sp,
                  int *pred_edge, int *lim_edge, double *lim_w);

/* Variable-order, variable-step BDF (the integrator family of the paper's DLSODES, Sec. 2.1),
 * linearly implicit: one Newton iteration per step on the block-tridiagonal system.
 * ora_bdf_coeffs: c[0..q] with y'(tau_0) ~ sum_j c_j y(tau_j) on nodes tau_0 > tau_1 > ... > tau_q
 * (derivatives of the Lagrange basis at tau_0); ora_bdf_extrap: w[0..m-1] with
 * y(t) ~ sum_j w_j y(tau_j) over m nodes (the degree m-1 interpolant at t). */
void ora_bdf_coeffs(int q, const double *tau, double *c);
void ora_bdf_extrap(int m, const double *tau, double t, double *w);
typedef struct {
    double rtol;        /* local error target, relative, on species above f_floor mixing ratio */
    int qmax;           /* largest order (1..5) */
    int fixed_order;    /* > 0: no order selection, this order once enough history exists */
    int fixed_step;     /* 1: every step h0 (no error control; for order-of-accuracy checks) */
    double grow;        /* largest step growth factor per step */
} ora_bdf_config;
typedef struct {
    int steps, accepted, rejected, converged;
    int order_steps[6]; /* accepted steps per order */
    double t, h, max_rel;
    int q;
    double err;         /* local-error estimate of the last attempt, in units of rtol */
} ora_bdf_info;
/* Integrates n from t = 0 to t_end (or to steady state when stop_at_steady), starting with step h0
 * at order 1; n is updated.  Returns 0 (reached t_end or steady state), 1 (max_steps), -1 (a
 * singular system), -2 (step below pol->dt_min). */
int ora_bdf_run(const ora_problem *p, const ora_policy *pol, const ora_bdf_config *cfg, double *n,
                double h0, double t_end, int stop_at_steady, int max_steps, ora_bdf_info *info);

/* Sec. 2.3.3: derivative of the direct-beam photolysis rates with respect to every density of the
 * column: dk [L*Rph][L*S] (the diffuse field's derivative not included). */
void ora_photolysis_dn(const ora_problem *p, const double *n, double *dk);
/* The linearly implicit step with the photolysis rates differentiated too (every layer couples to
 * the layers above it), one dense FP64 solve with iterative refinement: small columns only. */
int ora_step_delta_coupled(const ora_problem *p, const double *n, double dt, double *delta);

#ifdef __cplusplus
}
#endif
#endif
