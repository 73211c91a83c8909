/*
 * libxk — implicit time step of the 1-D photochemical kinetics system
 * (stiff chemistry plus vertical transport) on one NVIDIA GB300 (sm_103a).
 *
 * The problem is the one stated in the paper's model description (Ghosh et
 * al., XODIAC): the continuity equation dn_y/dt = P_y - L_y - dphi_y/dz
 * (Eq. 1) with the eddy + molecular-diffusion flux of Eq. 2, rate
 * coefficients of Sec. 2.3 (Kooij / modified Arrhenius, Lindemann three-body,
 * photolysis from the attenuated stellar flux, reverse rates from the Gibbs
 * energy of reaction with NASA-7 polynomials of Appendix A), and zero-flux
 * top and bottom boundaries (Sec. 2.5).  It is integrated by linearly
 * implicit (backward) Euler steps: (I/dt - J) delta = F(n), solved with a
 * block-tridiagonal LU (block Thomas) whose diagonal blocks are the dense
 * species-by-species chemistry Jacobians of each layer and whose couplings
 * are the diagonal transport terms.
 *
 * Conventions for every call:
 *  - return value: XK_OK (0) or a negative XK_E* code; xk_last_error() gives
 *    a message for the last failing call on that context.
 *  - host arrays are owned by the caller and copied in; row-major (C order).
 *  - layer 0 is the bottom of the atmosphere; state arrays are [L][S].
 *  - units: cgs; pressure in bar; wavelength in Angstrom; densities cm^-3.
 *  - device memory: the library allocates none for a column; the caller
 *    provides one device workspace (xk_workspace_bytes / xk_set_workspace),
 *    e.g. a PyTorch uint8 tensor.  The caller keeps it alive until
 *    xk_destroy.  Work is issued on the stream given in xk_config.
 *  - pointers documented as "device" must be device memory of the context's
 *    GPU; "host" pointers host memory.  Calls taking both say which.
 */
#ifndef XK_H
#define XK_H

#include <stddef.h>

#if defined(__GNUC__)
#define XK_API __attribute__((visibility("default")))
#else
#define XK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define XK_OK 0
#define XK_EINVAL (-1)    /* bad argument: shape, index, NaN input, order of calls */
#define XK_ENOMEM (-2)    /* workspace too small / footprint over budget */
#define XK_ENOCONV (-3)   /* no steady state within max steps / solver did not converge */
#define XK_ENEG (-4)      /* step size fell below dt_min (positivity could not be kept) */
#define XK_ECUDA (-5)     /* CUDA runtime error */
#define XK_ESINGULAR (-6) /* zero pivot in a diagonal block */
#define XK_ETIMEOUT (-7)  /* a bounded device-side wait gave up */

#define XK_PREC_FP64 0    /* FP64 block LU (plain path) */
#define XK_PREC_MIXED 1   /* FP32 block LU as preconditioner + FP64 GMRES refinement; a step whose
                             GMRES does not reach gmres_tol within gmres_max_iter is re-solved with
                             the FP64 block LU, and so is every later step at that dt or above */

#define XK_RX_TWO_BODY 0
#define XK_RX_THREE_BODY 1
#define XK_RX_PHOTO 2

typedef struct xk_ctx xk_ctx;

typedef struct {
    int precision;        /* XK_PREC_FP64 or XK_PREC_MIXED */
    int device;           /* CUDA device ordinal */
    void *stream;         /* cudaStream_t to issue work on (NULL: legacy default stream) */
    /* step control (same policy as the CPU reference): */
    double dt_max;        /* largest step (s) */
    double rel_reject;    /* reject a step whose max relative change exceeds this */
    double rel_target;    /* next dt = dt * clamp(rel_target / max_rel, shrink_min, grow_max) */
    double grow_max, shrink_min;
    double neg_tol;       /* reject when any n + delta < -neg_tol * n_gas */
    double f_floor;       /* relative change is measured over species with n > f_floor n_gas */
    double dt_min;        /* give up (XK_ENEG) below this step */
    double ss_dt;         /* steady state: accepted step with dt >= ss_dt ... */
    double ss_tol;        /* ... and max relative change < ss_tol */
    /* mixed precision solver: */
    int gmres_restart;    /* Krylov basis size m of FGMRES(m) */
    int gmres_max_iter;   /* total iterations per linear solve */
    double gmres_tol;     /* relative residual target in the scaled (relative) variables (1e-15) */
    /* factorization tuning (0: chosen by the library / autotuner) */
    int panel_width;      /* columns per panel of the blocked Gauss-Jordan block inversion */
    int factor_ctas;      /* CTAs of the persistent factorization kernel per column */
    int fp32_pivoting;    /* mixed mode: 0 (default) FP32 inversion without row pivoting, 1 with
                             implicit partial pivoting (grid-wide kernel) */
    int reuse_factorization; /* mixed mode: 1 = once steps go to FP64, precondition FGMRES on the
                             current FP64 operator with the last FP64 factorization (rescaled to
                             the current variables) and refactor only when FGMRES misses its
                             tolerance; 0 (default) = factor every step */
    int cluster_size;     /* mixed mode without pivoting: CTAs of the thread-block cluster that
                             holds each layer's FP32 block in distributed shared memory while it is
                             inverted (1..16; 0 = the largest that fits; -1 = grid-wide kernel with
                             the block in global memory).  panel_width 8 or 16 applies (default 8). */
    int reuse_max_iters;  /* with reuse_factorization: a solve on the reused FP64 factorization that
                             needs more FGMRES iterations than this (default 40; an iteration costs
                             about one FP64 sweep pair, a fresh factorization a few hundred) makes
                             the next FP64 step refactor */
    int twisted;          /* mixed mode, cluster-resident inversion: 1 (default) eliminates from both
                             ends of the column at once on two clusters and meets in the middle
                             layer (when two clusters fit and there are at least 3 layers); 0 keeps
                             the single top-down chain */
    int fp64_panel;       /* FP64 block inversion: 0 (default) runs Gauss-Jordan with partial
                             pivoting on each panel column by column on one CTA (panel width 8 or
                             16); 1 chooses each panel's pivots first on one CTA (elimination of the
                             unpivoted rows only) and forms the panel's multipliers on all CTAs by
                             triangular solves with the pivot block's LU factors (8, 16 or 32) */
    int refine_max_iter;  /* FGMRES iterations in FP64 on the exact FP64 operator around an FP64
                             factorization, used as the preconditioner: the plain FP64 path and the
                             mixed path's FP64 route (default 10; stops at gmres_tol).  A direct solve
                             with stored block inverses carries their backward error times the
                             system's condition number; the iterations bring the residual down to
                             gmres_tol.  0 = direct solve only */
    int fp32_bcr;         /* mixed mode: 1 factors the FP32 preconditioner by block cyclic reduction of
                             the layers (odd layers eliminated first, level by level) with every dense
                             product on the tensor cores (TF32 head/tail split, FP32 accuracy) and the
                             leaf block inversions in FP32 on the CUDA cores (the default); 0 by the
                             chain of block inversions
                             (cluster_size, panel_width, twisted, fp32_pivoting then apply) */
    long long wait_polls; /* every device-side wait on other CTAs (the grid barriers of the FP64
                             factorization) gives up after this many polls, about 0.1 us each, and
                             the call returns XK_ETIMEOUT with the context still usable (0: 2^24
                             polls, one to two seconds) */
    int use_graphs;       /* 1 (default): xk_run_to_steady and the batch calls capture a chunk of
                             controlled steps (every kernel of every step, with the device-side
                             gating of FGMRES iterations and of the FP64 route) in a CUDA graph once
                             and replay it, one graph launch per chunk; 0 launches every kernel from
                             the host.  Tracing (xk_profile) launches from the host either way. */
    int photo_jacobian;   /* 1: the direct-beam photolysis rates are differentiated too (Sec. 2.3.3): the
                             operator of FGMRES (mixed path; the refinement iterations of the FP64 path)
                             includes dk_ph/dn, which couples every layer to the layers above it, so the
                             step solves the fully linearised system while the block-tridiagonal
                             factorization stays its preconditioner.  A direct FP64 solve
                             (refine_max_iter = 0) ignores the coupling.  Not with the diffuse field
                             (XK_EINVAL at xk_set_workspace).  0 (default): rates lagged. */
} xk_config;

typedef struct {
    int accepted;         /* 1 accepted, 0 rejected */
    double dt_used, dt_next, max_rel;
    int n_neg;            /* entries clipped to zero on acceptance */
    int converged;        /* steady-state test passed on this step */
    int solver_iters;     /* FGMRES iterations (mixed) or 0 */
    double solver_resid;  /* final relative residual (mixed) or 0 */
    int used_fp64;        /* mixed mode: this step was solved by the FP64 factorization */
} xk_step_info;

typedef struct {
    int converged, steps, accepted, rejected;
    double t, dt, max_rel;
    long long solver_iters;   /* total FGMRES iterations */
    long long fp64_steps;     /* mixed mode: steps solved by the FP64 factorization */
    long long refactors;      /* mixed mode: FP64 factorizations computed (the others reused one) */
} xk_run_info;

/* Library version (major * 10000 + minor * 100 + patch). */
XK_API int xk_version(void);

/* Fill cfg with the default policy: FP64, dt_max 1e8 s, rel_reject 1.0,
 * rel_target 0.5, grow 3, shrink 0.5, neg_tol 1e-12, f_floor 1e-20,
 * dt_min 1e-20, ss_dt 1e8, ss_tol 1e-3, FGMRES(30), 40 iterations, tolerance
 * 1e-15, 10 refinement iterations around FP64 factorizations, the FP32
 * factorization by block cyclic reduction on the tensor cores. */
XK_API int xk_config_init(xk_config *cfg);

/* Create a context for one atmospheric column on cfg->device.  *out is set
 * to NULL on failure.  The context owns host-side copies of all inputs. */
XK_API int xk_create(xk_ctx **out, const xk_config *cfg);
XK_API int xk_destroy(xk_ctx *ctx);
XK_API const char *xk_last_error(const xk_ctx *ctx);

/* Chemical network (Sec. 2.2-2.3; Appendix A).  All host arrays.
 *  elem[S*E] element counts; mass[S] in u;
 *  rtype[R] XK_RX_*; reac[R*3], prod[R*3] species indices, -1 padded
 *    (a two-body or three-body reaction has >= 1 reactant and >= 1 product;
 *     a photolysis reaction exactly one reactant);
 *  arr[R*9] = alpha, beta, gamma (two-body) | alpha0, beta0, gamma0,
 *    alpha_inf, beta_inf, gamma_inf (three-body); k = alpha T_b^beta exp(-gamma/T);
 *  troe[R*4] = a, T***, T*, T** (a == 0: Lindemann without broadening);
 *  form[R] 0: Kooij (T_b = T/300), 1: modified Arrhenius (T_b = T);
 *  nasa[S*15] = T_mid, a1..a7 below T_mid, a1..a7 at and above T_mid.
 * XK_EINVAL on out-of-range indices or sizes. */
XK_API int xk_load_network(xk_ctx *ctx, int S, int E, int R, const int *elem, const double *mass,
                    const int *rtype, const int *reac, const int *prod, const double *arr,
                    const double *troe, const int *form, const double *nasa);

/* Photolysis inputs (Sec. 2.3.3), host arrays.  prow[R]: row of sigma for
 * each photolysis reaction (-1 otherwise); lambda[W], dlambda[W] (A);
 * J0[W] top-of-atmosphere photon flux (cm^-2 s^-1 A^-1); sigma[Rph*W]
 * dissociation cross sections; sigma_abs[S*W] absorption cross sections for
 * the optical depth; mu = cos(zenith); tf = irradiated time fraction.
 * Required (W may be 0) when the network has photolysis reactions. */
XK_API int xk_load_photo(xk_ctx *ctx, int W, int Rph, const int *prow, const double *lambda,
                  const double *dlambda, const double *J0, const double *sigma,
                  const double *sigma_abs, double mu, double tf);

/* Extinction by scattering and the diffuse field (Sec. 2.3.3), optional; after xk_load_photo and
 * before xk_set_workspace.  sigma_s [S*W] (host; NULL: no scattering): Rayleigh scattering cross
 * sections (cm^2) on the photolysis grid (W must equal its bin count), added to the absorption in
 * the optical depth tau = sum_i (sigma_a,i + sigma_s,i) n_i dz.  diffuse = 1 adds the diffuse field
 * J_diff = (J_up + J_down) / 2 to the direct beam J0 exp(-tau/mu).  The paper does not say how J_up
 * and J_down are found; here they come from a two-stream photon budget, layer by layer: the beam
 * photons a layer scatters (fraction dtau_s / dtau of those it removes) go half up, half down; a
 * diffuse flux crosses a layer with probability exp(-2 dtau) (the hemispheric mean path) and is
 * otherwise scattered (half back, half on) or absorbed; the lower boundary reflects the fraction
 * albedo (0..1) of the diffuse and direct light reaching it; nothing diffuse enters at the top.
 * J_up and J_down of a layer are the means of the fluxes through its two interfaces.  Photolysis
 * rates are evaluated at the start of a step; cfg.photo_jacobian adds the direct beam's derivative
 * (not the diffuse field's, which it refuses) to the step's FGMRES operator.
 * XK_EINVAL on a grid mismatch, a negative or non-finite cross section, albedo outside [0, 1]. */
XK_API int xk_load_scattering(xk_ctx *ctx, int W, const double *sigma_s, double albedo, int diffuse);

/* Atmosphere (Sec. 2.1, Fig. 3), host arrays of length L: pressure (bar),
 * temperature (K), Kzz (cm^2/s); dcoef[S]: molecular diffusion
 * D_y = dcoef_y T^0.75 / n_gas; g (cm/s^2); mbar (u); alpha_T thermal
 * diffusion factor.  Altitudes follow hydrostatic balance. */
XK_API int xk_load_atmosphere(xk_ctx *ctx, int L, const double *P_bar, const double *T, const double *Kzz,
                       const double *dcoef, double g, double mbar, double alpha_T);

/* Device workspace needed for the loaded network and atmosphere (bytes). */
XK_API int xk_workspace_bytes(xk_ctx *ctx, size_t *bytes);
/* Attach a device workspace of at least xk_workspace_bytes (256-byte
 * aligned) and upload the inputs.  Must follow the three loads. */
XK_API int xk_set_workspace(xk_ctx *ctx, void *device_ptr, size_t bytes);

/* State [L*S] number densities; on_device selects whether n is a device
 * (1) or host (0) pointer.  xk_set_mixing_ratios sets n = f * n_gas. */
XK_API int xk_set_state(xk_ctx *ctx, const double *n, int on_device);
XK_API int xk_set_mixing_ratios(xk_ctx *ctx, const double *f, int on_device);
XK_API int xk_get_state(xk_ctx *ctx, double *n, int on_device);

/* Gibbs energies, equilibrium constants and forward/reverse rate coefficients
 * of every thermal reaction in every layer (Sec. 2.3, Appendix A) for the
 * loaded atmosphere, kept in the workspace.  They depend on T and P only, so
 * steps evaluate them once (lazily if this is not called) until a network or
 * atmosphere is loaded again.  Synchronizes the stream. */
XK_API int xk_set_rate_coefficients(xk_ctx *ctx);

/* One controlled implicit step of size dt (dt <= 0: use the context's
 * current dt).  Evaluates photolysis, residual, Jacobian, factorization and
 * solve (rate coefficients once, see above), then accepts (n updated,
 * negatives clipped to 0) or rejects (n unchanged).  Synchronizes the stream
 * and fills *info. */
XK_API int xk_step(xk_ctx *ctx, double dt, xk_step_info *info);

/* Steps from dt0 (dt0 <= 0: keep the current dt) until the steady-state test
 * passes or max_steps attempts are made.  XK_ENOCONV if not converged. */
XK_API int xk_run_to_steady(xk_ctx *ctx, double dt0, int max_steps, xk_run_info *info);

/* ---- single rows of the step, on caller device buffers (for parity checks) ----
 * Each runs on the context's stream and synchronizes it before returning. */
/* grid: n_gas[L], z[L], dz[L], dzi[L-1] (device). */
XK_API int xk_eval_grid(xk_ctx *ctx, double *ngas, double *z, double *dz, double *dzi);
/* G/RT [L*S] and ln K_c [L*R] (device). */
XK_API int xk_eval_thermo(xk_ctx *ctx, double *grt, double *lnkc);
/* thermal k_f, k_r [L*R] (device; photolysis rows 0). */
XK_API int xk_eval_rates(xk_ctx *ctx, double *kf, double *kr);
/* photolysis rate constants kph [L*Rph] at state n (device). */
XK_API int xk_eval_photolysis(xk_ctx *ctx, const double *n, double *kph);
/* interface flux coefficients u, v [(L-1)*S] with phi = u n_k - v n_{k+1} (device). */
XK_API int xk_eval_transport(xk_ctx *ctx, double *u, double *v);
/* residual F(n) [L*S] (device). */
XK_API int xk_eval_residual(xk_ctx *ctx, const double *n, double *F);
/* I/dt - dF/dn: A [L*S*S], lo [L*S], up [L*S] (device). */
XK_API int xk_eval_jacobian(xk_ctx *ctx, const double *n, double dt, double *A, double *lo, double *up);
/* Solve the block-tridiagonal system given by A, lo, up (device, FP64) for
 * right-hand side f, writing x (device).  A is not modified.  Uses the FP64
 * factorization kernels and the context's workspace (either mode). */
XK_API int xk_block_solve(xk_ctx *ctx, const double *A, const double *lo, const double *up,
                   const double *f, double *x);
/* Approximate FP32 solve of a block-tridiagonal system (the mixed path's
 * preconditioner): A, lo, up (device, FP64, layout as for xk_block_solve) are
 * converted to FP32 and inverted by the FP32 kernels the context is
 * configured with (mixed contexts only).  The caller scales the system so
 * that FP32 can hold its entries (the mixed path uses diag(1/s) A diag(s)
 * with s = max(n, 1e-20 n_gas)).  The result carries FP32 rounding and no
 * refinement. */
XK_API int xk_block_solve32(xk_ctx *ctx, const double *A, const double *lo, const double *up,
                            const double *f, double *x);
/* delta solving (I/dt - J(n)) delta = F(n) with the context's precision
 * mode (device n, delta).  *iters / *resid report the FGMRES work (in mixed
 * mode *iters = -1 when the FP64 route solved the step; in FP64 mode the
 * refinement iterations around the FP64 factorization). */
XK_API int xk_step_delta(xk_ctx *ctx, const double *n, double dt, double *delta, int *iters, double *resid);

/* ---- chemical-equilibrium initial state (Sec. 2.5, option (i)) ----
 * For each layer, the ideal-gas mixture of minimum Gibbs energy
 *     G/RT = sum_y N_y (G_y/RT + ln(P/p0) + ln(N_y / N)),  N = sum_y N_y,
 * at the layer's T and P (G_y/RT from the NASA-7 sets, Appendix A), with fixed element totals
 * sum_y a_ey N_y = b_e (a = the network's element counts).  The paper starts runs from such a
 * composition computed by its equilibrium solver; every thermal reaction is then in balance,
 * sum nu ln n = ln K_c (Sec. 2.3.4).  Solved per layer on one CTA by Newton iterations on the
 * element potentials and the total moles; the mole fractions of species far below 1e-100 are exact
 * in relative terms, since they are rebuilt from the converged potentials.
 *  b [L*E]: element totals per layer (device; any common unit, e.g. atoms cm^-3), or NULL to take
 *    them from the context's current state; an element with b_e <= 0 is absent and every species
 *    holding it gets x = 0.
 *  x [L*S]: mole fractions, summing to 1 per layer (device; may be NULL).
 *  set_state: 1 also sets the context's state to n = x n_gas.
 *  max_iter, tol: Newton iterations per layer, and the bound on the N-weighted mean |d ln N_y| and
 *    on |d ln N| that ends them (1e-12 gives full FP64 accuracy in about 20-60 iterations).
 * Returns XK_OK, XK_ENOCONV (some layer did not converge: info says how many; x and the state hold
 * the last iterate), XK_ESINGULAR, XK_EINVAL (more than 30 elements, bad arguments).  Synchronizes. */
typedef struct {
    int iters_max;              /* most Newton iterations any layer took */
    int layers_not_converged;
    int layers_singular;
} xk_equilibrium_info;
XK_API int xk_equilibrium(xk_ctx *ctx, const double *b, double *x, int set_state, int max_iter, double tol,
                          xk_equilibrium_info *info);

/* ---- reaction-pathway analyser (Sec. 4) ----
 * The paper finds the kinetically fastest conversion route between two species with Dijkstra's
 * algorithm, minimising the summed inverse reaction rates, and names the slowest reaction of the
 * route its rate-limiting step.
 * xk_reaction_fluxes: forward and reverse rate of every reaction in every layer at state n
 *   (device [L*S]): q [L*R*2] (device), q[(k R + r) 2 + 0] = k_f prod n_reac (photolysis: k_ph n_A,
 *   with k_ph at state n), q[.. + 1] = k_r prod n_prod (0 for photolysis), molecules cm^-3 s^-1.
 * xk_pathways: the graph of layer k has an edge from every species a reaction direction consumes
 *   to every species it produces (itself excepted), of weight 1 / q for that direction's rate q > 0.
 *   Edge code = 2 r + direction (0 forward, 1 reverse).  For each source src[j] (host array,
 *   0 < nsrc <= S) and each layer, Dijkstra's search on one warp writes, at [(j L + k) S + y]
 *   (device arrays; any may be NULL, but lim_edge and lim_w go together):
 *     dist: least summed inverse rate from the source to y (s cm^3; +inf unreachable, 0 at the source);
 *     pred_sp, pred_edge: predecessor species and edge of y on that route (-1 none);
 *     lim_edge, lim_w: the route's slowest step (largest 1/q, the first on ties) and its weight.
 *   Ties are broken deterministically: the unfinished species of least distance with the lower
 *   index is finished next, and an edge replaces a predecessor only when it makes the distance
 *   strictly smaller, edges taken in increasing code; the same inputs give the same tree bit for
 *   bit.  Returns XK_OK or XK_EINVAL.  Synchronizes. */
XK_API int xk_reaction_fluxes(xk_ctx *ctx, const double *n, double *q);
XK_API int xk_pathways(xk_ctx *ctx, const double *q, int nsrc, const int *src, double *dist, int *pred_sp,
                       int *pred_edge, int *lim_edge, double *lim_w);

/* ---- variable-order BDF integrator (the DLSODES family of Sec. 2.1) ----
 * The paper integrates its stiff system with DLSODES, a variable-order, variable-step backward
 * differentiation method.  xk_bdf_run advances the context's state with BDF orders 1..qmax on the
 * same block-tridiagonal system as xk_step, linearly implicit (one Newton iteration per step):
 * order q asks that the polynomial through the new state at t + h and the last q accepted states
 * have the derivative F at t + h, c_0 y_new + sum_{j>=1} c_j y_j = F(y_new) with c_j the derivatives
 * of the Lagrange basis at t + h (variable steps), and linearises F about the predictor y_hat (the
 * polynomial through the last q + 1 states at t + h):
 *     (c_0 I - J(y_hat)) delta = F(y_hat) - c_0 y_hat - sum_{j>=1} c_j y_j,   y_new = y_hat + delta,
 * solved with the context's precision mode (order 1 from a constant predictor is the backward-Euler
 * step).  Local error (y_new - y_hat) / (q + 1), relative to y_new on species above f_floor mixing
 * ratio, in units of rtol; a step with error > 1, a non-finite state or a state below -neg_tol n_gas
 * is redone with h * max(0.2, min(0.9, 0.9 err^{-1/(q+1)})) (h / 4 for a bad state), and after two
 * rejections in a row the order drops by one.  Accepted states are clipped at zero.  After q + 1
 * steps at an order the next order is the one of q - 1, q, q + 1 whose estimate allows the largest
 * step (factors err^{-1/(order+1)} divided by 1.3, 1.2, 1.4); the step grows by at most `grow`
 * per step, never beyond dt_max or t_end.  Starts at order 1 with step h0 at t = 0 and stops at
 * t_end, or at steady state (an accepted step of h >= ss_dt with max relative change < ss_tol) when
 * stop_at_steady.  fixed_order > 0 pins the order (once the history allows it); fixed_step = 1 takes
 * every step h0 without error control.  The state is the last accepted one on return.
 * Returns XK_OK, XK_ENOCONV (max_steps attempts), XK_ENEG (step below dt_min, or a bad state at a
 * fixed step), XK_ESINGULAR, XK_ETIMEOUT, XK_EINVAL (rtol <= 0, qmax outside 1..5, grow < 1, h0,
 * t_end or max_steps not positive).  Synchronizes the stream after every step. */
typedef struct {
    double rtol;          /* local error target (relative) */
    int qmax;             /* largest order, 1..5 */
    int fixed_order;      /* > 0: no order selection */
    int fixed_step;       /* 1: constant step h0, no error control */
    double grow;          /* largest step growth per step (>= 1) */
} xk_bdf_config;
typedef struct {
    long long steps, accepted, rejected;
    int converged;
    long long order_steps[6];   /* accepted steps per order */
    double t, h, max_rel;       /* time reached, next step, last max relative change */
    int q;                      /* next order */
    long long solver_iters;     /* FGMRES iterations (mixed) or refinement iterations (FP64) */
} xk_bdf_info;
XK_API int xk_bdf_run(xk_ctx *ctx, const xk_bdf_config *cfg, double h0, double t_end, int stop_at_steady,
                      int max_steps, xk_bdf_info *info);

/* ---- Lagrangian parcel scheme (Sec. 2, Fig. 1 and Fig. 2) ----
 * The paper's own driver.  One global iteration carries an air parcel from the
 * bottom layer to the top and back (layers 0 .. L-1, then L-2 .. 0).  In layer
 * k the parcel spends the eddy mixing time tau_k = dz_k^2 / K_zz,k: eddy
 * diffusion is the parcel's motion.  There the parcel evolves under the layer's
 * chemistry (rate coefficients of Sec. 2.3, photolysis rates from the stored
 * profile at the start of the iteration).  Molecular diffusion is a
 * pseudo-reaction pair (Sec. 2.1, after Eq. 4: the molecular part of Eq. 2's
 * flux) with the stored densities of layers k -+ 1.
 * Time integration: linearly implicit Euler steps under the context's step
 * policy (dt_max, rel_reject, rel_target, grow_max, shrink_min, neg_tol, f_floor,
 * dt_min), each solved by Gaussian elimination with partial pivoting in FP64.
 * No step crosses the end of a visit, and the trial step is carried from
 * visit to visit.  The parcel keeps its mixing ratios from layer to layer;
 * each visit leaves its densities as the layer's.  The stored profile is the
 * context's state (xk_set_state / xk_get_state); every K_zz must be positive.
 *
 * xk_parcel_iteration: one global iteration.  info->h must hold the first
 *   trial step (> 0) and receives the next one.  steps / rejected count this
 *   iteration.  max_change is the largest |N_new - N_old| / N_new over entries
 *   above f_floor mixing ratio.  The whole iteration runs on one CTA, with no
 *   grid-wide waits.  Returns XK_ESINGULAR (zero pivot), XK_ENEG (a step below
 *   dt_min), XK_ENOCONV (more than max_visit_steps steps in one visit) or
 *   XK_OK; the profile is then partly swept.
 * xk_parcel_run: iterations until max_change < tol (Sec. 2: 0.1 %), or
 *   XK_ENOCONV after max_iter; steps and rejected count the whole run. */
typedef struct {
    double h;
    long long steps;
    long long rejected;
    double max_change;
} xk_parcel_info;
XK_API int xk_parcel_iteration(xk_ctx *ctx, int max_visit_steps, xk_parcel_info *info);
/* The same iteration in two halves, so that many columns' sweeps run at once (one CTA each, on
 * each context's own stream): begin enqueues it with first trial step h and returns;
 * end waits for it and fills *info (its return codes are those of xk_parcel_iteration). */
XK_API int xk_parcel_begin(xk_ctx *ctx, int max_visit_steps, double h);
XK_API int xk_parcel_end(xk_ctx *ctx, xk_parcel_info *info);
XK_API int xk_parcel_run(xk_ctx *ctx, int max_visit_steps, int max_iter, double tol, xk_parcel_info *info,
                         int *iterations);

/* ---- batches of columns: continuous batching on one GPU ----
 * A batch advances many columns together, each on its own stream, with the
 * persistent block-inversion kernels sized to a share of the SMs so that the
 * columns' work overlaps on the device.  Columns are admitted by their device
 * footprint (the workspace bytes of their contexts) against the batch's
 * budget, and can be admitted or removed between calls to xk_batch_step.
 *
 * xk_batch_create: budget_bytes = HBM the batch may hold in column
 *   workspaces; max_slots = most columns at once (also sets each column's
 *   share of the SMs: max(1, SMs / max_slots) CTAs per inversion kernel).
 * xk_batch_add: ctx must have its workspace and state set; its steps start
 *   from dt0 (> 0) with the context's step policy.  *slot receives the slot
 *   index.  XK_ENOMEM when the footprint does not fit the remaining budget
 *   or all slots are taken (nothing is changed then).  While in a batch the
 *   context issues its work on the batch's stream for that slot; calls on the
 *   context itself (xk_step, ...) must not be made until it is removed.
 * xk_batch_step: every admitted column that has not finished takes up to
 *   nsteps controlled steps; returns when all of them are done (the batch's
 *   streams are synchronized).  Finished columns take no further steps.
 * xk_batch_poll: run information of a slot and whether it has finished
 *   (converged, or stopped with an error recorded in *status).
 * xk_batch_remove: releases the slot and its budget; the context returns to
 *   its own stream and factorization plan.
 * xk_batch_last_error: message of the last failed batch call (the failing
 *   column's, for xk_batch_step); owned by the batch, valid until the next call.
 * xk_batch_submit / xk_batch_query: the asynchronous form, so that every column
 *   advances at its own pace: submit enqueues nsteps controlled steps for one
 *   slot on its stream and returns (XK_EINVAL if that slot's previous
 *   submission has not been queried done); query sets *done to 1 once they have
 *   run (then xk_batch_poll reads that slot's new state) and to 0 before,
 *   without blocking.  xk_batch_step refuses to run while a submission is in
 *   flight; xk_batch_remove waits for it. */
typedef struct xk_batch xk_batch;
XK_API int xk_batch_create(xk_batch **out, int device, size_t budget_bytes, int max_slots);
XK_API int xk_batch_destroy(xk_batch *batch);
XK_API int xk_batch_add(xk_batch *batch, xk_ctx *ctx, double dt0, int *slot);
XK_API int xk_batch_remove(xk_batch *batch, int slot);
XK_API int xk_batch_step(xk_batch *batch, int nsteps);
XK_API int xk_batch_poll(xk_batch *batch, int slot, xk_run_info *info, int *finished, int *status);
XK_API const char *xk_batch_last_error(xk_batch *batch);
XK_API int xk_batch_submit(xk_batch *batch, int slot, int nsteps);
/* Admission check before any allocation: *fits = 1 when a column whose
 * workspace needs `bytes` (xk_workspace_bytes) would be admitted now (a slot is
 * free and the bytes fit the remaining budget), 0 otherwise.  Host only. */
XK_API int xk_batch_fits(xk_batch *batch, size_t bytes, int *fits);
XK_API int xk_batch_query(xk_batch *batch, int slot, int *done);

/* ---- block solve without any device allocation ----
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc (code inside another framework's memory pool or allocator
 * hooks, hosts that forbid device allocations in plugins, work being set up
 * while other streams are captured).  It solves the same block-tridiagonal
 * system as xk_block_solve with the same FP64 kernels, without a context or
 * a workspace.  A [L*S*S], lo [L*S], up [L*S], f [L*S] and x [L*S] are
 * caller-owned device pointers of the current device (anything else, a host
 * pointer for instance, is refused with XK_EINVAL before any work is queued;
 * the caller answers for their extents); A is not modified;
 * stream is a cudaStream_t (NULL: legacy default stream).  The call
 * synchronizes the stream.
 * Scratch lives in one file-scope device array of XK_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that every GPU loading the library holds until the process exits;
 * the call needs about L*S*(8*round_up(S, 32) + 16) bytes of it and returns
 * XK_ENOMEM when that exceeds the array (e.g. S = 96 fits up to L = 445,
 * S = 594 up to L = 11).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and should come before any stream
 * capture on that device.  All calls share the array and it keeps the last
 * call's contents (the control flags and barrier words are cleared at the
 * start of each call), so calls that overlap on the GPU, from any thread or
 * stream, race and must be serialized by the caller.
 * A refused copy or clear of the scratch returns XK_ECUDA without launching
 * anything.  Returns XK_OK, XK_EINVAL, XK_ENOMEM, XK_ESINGULAR, XK_ETIMEOUT or
 * XK_ECUDA. */
#define XK_NOALLOC_SCRATCH_BYTES (32u << 20)
XK_API int xk_block_solve_noalloc(int L, int S, const double *A, const double *lo, const double *up,
                                  const double *f, double *x, void *stream);

/* ---- the tensor-core contraction, callable on its own ----
 * C = alpha A B + beta C for row-major FP32 device matrices A [M x lda],
 * B [K x ldb], C [M x ldc], computed on the 5th-generation tensor cores with
 * TF32 inputs split into head and tail (three products per step, at most
 * about 3 * 2^-22 of |a||b| per product) and FP32 accumulation; the product every dense
 * step of the mixed path's block factorization is made of.  M, N, K, lda, ldb
 * and ldc must be multiples of 32, A and B 256-byte aligned and C 16-byte
 * aligned (XK_EINVAL otherwise).  Runs on stream and synchronizes it; calls
 * are serialized (a single task slot in device memory). */
XK_API int xk_tc_gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                      float alpha, float beta, void *stream);

/* ---- tracing: CUDA events around each phase of every step ----
 * Phases: XK_PH_RATES (Gibbs energies + rate coefficients), XK_PH_PHOTO,
 * XK_PH_REACTION (w and its derivatives), XK_PH_RESIDUAL, XK_PH_JACOBIAN,
 * XK_PH_FACTOR (block inversions), XK_PH_SOLVE (block sweeps, or FGMRES with
 * its sweeps in mixed mode), XK_PH_CONTROL (accept/reject/update),
 * XK_PH_FALLBACK (mixed mode only: the FP64 Jacobian, factorization and
 * solve, whose kernels exit at once on steps that FGMRES solved), and within
 * the block cyclic reduction (fp32_bcr) XK_PH_TC and XK_PH_LEAF around every
 * launch of its tensor-core products and of its leaf inversions.
 * xk_profile(ctx, 1) starts recording (and clears totals); 0 stops.
 * xk_profile_read fills ms[n] with the summed device time of each phase and
 * calls[n] with the number of timed occurrences, synchronizing the stream.
 * Event pairs beyond 65536 per phase are not recorded (calls stops growing). */
#define XK_PH_RATES 0
#define XK_PH_PHOTO 1
#define XK_PH_REACTION 2
#define XK_PH_RESIDUAL 3
#define XK_PH_JACOBIAN 4
#define XK_PH_FACTOR 5
#define XK_PH_SOLVE 6
#define XK_PH_CONTROL 7
#define XK_PH_FALLBACK 8
#define XK_PH_TC 9        /* inside XK_PH_FACTOR with fp32_bcr: each launch of the tensor-core products */
#define XK_PH_LEAF 10     /* inside XK_PH_FACTOR with fp32_bcr: each launch of the leaf-block inversions */
#define XK_PH_COUNT 11
XK_API int xk_profile(xk_ctx *ctx, int enable);
XK_API int xk_profile_read(xk_ctx *ctx, double *ms, long long *calls, int n);
/* Work of the context's FP32 factorization (fp32_bcr): *mma_flops = 2 m n k summed over
 * every tensor-core product of one factorization (the tensor pipe executes three times
 * that: head x head, head x tail, tail x head); *leaf_flops = 2 n^3 summed over its leaf
 * inversions.  XK_EINVAL for contexts without the reduction. */
XK_API int xk_factor_work(xk_ctx *ctx, double *mma_flops, double *leaf_flops);
/* Testing aid for the bounded waits: makes the next grid barrier of the
 * context's FP64 factorization unreachable (its arrival count is raised past
 * any grid), as if a CTA never arrived.  The waiting CTAs give up after
 * cfg.wait_polls polls, the call that ran the factorization returns
 * XK_ETIMEOUT, and the library clears the barrier words, so that the next call
 * on the context runs normally.  Nothing faults: the kernels that follow a
 * timed-out factorization return at once. */
XK_API int xk_hold_next_barrier(xk_ctx *ctx);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * contexts of the process; kernels that exit at once because their solve or
 * step has finished are counted too). */
XK_API long long xk_launch_count(void);

/* Number of CUDA graph launches (captured chunks of steps, see cfg.use_graphs)
 * since the library was loaded; each replay also adds its kernel nodes to
 * xk_launch_count. */
XK_API long long xk_graph_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
