"""ctypes wrapper of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [
        ("S", C.c_int), ("E", C.c_int), ("R", C.c_int), ("L", C.c_int), ("W", C.c_int), ("Rph", C.c_int),
        ("elem", _ip), ("mass", _dp), ("rtype", _ip), ("reac", _ip), ("prod", _ip),
        ("arr", _dp), ("troe", _dp), ("form", _ip), ("nasa", _dp), ("prow", _ip),
        ("lam", _dp), ("dlam", _dp), ("J0", _dp), ("sigma", _dp), ("sigma_abs", _dp),
        ("mu", C.c_double), ("tf", C.c_double),
        ("P_bar", _dp), ("T", _dp), ("Kzz", _dp), ("dcoef", _dp),
        ("g", C.c_double), ("mbar", C.c_double), ("alpha_T", C.c_double),
        ("sigma_s", _dp), ("albedo", C.c_double), ("diffuse", C.c_int),
    ]


class Policy(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "dt_max", "rel_reject", "rel_target", "grow_max", "shrink_min",
        "neg_tol", "f_floor", "dt_min", "ss_dt", "ss_tol")]


class StepInfo(C.Structure):
    _fields_ = [("accepted", C.c_int), ("dt_used", C.c_double), ("dt_next", C.c_double),
                ("max_rel", C.c_double), ("n_neg", C.c_int)]


class RunInfo(C.Structure):
    _fields_ = [("converged", C.c_int), ("steps", C.c_int), ("accepted", C.c_int),
                ("rejected", C.c_int), ("t", C.c_double), ("dt", C.c_double), ("max_rel", C.c_double)]


class ParcelInfo(C.Structure):
    _fields_ = [("h", C.c_double), ("steps", C.c_int), ("rejected", C.c_int), ("max_change", C.c_double)]


class BdfConfig(C.Structure):
    _fields_ = [("rtol", C.c_double), ("qmax", C.c_int), ("fixed_order", C.c_int), ("fixed_step", C.c_int),
                ("grow", C.c_double)]


class BdfInfo(C.Structure):
    _fields_ = [("steps", C.c_int), ("accepted", C.c_int), ("rejected", C.c_int), ("converged", C.c_int),
                ("order_steps", C.c_int * 6), ("t", C.c_double), ("h", C.c_double), ("max_rel", C.c_double),
                ("q", C.c_int), ("err", C.c_double)]


def default_policy(**kw):
    """The step-control policy shared (by value, not by code) with the CUDA path."""
    vals = dict(dt_max=1e8, rel_reject=1.0, rel_target=0.5, grow_max=3.0, shrink_min=0.5,
                neg_tol=1e-12, f_floor=1e-20, dt_min=1e-20, ss_dt=1e8, ss_tol=1e-3)
    vals.update(kw)
    return Policy(**vals)


def build(force=False):
    """Compile oracle.c into a shared library (plain C, strict FP: no contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-std=c11", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        l = C.CDLL(_LIB_PATH)
        P = C.POINTER(_Problem)
        l.ora_grid.argtypes = [P, _dp, _dp, _dp, _dp]
        l.ora_gibbs_rt.argtypes = [_dp, C.c_double]; l.ora_gibbs_rt.restype = C.c_double
        l.ora_cp_r.argtypes = [_dp, C.c_double]; l.ora_cp_r.restype = C.c_double
        l.ora_thermo.argtypes = [P, _dp, _dp]
        l.ora_rate_coefficients.argtypes = [P, _dp, _dp]
        l.ora_photolysis.argtypes = [P, _dp, _dp]
        l.ora_transport.argtypes = [P, _dp, _dp]
        l.ora_residual.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
        l.ora_jacobian.argtypes = [P, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
        l.ora_block_solve.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
        l.ora_block_solve.restype = C.c_int
        l.ora_step_delta.argtypes = [P, _dp, C.c_double, _dp]; l.ora_step_delta.restype = C.c_int
        l.ora_block_solve_refined.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_int]
        l.ora_block_solve_refined.restype = C.c_int
        l.ora_step.argtypes = [P, C.POINTER(Policy), _dp, C.c_double, C.POINTER(StepInfo)]
        l.ora_run_to_steady.argtypes = [P, C.POINTER(Policy), _dp, C.c_double, C.c_int, C.POINTER(RunInfo)]
        l.ora_run_to_steady.restype = C.c_int
        l.ora_parcel_system.argtypes = [P, _dp, C.c_int, _dp, C.c_double, _dp, _dp]
        l.ora_parcel_system.restype = C.c_int
        l.ora_parcel_iteration.argtypes = [P, C.POINTER(Policy), C.c_int, _dp, C.POINTER(ParcelInfo)]
        l.ora_parcel_iteration.restype = C.c_int
        l.ora_parcel_run.argtypes = [P, C.POINTER(Policy), C.c_int, C.c_int, C.c_double, _dp,
                                     C.POINTER(ParcelInfo), _ip]
        l.ora_parcel_run.restype = C.c_int
        l.ora_photolysis_dn.argtypes = [P, _dp, _dp]
        l.ora_photolysis_dn.restype = None
        l.ora_step_delta_coupled.argtypes = [P, _dp, C.c_double, _dp]
        l.ora_step_delta_coupled.restype = C.c_int
        l.ora_bdf_coeffs.argtypes = [C.c_int, _dp, _dp]
        l.ora_bdf_coeffs.restype = None
        l.ora_bdf_extrap.argtypes = [C.c_int, _dp, C.c_double, _dp]
        l.ora_bdf_extrap.restype = None
        l.ora_bdf_run.argtypes = [P, C.POINTER(Policy), C.POINTER(BdfConfig), _dp, C.c_double, C.c_double, C.c_int,
                                  C.c_int, C.POINTER(BdfInfo)]
        l.ora_bdf_run.restype = C.c_int
        l.ora_two_stream.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        l.ora_two_stream.restype = C.c_int
        l.ora_equilibrium.argtypes = [P, _dp, _dp, C.c_int, C.c_double, _ip]
        l.ora_equilibrium.restype = C.c_int
        l.ora_fluxes.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
        l.ora_fluxes.restype = None
        l.ora_pathways.argtypes = [P, _dp, C.c_int, _dp, _ip, _ip, _ip, _dp]
        l.ora_pathways.restype = None
        _lib = l
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


class Oracle:
    """Holds contiguous copies of a synthetic Problem and calls the C oracle."""

    def __init__(self, prob):
        self.p = prob
        c = lambda a, t=np.float64: np.ascontiguousarray(a, dtype=t)
        self._keep = dict(
            elem=c(prob.elem, np.int32), mass=c(prob.mass), rtype=c(prob.rtype, np.int32),
            reac=c(prob.reac, np.int32), prod=c(prob.prod, np.int32), arr=c(prob.arr),
            troe=c(prob.troe), form=c(prob.form, np.int32), nasa=c(prob.nasa),
            prow=c(prob.prow, np.int32), lam=c(prob.lam), dlam=c(prob.dlam), J0=c(prob.J0),
            sigma=c(prob.sigma if prob.sigma.size else np.zeros(1)),
            sigma_abs=c(prob.sigma_abs if prob.sigma_abs.size else np.zeros(1)),
            P_bar=c(prob.P_bar), T=c(prob.T), Kzz=c(prob.Kzz), dcoef=c(prob.dcoef))
        sig_s = getattr(prob, "sigma_s", None)
        if sig_s is not None:
            self._keep["sigma_s"] = c(sig_s)
        k = self._keep
        for key in ("lam", "dlam", "J0"):
            if k[key].size == 0:
                k[key] = np.zeros(1)
        self.st = _Problem(
            S=prob.S, E=prob.E, R=prob.R, L=prob.L, W=prob.W, Rph=prob.Rph,
            elem=_i(k["elem"]), mass=_d(k["mass"]), rtype=_i(k["rtype"]), reac=_i(k["reac"]),
            prod=_i(k["prod"]), arr=_d(k["arr"]), troe=_d(k["troe"]), form=_i(k["form"]),
            nasa=_d(k["nasa"]), prow=_i(k["prow"]), lam=_d(k["lam"]), dlam=_d(k["dlam"]),
            J0=_d(k["J0"]), sigma=_d(k["sigma"]), sigma_abs=_d(k["sigma_abs"]),
            mu=float(prob.mu), tf=float(prob.tf), P_bar=_d(k["P_bar"]), T=_d(k["T"]),
            Kzz=_d(k["Kzz"]), dcoef=_d(k["dcoef"]), g=float(prob.g), mbar=float(prob.mbar),
            alpha_T=float(prob.alpha_T),
            sigma_s=_d(k["sigma_s"]) if "sigma_s" in k else None,
            albedo=float(getattr(prob, "albedo", 0.0)), diffuse=int(getattr(prob, "diffuse", 0)))
        self.L, self.S, self.R = prob.L, prob.S, prob.R

    # -- rows of the step --------------------------------------------------
    def grid(self):
        L = self.L
        ngas, z, dz, dzi = (np.zeros(L) for _ in range(4))
        lib().ora_grid(C.byref(self.st), _d(ngas), _d(z), _d(dz), _d(dzi))
        return ngas, z, dz, dzi[: max(L - 1, 0)]

    def initial_state(self):
        ngas = self.grid()[0]
        return np.ascontiguousarray(self.p.f0 * ngas[:, None])

    def thermo(self):
        grt = np.zeros((self.L, self.S)); lnkc = np.zeros((self.L, self.R))
        lib().ora_thermo(C.byref(self.st), _d(grt), _d(lnkc))
        return grt, lnkc

    def rate_coefficients(self):
        kf = np.zeros((self.L, self.R)); kr = np.zeros((self.L, self.R))
        lib().ora_rate_coefficients(C.byref(self.st), _d(kf), _d(kr))
        return kf, kr

    def photolysis(self, n):
        kph = np.zeros((self.L, max(self.p.Rph, 1)))
        lib().ora_photolysis(C.byref(self.st), _d(np.ascontiguousarray(n, np.float64)), _d(kph))
        return kph[:, : self.p.Rph]

    def transport(self):
        m = max(self.L - 1, 1)
        u = np.zeros((m, self.S)); v = np.zeros((m, self.S))
        lib().ora_transport(C.byref(self.st), _d(u), _d(v))
        return u[: self.L - 1], v[: self.L - 1]

    def residual(self, n, kf=None, kr=None, kph=None):
        n = np.ascontiguousarray(n, np.float64)
        if kf is None:
            kf, kr = self.rate_coefficients()
        if kph is None:
            kph = self.photolysis(n)
        kph = np.ascontiguousarray(kph if kph.size else np.zeros((self.L, 1)))
        F = np.zeros((self.L, self.S))
        lib().ora_residual(C.byref(self.st), _d(kf), _d(kr), _d(kph), _d(n), _d(F))
        return F

    def jacobian(self, n, dt, kf=None, kr=None, kph=None):
        n = np.ascontiguousarray(n, np.float64)
        if kf is None:
            kf, kr = self.rate_coefficients()
        if kph is None:
            kph = self.photolysis(n)
        kph = np.ascontiguousarray(kph if kph.size else np.zeros((self.L, 1)))
        A = np.zeros((self.L, self.S, self.S)); lo = np.zeros((self.L, self.S)); up = np.zeros((self.L, self.S))
        lib().ora_jacobian(C.byref(self.st), _d(kf), _d(kr), _d(kph), _d(n), float(dt), _d(A), _d(lo), _d(up))
        return A, lo, up

    def block_solve(self, A, lo, up, f):
        A = np.array(A, np.float64, order="C", copy=True)
        x = np.zeros((self.L, self.S))
        rc = lib().ora_block_solve(self.L, self.S, _d(A), _d(np.ascontiguousarray(lo)),
                                   _d(np.ascontiguousarray(up)), _d(np.ascontiguousarray(f)), _d(x))
        if rc != 0:
            raise ZeroDivisionError("singular block")
        return x

    def block_solve_refined(self, A, lo, up, f, sweeps=4):
        x = np.zeros((self.L, self.S))
        rc = lib().ora_block_solve_refined(self.L, self.S, _d(np.ascontiguousarray(A, np.float64)),
                                           _d(np.ascontiguousarray(lo)), _d(np.ascontiguousarray(up)),
                                           _d(np.ascontiguousarray(f)), _d(x), int(sweeps))
        if rc != 0:
            raise ZeroDivisionError("singular block")
        return x

    def step_delta(self, n, dt):
        d = np.zeros((self.L, self.S))
        rc = lib().ora_step_delta(C.byref(self.st), _d(np.ascontiguousarray(n, np.float64)), float(dt), _d(d))
        if rc != 0:
            raise ZeroDivisionError("singular block")
        return d

    def step(self, n, dt, policy=None):
        """Controlled step; returns (new n, StepInfo).  The input array is not modified."""
        pol = policy or default_policy()
        m = np.array(n, np.float64, order="C", copy=True)
        info = StepInfo()
        lib().ora_step(C.byref(self.st), C.byref(pol), _d(m), float(dt), C.byref(info))
        return m, info

    def run_to_steady(self, n, dt0=1e-8, max_steps=5000, policy=None):
        pol = policy or default_policy()
        m = np.array(n, np.float64, order="C", copy=True)
        info = RunInfo()
        lib().ora_run_to_steady(C.byref(self.st), C.byref(pol), _d(m), float(dt0), int(max_steps), C.byref(info))
        return m, info

    # -- Lagrangian parcel scheme (Sec. 2, Fig. 2) ------------------------------
    def parcel_system(self, N, k, pk, h):
        """F and A = I/h - dF/dpk of the parcel with densities pk visiting layer k."""
        F = np.zeros(self.S)
        A = np.zeros((self.S, self.S))
        rc = lib().ora_parcel_system(C.byref(self.st), _d(np.ascontiguousarray(N, np.float64)), int(k),
                                     _d(np.ascontiguousarray(pk, np.float64)), float(h), _d(F), _d(A))
        if rc != 0:
            raise ValueError("bad layer or step")
        return F, A

    def parcel_iteration(self, N, h=1e-8, policy=None, max_visit_steps=100000):
        """One global iteration; returns (new profile, ParcelInfo).  N is not modified."""
        pol = policy or default_policy()
        m = np.array(N, np.float64, order="C", copy=True)
        info = ParcelInfo(h=float(h))
        rc = lib().ora_parcel_iteration(C.byref(self.st), C.byref(pol), int(max_visit_steps), _d(m), C.byref(info))
        if rc != 0:
            raise ArithmeticError(f"parcel iteration failed ({rc})")
        return m, info

    def parcel_run(self, N, h=1e-8, policy=None, max_iter=200, tol=1e-3, max_visit_steps=100000):
        """Global iterations to convergence; returns (profile, iterations, ParcelInfo, converged)."""
        pol = policy or default_policy()
        m = np.array(N, np.float64, order="C", copy=True)
        info = ParcelInfo(h=float(h))
        it = C.c_int(0)
        rc = lib().ora_parcel_run(C.byref(self.st), C.byref(pol), int(max_visit_steps), int(max_iter), float(tol),
                                  _d(m), C.byref(info), C.byref(it))
        if rc < 0:
            raise ArithmeticError(f"parcel run failed ({rc})")
        return m, it.value, info, rc == 0

    # -- equilibrium initial state (Sec. 2.5) and pathway analysis (Sec. 4) ---------
    def element_totals(self, n):
        """Element totals b [L][E] = sum_y a_ey n_y of a state (a plain contraction)."""
        return np.ascontiguousarray(np.asarray(n, np.float64) @ self.p.elem.astype(np.float64))

    def equilibrium(self, b, max_iter=300, tol=1e-12):
        """Mole fractions [L][S] of the Gibbs minimum for element totals b [L][E]; returns
        (x, iterations, converged)."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros((self.L, self.S))
        it = C.c_int(0)
        rc = lib().ora_equilibrium(C.byref(self.st), _d(b), _d(x), int(max_iter), float(tol), C.byref(it))
        if rc < 0:
            raise ArithmeticError("equilibrium: singular system")
        return x, it.value, rc == 0

    def fluxes(self, n, kf=None, kr=None, kph=None):
        """Forward and reverse rate of every reaction: q [L][R][2]."""
        if kf is None:
            kf, kr = self.rate_coefficients()
        if kph is None:
            kph = self.photolysis(n)
        q = np.zeros((self.L, self.R, 2))
        lib().ora_fluxes(C.byref(self.st), _d(np.ascontiguousarray(kf)), _d(np.ascontiguousarray(kr)),
                         _d(np.ascontiguousarray(kph if np.size(kph) else np.zeros(1))),
                         _d(np.ascontiguousarray(n, np.float64)), _d(q))
        return q

    def pathways(self, q_layer, src):
        """Dijkstra from src on one layer's rates q_layer [R][2]; returns dict of dist, pred_sp,
        pred_edge, lim_edge, lim_w."""
        S = self.S
        dist = np.zeros(S); lim_w = np.zeros(S)
        pred_sp = np.zeros(S, np.int32); pred_edge = np.zeros(S, np.int32); lim_edge = np.zeros(S, np.int32)
        lib().ora_pathways(C.byref(self.st), _d(np.ascontiguousarray(q_layer, np.float64)), int(src), _d(dist),
                           _i(pred_sp), _i(pred_edge), _i(lim_edge), _d(lim_w))
        return dict(dist=dist, pred_sp=pred_sp, pred_edge=pred_edge, lim_edge=lim_edge, lim_w=lim_w)

    # -- photolysis rates in the Jacobian (Sec. 2.3.3) ----------------------------------
    def photolysis_dn(self, n):
        """d k_ph / d n of the direct beam: [L*Rph, L*S]."""
        Rph = max(self.p.Rph, 1)
        dk = np.zeros((self.L * Rph, self.L * self.S))
        lib().ora_photolysis_dn(C.byref(self.st), _d(np.ascontiguousarray(n, np.float64)), _d(dk))
        return dk[: self.L * self.p.Rph]

    def step_delta_coupled(self, n, dt):
        """The step with dk_ph/dn in the Jacobian (dense solve; small columns)."""
        d = np.zeros((self.L, self.S))
        rc = lib().ora_step_delta_coupled(C.byref(self.st), _d(np.ascontiguousarray(n, np.float64)), float(dt), _d(d))
        if rc != 0:
            raise ArithmeticError("singular coupled system")
        return d

    # -- variable-order BDF (the DLSODES family, Sec. 2.1) -----------------------------
    def bdf_run(self, n, h0=1e-8, t_end=1e30, stop_at_steady=False, max_steps=1000, rtol=1e-3, qmax=5,
                fixed_order=0, fixed_step=0, grow=5.0, policy=None):
        """Integrates from n (not modified); returns (state, BdfInfo, return code)."""
        pol = policy or default_policy()
        m = np.array(n, np.float64, order="C", copy=True)
        cfg = BdfConfig(rtol=float(rtol), qmax=int(qmax), fixed_order=int(fixed_order), fixed_step=int(fixed_step),
                        grow=float(grow))
        info = BdfInfo()
        rc = lib().ora_bdf_run(C.byref(self.st), C.byref(pol), C.byref(cfg), _d(m), float(h0), float(t_end),
                               int(bool(stop_at_steady)), int(max_steps), C.byref(info))
        return m, info, rc


def bdf_coeffs(tau):
    """Derivative weights c_j at tau[0] of the Lagrange basis on the nodes tau (q = len(tau) - 1)."""
    t = np.ascontiguousarray(tau, np.float64)
    c = np.zeros(len(t))
    lib().ora_bdf_coeffs(len(t) - 1, _d(t), _d(c))
    return c


def bdf_extrap(tau, t):
    """Weights of the interpolant through the nodes tau evaluated at t."""
    tt = np.ascontiguousarray(tau, np.float64)
    w = np.zeros(len(tt))
    lib().ora_bdf_extrap(len(tt), _d(tt), float(t), _d(w))
    return w


def two_stream(dtau_a, dtau_s, F0, mu, albedo):
    """Diffuse field of one wavelength (Sec. 2.3.3): returns (U [L+1], D [L+1], Jdiff [L])."""
    ta = np.ascontiguousarray(dtau_a, np.float64)
    ts = np.ascontiguousarray(dtau_s, np.float64)
    L = ta.shape[0]
    U = np.zeros(L + 1); D = np.zeros(L + 1); Jd = np.zeros(L)
    rc = lib().ora_two_stream(int(L), _d(ta), _d(ts), float(F0), float(mu), float(albedo), _d(U), _d(D), _d(Jd))
    if rc != 0:
        raise ArithmeticError("two-stream system singular")
    return U, D, Jd
