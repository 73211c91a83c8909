"""Thin Python binding of libxk (ctypes).  Argument marshalling only: every
row of the implicit step runs in the library's CUDA kernels.  PyTorch supplies
device memory (the workspace and the caller's buffers) and the stream.

The functions keep the C names without the ``xk_`` prefix where they are
methods of :class:`Column`; the raw C functions are reachable through
:func:`lib`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p

XK_OK = 0
ERRORS = {-1: "XK_EINVAL", -2: "XK_ENOMEM", -3: "XK_ENOCONV", -4: "XK_ENEG", -5: "XK_ECUDA",
          -6: "XK_ESINGULAR", -7: "XK_ETIMEOUT"}
PREC = {"fp64": 0, "mixed": 1}


class Config(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("device", C.c_int), ("stream", C.c_void_p),
        ("dt_max", C.c_double), ("rel_reject", C.c_double), ("rel_target", C.c_double),
        ("grow_max", C.c_double), ("shrink_min", C.c_double), ("neg_tol", C.c_double),
        ("f_floor", C.c_double), ("dt_min", C.c_double), ("ss_dt", C.c_double), ("ss_tol", C.c_double),
        ("gmres_restart", C.c_int), ("gmres_max_iter", C.c_int), ("gmres_tol", C.c_double),
        ("panel_width", C.c_int), ("factor_ctas", C.c_int), ("fp32_pivoting", C.c_int),
        ("reuse_factorization", C.c_int), ("cluster_size", C.c_int), ("reuse_max_iters", C.c_int),
        ("twisted", C.c_int),
        ("fp64_panel", C.c_int), ("refine_max_iter", C.c_int), ("fp32_bcr", C.c_int),
        ("wait_polls", C.c_longlong), ("use_graphs", C.c_int), ("photo_jacobian", C.c_int),
    ]


class StepInfo(C.Structure):
    _fields_ = [("accepted", C.c_int), ("dt_used", C.c_double), ("dt_next", C.c_double),
                ("max_rel", C.c_double), ("n_neg", C.c_int), ("converged", C.c_int),
                ("solver_iters", C.c_int), ("solver_resid", C.c_double), ("used_fp64", C.c_int)]


class ParcelInfo(C.Structure):
    _fields_ = [("h", C.c_double), ("steps", C.c_longlong), ("rejected", C.c_longlong), ("max_change", C.c_double)]


class RunInfo(C.Structure):
    _fields_ = [("converged", C.c_int), ("steps", C.c_int), ("accepted", C.c_int), ("rejected", C.c_int),
                ("t", C.c_double), ("dt", C.c_double), ("max_rel", C.c_double), ("solver_iters", C.c_longlong),
                ("fp64_steps", C.c_longlong), ("refactors", C.c_longlong)]


class EquilibriumInfo(C.Structure):
    _fields_ = [("iters_max", C.c_int), ("layers_not_converged", C.c_int), ("layers_singular", C.c_int)]


class BdfConfig(C.Structure):
    _fields_ = [("rtol", C.c_double), ("qmax", C.c_int), ("fixed_order", C.c_int), ("fixed_step", C.c_int),
                ("grow", C.c_double)]


class BdfInfo(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("accepted", C.c_longlong), ("rejected", C.c_longlong),
                ("converged", C.c_int), ("order_steps", C.c_longlong * 6), ("t", C.c_double), ("h", C.c_double),
                ("max_rel", C.c_double), ("q", C.c_int), ("solver_iters", C.c_longlong)]


class XkError(RuntimeError):
    def __init__(self, where, code, msg):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


# name -> (restype, argtypes); mirrors include/xk.h
SIGNATURES = {
    "xk_version": (C.c_int, []),
    "xk_config_init": (C.c_int, [C.POINTER(Config)]),
    "xk_create": (C.c_int, [C.POINTER(_vp), C.POINTER(Config)]),
    "xk_destroy": (C.c_int, [_vp]),
    "xk_last_error": (C.c_char_p, [_vp]),
    "xk_load_network": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _ip, _dp, _ip, _ip, _ip, _dp, _dp, _ip, _dp]),
    "xk_load_photo": (C.c_int, [_vp, C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double]),
    "xk_load_scattering": (C.c_int, [_vp, C.c_int, _dp, C.c_double, C.c_int]),
    "xk_load_atmosphere": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double]),
    "xk_workspace_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "xk_set_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "xk_set_state": (C.c_int, [_vp, _vp, C.c_int]),
    "xk_set_mixing_ratios": (C.c_int, [_vp, _vp, C.c_int]),
    "xk_get_state": (C.c_int, [_vp, _vp, C.c_int]),
    "xk_set_rate_coefficients": (C.c_int, [_vp]),
    "xk_step": (C.c_int, [_vp, C.c_double, C.POINTER(StepInfo)]),
    "xk_run_to_steady": (C.c_int, [_vp, C.c_double, C.c_int, C.POINTER(RunInfo)]),
    "xk_parcel_iteration": (C.c_int, [_vp, C.c_int, C.POINTER(ParcelInfo)]),
    "xk_parcel_begin": (C.c_int, [_vp, C.c_int, C.c_double]),
    "xk_parcel_end": (C.c_int, [_vp, C.POINTER(ParcelInfo)]),
    "xk_parcel_run": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.POINTER(ParcelInfo), C.POINTER(C.c_int)]),
    "xk_eval_grid": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "xk_eval_thermo": (C.c_int, [_vp, _vp, _vp]),
    "xk_eval_rates": (C.c_int, [_vp, _vp, _vp]),
    "xk_eval_photolysis": (C.c_int, [_vp, _vp, _vp]),
    "xk_eval_transport": (C.c_int, [_vp, _vp, _vp]),
    "xk_eval_residual": (C.c_int, [_vp, _vp, _vp]),
    "xk_eval_jacobian": (C.c_int, [_vp, _vp, C.c_double, _vp, _vp, _vp]),
    "xk_block_solve": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "xk_block_solve32": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "xk_step_delta": (C.c_int, [_vp, _vp, C.c_double, _vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "xk_block_solve_noalloc": (C.c_int, [C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
    "xk_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_size_t, C.c_int]),
    "xk_batch_destroy": (C.c_int, [_vp]),
    "xk_batch_add": (C.c_int, [_vp, _vp, C.c_double, C.POINTER(C.c_int)]),
    "xk_batch_remove": (C.c_int, [_vp, C.c_int]),
    "xk_batch_step": (C.c_int, [_vp, C.c_int]),
    "xk_batch_poll": (C.c_int, [_vp, C.c_int, C.POINTER(RunInfo), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "xk_batch_last_error": (C.c_char_p, [_vp]),
    "xk_batch_submit": (C.c_int, [_vp, C.c_int, C.c_int]),
    "xk_batch_query": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "xk_batch_fits": (C.c_int, [_vp, C.c_size_t, C.POINTER(C.c_int)]),
    "xk_profile": (C.c_int, [_vp, C.c_int]),
    "xk_launch_count": (C.c_longlong, []),
    "xk_graph_launch_count": (C.c_longlong, []),
    "xk_hold_next_barrier": (C.c_int, [_vp]),
    "xk_tc_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, C.c_int, _vp, C.c_int, _vp, C.c_int, C.c_float, C.c_float,
                             _vp]),
    "xk_profile_read": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong), C.c_int]),
    "xk_factor_work": (C.c_int, [_vp, _dp, _dp]),
    "xk_equilibrium": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_double, C.POINTER(EquilibriumInfo)]),
    "xk_reaction_fluxes": (C.c_int, [_vp, _vp, _vp]),
    "xk_bdf_run": (C.c_int, [_vp, C.POINTER(BdfConfig), C.c_double, C.c_double, C.c_int, C.c_int,
                             C.POINTER(BdfInfo)]),
    "xk_pathways": (C.c_int, [_vp, _vp, C.c_int, _ip, _vp, _vp, _vp, _vp, _vp]),
}

PHASES = ["rates", "photolysis", "reaction", "residual", "jacobian", "factor", "solve", "control", "fallback",
          "tc", "leaf"]


def lib(build_if_missing=False):
    """Load libxk.so; raises if it is not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libxk is not built ({path}); run paper_2512_06729_gb300.build.build()")
        l = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def default_config(**kw):
    cfg = Config()
    lib().xk_config_init(C.byref(cfg))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        setattr(cfg, k, v)
    return cfg


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def tc_gemm(A, B, C=None, alpha=1.0, beta=0.0):
    """C = alpha A B + beta C on the tensor cores (FP32 torch tensors on the device, sizes multiples of 32)."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    stream = torch.cuda.current_stream(A.device).cuda_stream
    rc = lib().xk_tc_gemm(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(),
                          B.stride(0), C.data_ptr(), C.stride(0), float(alpha), float(beta), stream)
    if rc != XK_OK:
        raise XkError("xk_tc_gemm", rc, "bad sizes, alignment or a CUDA error")
    return C


class Column:
    """One atmospheric column on one GPU: owns an xk context and its workspace."""

    def __init__(self, prob, precision="fp64", device=0, stream=None, allocate=True, **cfg_kw):
        """With allocate=False only the context and its inputs are set up (workspace_bytes is then the
        device footprint); allocate() creates the workspace."""
        import torch
        self._torch = torch
        self.prob = prob
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.cfg = default_config(precision=precision, device=device, stream=stream.cuda_stream, **cfg_kw)
        self.precision = precision
        l = lib()
        h = _vp()
        rc = l.xk_create(C.byref(h), C.byref(self.cfg))
        if rc != XK_OK:
            raise XkError("xk_create", rc, "could not create context")
        self.h = h
        self.S, self.L, self.R = prob.S, prob.L, prob.R
        self._keep = []
        p = prob
        d = lambda a: self._keep_arr(_np(a, np.float64)).ctypes.data_as(_dp)
        i = lambda a: self._keep_arr(_np(a, np.int32)).ctypes.data_as(_ip)
        self._call("xk_load_network", p.S, p.E, p.R, i(p.elem), d(p.mass), i(p.rtype), i(p.reac), i(p.prod),
                   d(p.arr), d(p.troe), i(p.form), d(p.nasa))
        W, Rph = p.W, p.Rph
        if Rph > 0 or W > 0:
            one = np.zeros(1)
            self._call("xk_load_photo", W, Rph, i(p.prow), d(p.lam if W else one), d(p.dlam if W else one),
                       d(p.J0 if W else one), d(p.sigma if p.sigma.size else one),
                       d(p.sigma_abs if p.sigma_abs.size else one), float(p.mu), float(p.tf))
            sig_s = getattr(p, "sigma_s", None)
            if W > 0 and (sig_s is not None or getattr(p, "diffuse", 0)):
                self._call("xk_load_scattering", W, d(sig_s) if sig_s is not None else None,
                           float(getattr(p, "albedo", 0.0)), int(getattr(p, "diffuse", 0)))
        self._call("xk_load_atmosphere", p.L, d(p.P_bar), d(p.T), d(p.Kzz), d(p.dcoef), float(p.g),
                   float(p.mbar), float(p.alpha_T))
        nbytes = C.c_size_t()
        self._call("xk_workspace_bytes", C.byref(nbytes))
        self.workspace_bytes = int(nbytes.value)
        self.ws = None
        if allocate:
            self.allocate()

    def allocate(self):
        """Create the device workspace (workspace_bytes) and upload the inputs."""
        if self.ws is not None:
            return
        self.ws = self._torch.empty(self.workspace_bytes + 256, dtype=self._torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        self._call("xk_set_workspace", _vp(aligned), C.c_size_t(self.workspace_bytes))
        self._keep = []

    def _keep_arr(self, a):
        self._keep.append(a)
        return a

    def _call(self, name, *args):
        rc = getattr(lib(), name)(self.h, *args)
        if rc != XK_OK:
            msg = lib().xk_last_error(self.h)
            raise XkError(name, rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().xk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -----------------------------------------------------------
    def _dev(self, *shape):
        return self._torch.empty(*shape, dtype=self._torch.float64, device=self.device)

    def _ptr(self, t):
        assert t.is_cuda and t.is_contiguous() and t.dtype == self._torch.float64
        return _vp(t.data_ptr())

    # -- state ---------------------------------------------------------------
    def set_mixing_ratios(self, f):
        t = self._torch.as_tensor(_np(f, np.float64), device=self.device).contiguous()
        self._call("xk_set_mixing_ratios", self._ptr(t), 1)

    def set_state(self, n):
        """n: numpy array or torch tensor (host, e.g. pinned, or on this device), [L, S] FP64."""
        if isinstance(n, np.ndarray):
            a = _np(n, np.float64)
            self._call("xk_set_state", _vp(a.ctypes.data), 0)
        else:
            t = n.contiguous()
            if t.dtype != self._torch.float64 or t.numel() != self.L * self.S:
                raise ValueError("state must be FP64 with L x S entries")
            self._call("xk_set_state", _vp(t.data_ptr()), 0 if t.device.type == "cpu" else 1)

    def get_state(self, device=False, out=None):
        """The state [L, S]: a new numpy array, a new device tensor (device=True), or into `out`
        (a contiguous FP64 torch tensor on the host, e.g. pinned, or on this device)."""
        if out is not None:
            if out.dtype != self._torch.float64 or out.numel() != self.L * self.S or not out.is_contiguous():
                raise ValueError("out must be a contiguous FP64 tensor with L x S entries")
            self._call("xk_get_state", _vp(out.data_ptr()), 0 if out.device.type == "cpu" else 1)
            return out
        if device:
            out = self._dev(self.L, self.S)
            self._call("xk_get_state", self._ptr(out), 1)
            return out
        out = np.zeros((self.L, self.S))
        self._call("xk_get_state", _vp(out.ctypes.data), 0)
        return out

    def step(self, dt=0.0):
        info = StepInfo()
        self._call("xk_step", float(dt), C.byref(info))
        return info

    def set_rate_coefficients(self):
        self._call("xk_set_rate_coefficients")

    def run_to_steady(self, dt0=1e-8, max_steps=5000, raise_on_noconv=False):
        info = RunInfo()
        rc = lib().xk_run_to_steady(self.h, float(dt0), int(max_steps), C.byref(info))
        if rc != XK_OK and (raise_on_noconv or rc != -3):
            msg = lib().xk_last_error(self.h)
            raise XkError("xk_run_to_steady", rc, msg.decode() if msg else "")
        return info

    # -- Lagrangian parcel scheme (Sec. 2, Fig. 2) ---------------------------
    def parcel_iteration(self, h=1e-8, max_visit_steps=100000):
        """One global iteration on the context's state; returns ParcelInfo (h = the next trial step)."""
        info = ParcelInfo(h=float(h))
        self._call("xk_parcel_iteration", int(max_visit_steps), C.byref(info))
        return info

    def parcel_begin(self, h=1e-8, max_visit_steps=100000):
        """Enqueue one global iteration on this column's stream and return at once."""
        self._call("xk_parcel_begin", int(max_visit_steps), float(h))

    def parcel_end(self):
        """Wait for the iteration begun last; returns its ParcelInfo."""
        info = ParcelInfo()
        self._call("xk_parcel_end", C.byref(info))
        return info

    def parcel_run(self, h=1e-8, max_iter=200, tol=1e-3, max_visit_steps=100000):
        """Global iterations until the change is below tol; returns (iterations, ParcelInfo, converged)."""
        info = ParcelInfo(h=float(h))
        it = C.c_int(0)
        rc = lib().xk_parcel_run(self.h, int(max_visit_steps), int(max_iter), float(tol), C.byref(info), C.byref(it))
        if rc not in (XK_OK, -3):
            msg = lib().xk_last_error(self.h)
            raise XkError("xk_parcel_run", rc, msg.decode() if msg else "")
        return int(it.value), info, rc == XK_OK

    # -- rows ----------------------------------------------------------------
    def eval_grid(self):
        L = self.L
        ng, z, dz, dzi = self._dev(L), self._dev(L), self._dev(L), self._dev(max(L - 1, 1))
        self._call("xk_eval_grid", self._ptr(ng), self._ptr(z), self._ptr(dz), self._ptr(dzi))
        return ng, z, dz, dzi[: L - 1]

    def eval_thermo(self):
        grt, lnkc = self._dev(self.L, self.S), self._dev(self.L, self.R)
        self._call("xk_eval_thermo", self._ptr(grt), self._ptr(lnkc))
        return grt, lnkc

    def eval_rates(self):
        kf, kr = self._dev(self.L, self.R), self._dev(self.L, self.R)
        self._call("xk_eval_rates", self._ptr(kf), self._ptr(kr))
        return kf, kr

    def eval_photolysis(self, n):
        kph = self._dev(self.L, max(self.prob.Rph, 1))
        self._call("xk_eval_photolysis", self._ptr(n.contiguous()), self._ptr(kph))
        return kph[:, : self.prob.Rph]

    def eval_transport(self):
        m = max(self.L - 1, 1)
        u, v = self._dev(m, self.S), self._dev(m, self.S)
        self._call("xk_eval_transport", self._ptr(u), self._ptr(v))
        return u[: self.L - 1], v[: self.L - 1]

    def eval_residual(self, n):
        F = self._dev(self.L, self.S)
        self._call("xk_eval_residual", self._ptr(n.contiguous()), self._ptr(F))
        return F

    def eval_jacobian(self, n, dt):
        A = self._dev(self.L, self.S, self.S)
        lo, up = self._dev(self.L, self.S), self._dev(self.L, self.S)
        self._call("xk_eval_jacobian", self._ptr(n.contiguous()), float(dt), self._ptr(A), self._ptr(lo), self._ptr(up))
        return A, lo, up

    # -- variable-order BDF (the DLSODES family, Sec. 2.1) ----------------------------
    def bdf_run(self, h0=1e-8, t_end=1e30, stop_at_steady=False, max_steps=1000, rtol=1e-3, qmax=5,
                fixed_order=0, fixed_step=0, grow=5.0, raise_on_noconv=False):
        """Advances the state with xk_bdf_run; returns (BdfInfo, return code)."""
        cfg = BdfConfig(rtol=float(rtol), qmax=int(qmax), fixed_order=int(fixed_order),
                        fixed_step=int(fixed_step), grow=float(grow))
        info = BdfInfo()
        rc = lib().xk_bdf_run(self.h, C.byref(cfg), float(h0), float(t_end), int(bool(stop_at_steady)),
                              int(max_steps), C.byref(info))
        if rc != XK_OK and (raise_on_noconv or rc != -3):
            msg = lib().xk_last_error(self.h)
            raise XkError("xk_bdf_run", rc, msg.decode() if msg else "")
        return info, rc

    # -- equilibrium initial state (Sec. 2.5) and pathway analyser (Sec. 4) --------
    def equilibrium(self, b=None, set_state=False, max_iter=300, tol=1e-12):
        """Mole fractions [L, S] (device) of the Gibbs minimum at element totals b ([L, E] device
        tensor, or None for the current state's); set_state also makes n = x n_gas the state."""
        x = self._dev(self.L, self.S)
        bp = None if b is None else self._ptr(b.contiguous())
        info = EquilibriumInfo()
        self._call("xk_equilibrium", bp, self._ptr(x), int(bool(set_state)), int(max_iter), float(tol),
                   C.byref(info))
        return x, info

    def reaction_fluxes(self, n):
        """Forward and reverse rate of every reaction at state n: [L, R, 2] (device)."""
        q = self._dev(self.L, self.R, 2)
        self._call("xk_reaction_fluxes", self._ptr(n.contiguous()), self._ptr(q))
        return q

    def pathways(self, q, sources):
        """Dijkstra from each source species in every layer of rates q [L, R, 2]: dict of device
        tensors [nsrc, L, S] dist, pred_sp, pred_edge, lim_edge, lim_w."""
        t = self._torch
        src = np.ascontiguousarray(np.atleast_1d(sources), np.int32)
        shape = (len(src), self.L, self.S)
        out = dict(dist=self._dev(*shape), lim_w=self._dev(*shape),
                   pred_sp=t.empty(shape, dtype=t.int32, device=self.device),
                   pred_edge=t.empty(shape, dtype=t.int32, device=self.device),
                   lim_edge=t.empty(shape, dtype=t.int32, device=self.device))
        self._call("xk_pathways", self._ptr(q.contiguous()), len(src), src.ctypes.data_as(_ip),
                   self._ptr(out["dist"]), _vp(out["pred_sp"].data_ptr()), _vp(out["pred_edge"].data_ptr()),
                   _vp(out["lim_edge"].data_ptr()), self._ptr(out["lim_w"]))
        return out

    def block_solve(self, A, lo, up, f):
        x = self._dev(self.L, self.S)
        self._call("xk_block_solve", self._ptr(A.contiguous()), self._ptr(lo.contiguous()),
                   self._ptr(up.contiguous()), self._ptr(f.contiguous()), self._ptr(x))
        return x

    @staticmethod
    def lib_launches():
        return int(lib().xk_launch_count())

    @staticmethod
    def graph_launches():
        return int(lib().xk_graph_launch_count())

    def profile(self, enable=True):
        self._call("xk_profile", 1 if enable else 0)

    def profile_read(self):
        ms = (C.c_double * len(PHASES))()
        calls = (C.c_longlong * len(PHASES))()
        self._call("xk_profile_read", ms, calls, len(PHASES))
        return {p: (float(ms[i]), int(calls[i])) for i, p in enumerate(PHASES)}

    def factor_work(self):
        """(tensor-core product flops 2mnk, leaf inversion flops 2n^3) of one FP32 factorization."""
        m, l = C.c_double(), C.c_double()
        self._call("xk_factor_work", C.byref(m), C.byref(l))
        return m.value, l.value

    def block_solve32(self, A, lo, up, f):
        x = self._dev(self.L, self.S)
        self._call("xk_block_solve32", self._ptr(A.contiguous()), self._ptr(lo.contiguous()),
                   self._ptr(up.contiguous()), self._ptr(f.contiguous()), self._ptr(x))
        return x

    def hold_next_barrier(self):
        """Testing aid: the next grid barrier of the FP64 factorization never completes."""
        self._call("xk_hold_next_barrier")

    def step_delta(self, n, dt):
        d = self._dev(self.L, self.S)
        it = C.c_int()
        res = C.c_double()
        self._call("xk_step_delta", self._ptr(n.contiguous()), float(dt), self._ptr(d), C.byref(it), C.byref(res))
        return d, int(it.value), float(res.value)


class Batch:
    """Continuous batching of columns on one GPU (wraps xk_batch_*)."""

    def __init__(self, budget_bytes, max_slots, device=0):
        h = _vp()
        rc = lib().xk_batch_create(C.byref(h), int(device), C.c_size_t(int(budget_bytes)), int(max_slots))
        if rc != XK_OK:
            raise XkError("xk_batch_create", rc, "")
        self.h = h
        self.cols = {}

    def fits(self, nbytes):
        """Whether a column of this device footprint would be admitted now (no allocation)."""
        ok = C.c_int(0)
        rc = lib().xk_batch_fits(self.h, C.c_size_t(int(nbytes)), C.byref(ok))
        if rc != XK_OK:
            raise XkError("xk_batch_fits", rc, "")
        return bool(ok.value)

    def add(self, col, dt0=1e-8):
        """Admit a column; returns the slot, or None when it does not fit (footprint or slots)."""
        slot = C.c_int(-1)
        rc = lib().xk_batch_add(self.h, col.h, float(dt0), C.byref(slot))
        if rc == -2:
            return None
        if rc != XK_OK:
            msg = lib().xk_last_error(col.h)
            raise XkError("xk_batch_add", rc, msg.decode() if msg else "")
        self.cols[slot.value] = col
        return slot.value

    def remove(self, slot):
        rc = lib().xk_batch_remove(self.h, int(slot))
        if rc != XK_OK:
            raise XkError("xk_batch_remove", rc, "")
        return self.cols.pop(slot)

    def step(self, nsteps=1):
        rc = lib().xk_batch_step(self.h, int(nsteps))
        if rc != XK_OK:
            msg = lib().xk_batch_last_error(self.h)
            raise XkError("xk_batch_step", rc, msg.decode() if msg else "")

    def _raise(self, name, rc):
        msg = lib().xk_batch_last_error(self.h)
        raise XkError(name, rc, msg.decode() if msg else "")

    def submit(self, slot, nsteps):
        """Enqueue nsteps controlled steps for one slot without waiting."""
        rc = lib().xk_batch_submit(self.h, int(slot), int(nsteps))
        if rc != XK_OK:
            self._raise("xk_batch_submit", rc)

    def query(self, slot):
        """True once the slot's submitted steps have run (then poll() is current)."""
        done = C.c_int(0)
        rc = lib().xk_batch_query(self.h, int(slot), C.byref(done))
        if rc != XK_OK:
            self._raise("xk_batch_query", rc)
        return bool(done.value)

    def poll(self, slot):
        info = RunInfo()
        fin = C.c_int()
        st = C.c_int()
        rc = lib().xk_batch_poll(self.h, int(slot), C.byref(info), C.byref(fin), C.byref(st))
        if rc != XK_OK:
            raise XkError("xk_batch_poll", rc, "")
        return info, bool(fin.value), int(st.value)

    def close(self):
        if getattr(self, "h", None):
            lib().xk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

