"""Lagrangian parcel scheme (Sec. 2, Fig. 2) on the GPU against the oracle, through the C-ABI:
one global iteration and several, on the tiny and small columns, element by element on every
species above 1e-20 mixing ratio, with the same step-controller decisions (accepted and rejected
step counts); the closed-form two-species sweep; the stopping rule; argument errors.

Tolerance: both sides take the same linearly implicit Euler steps; they differ in the rounding
of the dense solves (the oracle adds two refinement sweeps; the kernel eliminates in another
order), a few ulp times the condition number of each step's matrix, carried through the sweep.
1e-9 relative leaves room for that and fails on any wrong term, index or decision."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle.oracle import Oracle, default_policy  # noqa: E402
from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import synth, xk  # noqa: E402
from tests.test_oracle_parcel import _two_species_column, _visits  # noqa: E402

xkbuild.build()
TOL = 1e-9


def _rel(a, b, ngas):
    keep = b > 1e-20 * ngas[:, None]
    return float(np.max(np.abs(a[keep] - b[keep]) / b[keep]))


def _pair(p, **kw):
    o = Oracle(p)
    col = xk.Column(p, "fp64", **kw)
    n0 = o.initial_state()
    col.set_state(n0)
    return o, col, n0


@pytest.mark.parametrize("make", [synth.tiny_column, synth.small_column,
                                  lambda: synth.small_column(S=30, L=45, n_two=80, n_three=20, n_photo=6, seed=9, W=120)])
@pytest.mark.parametrize("iterations", [1, 4])
def test_parcel_iterations_match_oracle(make, iterations):
    p = make()
    o, col, n0 = _pair(p)
    ngas = o.grid()[0]
    N = n0
    h_o = h_g = 1e-8
    for it in range(iterations):
        N, oi = o.parcel_iteration(N, h=h_o)
        gi = col.parcel_iteration(h=h_g)
        assert (gi.steps, gi.rejected) == (oi.steps, oi.rejected), it
        assert gi.h == pytest.approx(oi.h, rel=1e-6)
        assert gi.max_change == pytest.approx(oi.max_change, rel=1e-6, abs=1e-12)
        h_o, h_g = oi.h, gi.h
    got = col.get_state()
    assert _rel(got, N, ngas) <= TOL
    assert got.min() >= 0.0


def test_parcel_two_species_closed_form():
    """One implicit Euler step per visit: the distance from equilibrium shrinks by
    1 / (1 + (kf + kr) tau_k) at each visit, tau_k = dz_k^2 / K_zz,k."""
    p = _two_species_column()
    o = Oracle(p)
    ngas, _, dz, _ = o.grid()
    kf, kr = o.rate_coefficients()
    lam = kf[0, 0] + kr[0, 0]
    xeq = kr[0, 0] / lam
    col = xk.Column(p, "fp64", dt_max=1e300, rel_reject=math.inf, grow_max=1.0, shrink_min=1.0)
    col.set_state(o.initial_state())
    info = col.parcel_iteration(h=1e300)
    assert info.steps == 2 * p.L - 1 and info.rejected == 0
    x = p.f0[0, 0]
    expect = np.zeros(p.L)
    for k in _visits(p.L):
        x = xeq + (x - xeq) / (1.0 + lam * dz[k] ** 2 / p.Kzz[k])
        expect[k] = x
    np.testing.assert_allclose(col.get_state()[:, 0] / ngas, expect, rtol=1e-12)


def test_parcel_run_stops_like_the_oracle():
    p = synth.tiny_column()
    o, col, n0 = _pair(p)
    ngas = o.grid()[0]
    N, it_o, oi, ok_o = o.parcel_run(n0, tol=0.1, max_iter=400)
    it_g, gi, ok_g = col.parcel_run(tol=0.1, max_iter=400)
    assert ok_o and ok_g and it_g == it_o
    assert (gi.steps, gi.rejected) == (oi.steps, oi.rejected)
    assert _rel(col.get_state(), N, ngas) <= TOL


def test_parcel_needs_positive_kzz():
    p = synth.tiny_column()
    p.Kzz = p.Kzz.copy()
    p.Kzz[3] = 0.0
    col = xk.Column(p, "fp64")
    col.set_mixing_ratios(p.f0)
    with pytest.raises(xk.XkError) as e:
        col.parcel_iteration()
    assert e.value.code == -1
    with pytest.raises(xk.XkError):
        col.parcel_iteration(h=0.0)
