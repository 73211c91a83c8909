"""Lagrangian parcel scheme (Sec. 2, Fig. 2) on the GPU against the oracle, through the C-ABI:
global iterations on the tiny, small and 30-species columns element by element; the closed-form
two-species sweep; element mixing ratios carried unchanged without diffusion; the stopping rule;
many columns swept at once on their own streams; argument errors.

Tolerance.  Both sides take the same linearly implicit Euler steps, each solved to a few ulp
(partial-pivot LU plus two FP64 refinement sweeps), but they sum each species' production and
loss in different orders, and the net right-hand side of a trace species is a small difference
of large terms.  The sweep then carries that rounding through hundreds of long implicit steps: the
oracle itself, given its input perturbed by 1e-13 relative, moves by 1e-5 (tiny column) to 1e-2
(30 species) after one iteration.  So the bound is derived in the test from that spread, 10 x the
larger of two such perturbed oracle runs (at least 1e-9), and the accepted and rejected step
counts must agree whenever the perturbed oracle runs agree on them.  The closed form and the
conservation test below are the tight checks (1e-12)."""
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
PERTURB = 1e-13


def _rel(a, b, ngas):
    keep = b > 1e-20 * ngas[:, None]
    return float(np.max(np.abs(a[keep] - b[keep]) / b[keep]))


def _oracle_iterations(o, N, h, iterations):
    out = []
    for _ in range(iterations):
        N, info = o.parcel_iteration(N, h=h)
        out.append((N, info))
        h = info.h
    return out


def _spread(o, N, h, iterations, ngas):
    """The oracle's own sensitivity: two runs from N perturbed by PERTURB relative."""
    ref = _oracle_iterations(o, N, h, iterations)
    rng = np.random.default_rng(7)
    state, hspread, counts_stable = 0.0, 0.0, True
    for _ in range(2):
        run = _oracle_iterations(o, N * (1.0 + PERTURB * rng.standard_normal(N.shape)), h, iterations)
        for (Na, ia), (Nb, ib) in zip(ref, run):
            counts_stable &= (ia.steps, ia.rejected) == (ib.steps, ib.rejected)
            hspread = max(hspread, abs(ia.h - ib.h) / ia.h)
        state = max(state, _rel(run[-1][0], ref[-1][0], ngas))
    return ref, state, hspread, counts_stable


CASES = {
    "tiny": synth.tiny_column,
    "small": synth.small_column,
    "s30": lambda: synth.small_column(S=30, L=45, n_two=80, n_three=20, n_photo=6, seed=9, W=120),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("start", ["initial", "relaxed"])
@pytest.mark.parametrize("iterations", [1, 3])
def test_parcel_iterations_match_oracle(case, start, iterations):
    p = CASES[case]()
    o = Oracle(p)
    ngas = o.grid()[0]
    N0, h0 = o.initial_state(), 1e-8
    if start == "relaxed":                  # three oracle iterations first: past the initial transient
        N0, info = _oracle_iterations(o, N0, h0, 3)[-1]
        h0 = info.h
    ref, spread, hspread, stable = _spread(o, N0, h0, iterations, ngas)
    bound = max(10.0 * spread, 1e-9)
    col = xk.Column(p, "fp64")
    col.set_state(N0)
    h = h0
    for it, (N, oi) in enumerate(ref):
        gi = col.parcel_iteration(h=h)
        if stable:
            assert (gi.steps, gi.rejected) == (oi.steps, oi.rejected), it
        assert abs(gi.h - oi.h) <= max(10.0 * hspread, 1e-9) * oi.h, it
        h = gi.h
    got = col.get_state()
    err = _rel(got, ref[-1][0], ngas)
    assert err <= bound, (err, bound)
    assert got.min() >= 0.0


def test_parcel_keeps_element_mixing_ratios():
    """No molecular diffusion and no negative density accepted: the GPU sweep carries the bottom
    layer's element mixing ratios to every layer (chemistry and photolysis conserve elements)."""
    p = synth.small_column(S=24, L=10, n_two=40, n_three=10, n_photo=6, W=60, elements="cho")
    p.dcoef = np.zeros(p.S)
    o = Oracle(p)
    ngas = o.grid()[0]
    N0 = o.initial_state()
    col = xk.Column(p, "fp64", neg_tol=0.0)
    col.set_state(N0)
    info = col.parcel_iteration()
    assert info.steps >= 2 * p.L - 1
    N = col.get_state()
    E = p.elem.astype(float)
    start = (N0[0] / ngas[0]) @ E
    got = (N / ngas[:, None]) @ E
    scale = (N0[0] / ngas[0]).sum() * E.max()
    np.testing.assert_allclose(got, np.tile(start, (p.L, 1)), rtol=0, atol=1e-12 * scale)


def test_parcel_columns_at_once_equal_one_by_one():
    """begin/end on several columns with their own streams: each result equals the same column's
    iteration run alone (same kernel, same inputs: bit for bit)."""
    probs = [synth.small_column(S=S, L=30, n_two=40, n_three=10, n_photo=4, seed=40, W=60) for S in (24, 28, 32, 36)]
    alone = []
    for p in probs:
        c = xk.Column(p, "fp64")
        c.set_mixing_ratios(p.f0)
        info = c.parcel_iteration()
        alone.append((c.get_state(), info))
    streams = [torch.cuda.Stream() for _ in probs]
    cols = []
    for p, st in zip(probs, streams):
        c = xk.Column(p, "fp64", stream=st)
        c.set_mixing_ratios(p.f0)
        cols.append(c)
    for c in cols:
        c.parcel_begin()
    for c, (n_alone, ia) in zip(cols, alone):
        ib = c.parcel_end()
        assert (ib.steps, ib.rejected, ib.h, ib.max_change) == (ia.steps, ia.rejected, ia.h, ia.max_change)
        assert np.array_equal(c.get_state(), n_alone)


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
    """Iterations until the change falls below 10 % (the tiny column reaches it in a few)."""
    p = synth.tiny_column()
    o = Oracle(p)
    ngas = o.grid()[0]
    n0 = o.initial_state()
    N, it_o, oi, ok_o = o.parcel_run(n0, tol=0.1, max_iter=400)
    col = xk.Column(p, "fp64")
    col.set_state(n0)
    it_g, gi, ok_g = col.parcel_run(tol=0.1, max_iter=400)
    assert ok_o and ok_g and it_g == it_o
    _, spread, _, _ = _spread(o, n0, 1e-8, it_o, ngas)
    assert _rel(col.get_state(), N, ngas) <= max(10.0 * spread, 1e-9)


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
