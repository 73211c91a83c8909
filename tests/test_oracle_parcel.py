"""Pins of the oracle's Lagrangian parcel scheme (Sec. 2, Fig. 2: one global
iteration carries an air parcel from the bottom of the atmosphere to the top and
back; eddy mixing is the parcel's motion, molecular diffusion a pseudo-reaction
pair with the neighbouring layers, Sec. 2.1).  No GPU needed.

Each pin checks one part of the sweep against something the oracle does not
compute itself: a closed form, an invariant, a limit, finite differences."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, default_policy
from paper_2512_06729_gb300 import synth
from tests.helpers import custom_problem, nasa_const_cp


def _visits(L):
    return list(range(L)) + list(range(L - 2, -1, -1))


def _two_species_column(L=7, T=900.0, dcoef=0.0, kf=3.0e-8):
    """kf (1/s) of the order of 1 / tau_k, so that every visit relaxes the parcel partly."""
    nasa = np.stack([nasa_const_cp(3.0, 0.0, 1.0), nasa_const_cp(3.0, -800.0, 0.5)])
    rx = [dict(type=0, reac=[0], prod=[1], arr=[kf, 0.0, 0.0])]
    P = np.geomspace(1.0, 1e-4, L)
    Kzz = np.geomspace(3e7, 5e9, L)            # residence times differ from layer to layer
    f0 = np.tile([0.9, 0.1], (L, 1))
    f0[:, 0] = np.linspace(0.9, 0.2, L)       # the profile above the bottom is overwritten
    f0[:, 1] = 1.0 - f0[:, 0]
    return custom_problem(np.array([[1], [1]], np.int32), [10.0, 10.0], rx, nasa, P, np.full(L, T),
                          Kzz=Kzz, dcoef=np.full(2, dcoef), f0=f0)


def test_two_species_sweep_closed_form():
    """A <-> B, isothermal, no diffusion, one implicit Euler step per visit (no
    step limit, no rejection, no growth): each visit of layer k divides the
    parcel's distance from equilibrium by (1 + (kf + kr) tau_k), tau_k = dz_k^2 /
    K_zz,k; the mixing ratio is carried from layer to layer, and layer k keeps the
    parcel's state at its last visit (on the way down; the top layer once)."""
    p = _two_species_column()
    o = Oracle(p)
    ngas, _, dz, _ = o.grid()
    kf, kr = o.rate_coefficients()
    lam = kf[0, 0] + kr[0, 0]
    assert np.allclose(kf[:, 0], kf[0, 0], rtol=0) and np.allclose(kr[:, 0], kr[0, 0], rtol=1e-15)
    xeq = kr[0, 0] / lam
    N0 = o.initial_state()
    pol = default_policy(dt_max=1e300, rel_reject=math.inf, grow_max=1.0, shrink_min=1.0)
    N, info = o.parcel_iteration(N0, h=1e300, policy=pol)
    assert info.steps == 2 * p.L - 1 and info.rejected == 0
    x = p.f0[0, 0]
    expect = np.zeros(p.L)
    for k in _visits(p.L):
        x = xeq + (x - xeq) / (1.0 + lam * dz[k] ** 2 / p.Kzz[k])
        expect[k] = x
    np.testing.assert_allclose(N[:, 0] / ngas, expect, rtol=1e-12)
    np.testing.assert_allclose(N.sum(axis=1), ngas, rtol=1e-12)     # A + B carried with the gas
    rel = np.abs(N - N0) / N
    assert info.max_change == pytest.approx(rel.max(), rel=1e-14)


def test_two_species_adaptive_visits_follow_the_exponential():
    """The same column under a tight step controller (relative change per step
    at most 2e-4): the visits integrate dx/dt = -(kf + kr)(x - x_eq) over
    exactly tau_k each, so layer k holds x_eq + (x_0 - x_eq) exp(-(kf + kr) t_k),
    t_k the parcel's time up to its last visit of k (backward Euler's error at
    that step size: well under 0.5 % of the distance from equilibrium)."""
    p = _two_species_column()
    o = Oracle(p)
    ngas, _, dz, _ = o.grid()
    kf, kr = o.rate_coefficients()
    lam = kf[0, 0] + kr[0, 0]
    xeq = kr[0, 0] / lam
    pol = default_policy(rel_target=1e-4, rel_reject=2e-4)
    N, info = o.parcel_iteration(o.initial_state(), h=1e-3, policy=pol)
    assert info.steps > 10 * (2 * p.L - 1)
    t = 0.0
    x0 = p.f0[0, 0]
    expect = np.zeros(p.L)
    for k in _visits(p.L):
        t += dz[k] ** 2 / p.Kzz[k]
        expect[k] = xeq + (x0 - xeq) * math.exp(-lam * t)
    got = N[:, 0] / ngas
    np.testing.assert_allclose(got - xeq, expect - xeq, rtol=5e-3)


def test_element_mixing_ratios_carried_without_diffusion():
    """Without molecular diffusion the parcel exchanges nothing with the layers:
    chemistry (photolysis included) conserves each element's mixing ratio, so
    after one iteration every layer holds the element mixing ratios of the
    bottom layer's starting composition."""
    p = synth.small_column(S=24, L=10, n_two=40, n_three=10, n_photo=6, W=60, elements="cho")
    p.dcoef = np.zeros(p.S)
    o = Oracle(p)
    ngas = o.grid()[0]
    N0 = o.initial_state()
    # no negative density accepted, so nothing is clipped
    N, info = o.parcel_iteration(N0, policy=default_policy(neg_tol=0.0))
    assert N.min() >= 0.0 and info.steps >= 2 * p.L - 1
    E = p.elem.astype(float)
    start = (N0[0] / ngas[0]) @ E
    got = (N / ngas[:, None]) @ E
    # rounding of the largest densities sets the floor: relative to the total mixing ratio
    scale = (N0[0] / ngas[0]).sum() * E.max()
    np.testing.assert_allclose(got, np.tile(start, (p.L, 1)), rtol=0, atol=1e-12 * scale)


def test_zero_residence_time_carries_the_bottom_composition():
    """K_zz -> infinity: the parcel spends no time in any layer, so the sweep
    only carries the bottom layer's mixing ratios to every layer."""
    p = synth.tiny_column()
    p.Kzz = np.full(p.L, 1e40)
    o = Oracle(p)
    ngas = o.grid()[0]
    N0 = o.initial_state()
    N, info = o.parcel_iteration(N0)
    assert info.steps == 2 * p.L - 1
    np.testing.assert_allclose(N / ngas[:, None], np.tile(N0[0] / ngas[0], (p.L, 1)), rtol=1e-12)


def test_visit_system_jacobian_matches_central_differences():
    """A = I/h - dF/dpk with h -> infinity is minus the derivative of F, the
    diffusion exchange included (the neighbours' stored densities are fixed)."""
    p = synth.small_column(S=18, L=5, n_two=20, n_three=6, n_photo=3, W=40, elements="cho")
    p.dcoef = np.full(p.S, 3e18)
    o = Oracle(p)
    ngas = o.grid()[0]
    rng = np.random.default_rng(3)
    N = ngas[:, None] * rng.uniform(0.5, 1.5, size=(p.L, p.S)) / p.S
    for k in (0, 2, p.L - 1):
        pk = N[k] * rng.uniform(0.8, 1.2, size=p.S)
        F, A = o.parcel_system(N, k, pk, 1e300)
        fd = np.zeros((p.S, p.S))
        for j in range(p.S):
            h = 1e-5 * pk[j]
            e = np.zeros(p.S); e[j] = h
            fd[:, j] = -(o.parcel_system(N, k, pk + e, 1e300)[0] - o.parcel_system(N, k, pk - e, 1e300)[0]) / (2 * h)
        scale = np.abs(A).max(axis=1, keepdims=True) + 1e-300
        assert np.abs((A - fd) / scale).max() < 1e-6, k


def test_diffusion_pair_is_the_molecular_flux_and_conserves():
    """Chemistry off, parcel equal to the stored layer: the pseudo-reaction pair
    is the molecular part of Eq. 2's flux divergence, so sum_k dz_k F_k = 0
    (zero flux at both ends), and a uniform mixing ratio on an isothermal column
    is pulled towards diffusive equilibrium: light species up, heavy down."""
    L = 12
    P = np.geomspace(1.0, 1e-3, L)
    S = 2
    p = custom_problem(np.eye(S, dtype=np.int32), [2.0, 40.0], [], np.stack([nasa_const_cp(2.5, 0, 0)] * S),
                       P, np.full(L, 1000.0), Kzz=np.full(L, 1e8), dcoef=np.full(S, 1e17),
                       f0=np.tile([0.5, 0.5], (L, 1)))
    o = Oracle(p)
    ngas, _, dz, _ = o.grid()
    N = o.initial_state()
    F = np.stack([o.parcel_system(N, k, N[k], 1e300)[0] for k in range(L)])
    scale = np.abs(F).max()
    assert scale > 0
    np.testing.assert_allclose((dz[:, None] * F).sum(axis=0), 0.0, atol=1e-12 * scale * dz.max())
    # well mixed in n_gas: the light species gains at the top, the heavy one at the bottom
    assert F[-1, 0] > 0 and F[0, 0] < 0
    assert F[-1, 1] < 0 and F[0, 1] > 0


def test_run_stops_at_the_tolerance():
    """Sec. 2: global iterations until successive profiles differ by less than
    the tolerance (0.1 % in the paper; here 10 %, which the tiny column reaches in
    a few iterations: its slowest trace species decay by a few % per iteration)."""
    p = synth.tiny_column()
    o = Oracle(p)
    N0 = o.initial_state()
    N, iters, info, ok = o.parcel_run(N0, tol=0.1, max_iter=400)
    assert ok and info.max_change < 0.1 and iters >= 2
    # one iteration fewer had not converged
    _, it2, info2, ok2 = o.parcel_run(N0, tol=0.1, max_iter=iters - 1)
    assert not ok2 and info2.max_change >= 0.1 and it2 == iters - 1
    assert np.all(np.isfinite(N)) and N.min() >= 0.0
