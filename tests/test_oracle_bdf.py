"""Pins of the oracle's variable-order, variable-step BDF integrator (the DLSODES family of
Sec. 2.1): textbook coefficients, exactness on polynomials, the corrector equation on a linear
network at every order and step, and convergence with the tolerance (no GPU needed)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, bdf_coeffs, bdf_extrap, default_policy
from paper_2512_06729_gb300 import synth
from tests.helpers import custom_problem, nasa_const_cp

# textbook fixed-step BDF coefficients (h = 1): c_0 y_{n+1} + c_1 y_n + ... = f(y_{n+1})
TEXTBOOK = {
    1: [1.0, -1.0],
    2: [3 / 2, -2.0, 1 / 2],
    3: [11 / 6, -3.0, 3 / 2, -1 / 3],
    4: [25 / 12, -4.0, 3.0, -4 / 3, 1 / 4],
    5: [137 / 60, -5.0, 5.0, -10 / 3, 5 / 4, -1 / 5],
}


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_fixed_step_coefficients_are_the_textbook_bdf(q):
    for h in (1.0, 0.37):
        tau = [10.0 - j * h for j in range(q + 1)]
        np.testing.assert_allclose(bdf_coeffs(tau) * h, TEXTBOOK[q], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_variable_step_coefficients_differentiate_polynomials(q):
    """On uneven nodes sum_j c_j p(tau_j) = p'(tau_0) for every polynomial of degree <= q."""
    rng = np.random.default_rng(q)
    tau = 5.0 - np.concatenate([[0.0], np.cumsum(rng.uniform(0.1, 2.0, q))])
    c = bdf_coeffs(tau)
    for d in range(q + 1):
        p = lambda t: (t - 4.0) ** d
        dp = d * (tau[0] - 4.0) ** (d - 1) if d else 0.0
        assert np.dot(c, p(tau)) == pytest.approx(dp, rel=1e-10, abs=1e-10)
    # degree q + 1 is not exact in general: the formula has order q
    p = (tau - 4.0) ** (q + 1)
    assert abs(np.dot(c, p) - (q + 1) * (tau[0] - 4.0) ** q) > 1e-6


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_extrapolation_reproduces_polynomials(m):
    rng = np.random.default_rng(10 + m)
    tau = np.sort(rng.uniform(0, 3, m))[::-1].copy()
    t = 3.5
    w = bdf_extrap(tau, t)
    assert w.sum() == pytest.approx(1.0, rel=1e-12)
    for d in range(m):
        assert np.dot(w, (tau - 1.0) ** d) == pytest.approx((t - 1.0) ** d, rel=1e-9, abs=1e-9)


def _ab_problem():
    T = 900.0
    nasa = np.stack([nasa_const_cp(3.0, 0.0, 1.0), nasa_const_cp(3.0, -800.0, 0.5)])
    elem = np.array([[1], [1]], np.int32)
    rx = [dict(type=0, reac=[0], prod=[1], arr=[2.0e-3, 0.0, 0.0])]
    return custom_problem(elem, [10.0, 10.0], rx, nasa, [1.0], [T], f0=np.array([[0.9, 0.1]]))


def test_corrector_equation_holds_at_every_step():
    """A <-> B is linear, so the linearly implicit step is the exact BDF step: after every accepted
    step, c_0 y_new + sum c_j y_j = F(y_new) with the variable-step coefficients of that step's
    order, read off the run (each prefix of a run is a run with fewer steps)."""
    p = _ab_problem()
    o = Oracle(p)
    kf, kr = (x[0, 0] for x in o.rate_coefficients())
    n0 = o.initial_state()
    states, times, orders = [n0[0].copy()], [0.0], []
    prev_hist = [0] * 6
    for N in range(1, 60):
        m, info, rc = o.bdf_run(n0, h0=1e-3, t_end=1e4, max_steps=N, rtol=1e-5)
        if info.accepted == len(states):           # the N-th attempt was accepted
            hist = list(info.order_steps)
            q = [i for i in range(6) if hist[i] != prev_hist[i]][0]
            prev_hist = hist
            states.append(m[0].copy())
            times.append(info.t)
            orders.append(q)
    assert max(orders) >= 3, orders
    for i, q in enumerate(orders, start=1):
        tau = [times[i]] + [times[i - j] for j in range(1, q + 1)]
        c = bdf_coeffs(tau)
        lhs = c[0] * states[i] + sum(c[j] * states[i - j] for j in range(1, q + 1))
        y = states[i]
        F = np.array([-kf * y[0] + kr * y[1], kf * y[0] - kr * y[1]])
        scale = abs(c[0]) * abs(y).max()
        assert np.max(np.abs(lhs - F)) < 1e-10 * scale, (i, q)


def test_error_falls_with_the_tolerance():
    p = _ab_problem()
    o = Oracle(p)
    kf, kr = (x[0, 0] for x in o.rate_coefficients())
    n0 = o.initial_state()
    ntot = n0.sum()
    neq = ntot * kr / (kf + kr)
    T = 2.0 / (kf + kr)
    errs = []
    rtols = (1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8)
    for rtol in rtols:
        m, info, rc = o.bdf_run(n0, h0=1e-6, t_end=T, max_steps=100000, rtol=rtol)
        assert rc == 0 and info.t == pytest.approx(T, rel=1e-12)
        exact = neq + (n0[0, 0] - neq) * math.exp(-(kf + kr) * T)
        errs.append(abs(m[0, 0] - exact) / exact)
        assert errs[-1] < 10 * rtol
        assert m.sum() == pytest.approx(ntot, rel=1e-12)
    # the global error follows the local tolerance: two decades tighter, a smaller error
    for a, b in zip(errs, errs[2:]):
        assert b < a
    assert errs[-1] < errs[0] / 1000


def test_local_error_estimate_of_order_one():
    """At order 1 with a linear predictor the estimate (y_new - y_hat) / 2 is the step's true local
    error h^2 y''/2 (A <-> B: exact solution from the previous accepted state)."""
    p = _ab_problem()
    o = Oracle(p)
    kf, kr = (x[0, 0] for x in o.rate_coefficients())
    n0 = o.initial_state()
    ntot = n0.sum()
    neq = ntot * kr / (kf + kr)
    ratios = []
    prev = None
    for N in range(1, 40):
        m, info, rc = o.bdf_run(n0, h0=1e-2, t_end=1e5, max_steps=N, rtol=1e-4, fixed_order=1)
        if prev is not None and info.accepted == prev[1].accepted + 1 and N > 5:
            h = info.t - prev[1].t
            xa = neq + (prev[0][0, 0] - neq) * np.exp(-(kf + kr) * h)
            exact = np.array([xa, ntot - xa])
            true = np.max(np.abs(m[0] - exact) / m[0])
            ratios.append(info.err * 1e-4 / true)
        prev = (m, info)
    assert len(ratios) > 10
    assert 0.7 < np.median(ratios) < 1.4, ratios


def test_fixed_order_converges_at_its_order():
    """Fixed steps at order 1 and 2 (order 2 starts with one backward-Euler step, itself of local
    order 2): halving h divides the error at T by about 2^q."""
    p = _ab_problem()
    o = Oracle(p)
    kf, kr = (x[0, 0] for x in o.rate_coefficients())
    n0 = o.initial_state()
    neq = n0.sum() * kr / (kf + kr)
    T = 1.0 / (kf + kr)
    exact = neq + (n0[0, 0] - neq) * math.exp(-(kf + kr) * T)
    for q in (1, 2):
        e = []
        for N in (40, 80, 160):
            m, info, rc = o.bdf_run(n0, h0=T / N, t_end=T, max_steps=10 * N, fixed_order=q, fixed_step=1, qmax=q)
            assert rc == 0 and info.accepted == N
            e.append(abs(m[0, 0] - exact))
        for a, b in zip(e, e[1:]):
            assert a / b == pytest.approx(2.0 ** q, rel=0.1)


def _relative_residual(o, p, m):
    """max |F| over the gross production + loss + transport flux of each entry above 1e-20."""
    q = o.fluxes(m)
    F = o.residual(m)
    nu = np.zeros((p.R, p.S))
    for r in range(p.R):
        for s in p.reac[r]:
            if s >= 0:
                nu[r, s] -= 1
        for s in p.prod[r]:
            if s >= 0:
                nu[r, s] += 1
    gross = (q[:, :, 0] + q[:, :, 1]) @ np.abs(nu)
    u, v = o.transport()
    ngas, _, dz, _ = o.grid()
    tr = np.zeros_like(m)
    g = np.abs(u * m[:-1]) + np.abs(v * m[1:])
    tr[:-1] += g / dz[:-1, None]
    tr[1:] += g / dz[1:, None]
    keep = m > 1e-20 * ngas[:, None]
    return float(np.max(np.abs(F[keep]) / (gross + tr)[keep]))


def test_variable_order_run_reaches_the_steady_state():
    """On the tiny column the adaptive run climbs to high orders and ends at a fixed point: F = 0
    to 1e-9 of the gross fluxes under a tight steady-state test (the initial state is at ~1)."""
    p = synth.tiny_column()
    o = Oracle(p)
    n0 = o.initial_state()
    pol = default_policy(ss_tol=1e-9, ss_dt=1e11, dt_max=1e13)
    m, info, rc = o.bdf_run(n0, h0=1e-8, stop_at_steady=True, max_steps=8000, policy=pol)
    assert rc == 0 and info.converged
    assert info.order_steps[4] + info.order_steps[5] > info.accepted // 2
    assert _relative_residual(o, p, n0) > 0.5
    assert _relative_residual(o, p, m) < 1e-9
