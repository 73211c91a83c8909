"""Pins of the oracle's extinction and diffuse field (Sec. 2.3.3): Rayleigh scattering in the
optical depth, and the two-stream photon budget behind J_diff = (J_up + J_down) / 2 (no GPU)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, two_stream
from paper_2512_06729_gb300 import synth


def _layers(rng, L, scatter=True):
    ta = 10.0 ** rng.uniform(-3, 0.5, L)
    ts = 10.0 ** rng.uniform(-3, 0.5, L) if scatter else np.zeros(L)
    return ta, ts


def _coeffs(ta, ts):
    dt = ta + ts
    om = np.where(dt > 0, ts / np.where(dt > 0, dt, 1), 0.0)
    t = np.exp(-dt / 0.5)
    return dt, om, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_two_stream_photon_budget(seed):
    """Every photon of the beam (mu F0 per unit horizontal area) leaves through the top, is
    absorbed in a layer (beam or diffuse) or is absorbed by the lower boundary."""
    rng = np.random.default_rng(seed)
    L = 40
    ta, ts = _layers(rng, L)
    mu, F0, A = rng.uniform(0.2, 1.0), 10.0 ** rng.uniform(8, 14), rng.uniform(0, 1)
    U, D, Jd = two_stream(ta, ts, F0, mu, A)
    dt, om, t = _coeffs(ta, ts)
    tau_top = np.concatenate([np.cumsum(dt[::-1])[::-1][1:], [0.0]])   # optical depth above each layer
    beam_lost = mu * F0 * (np.exp(-tau_top / mu) - np.exp(-(tau_top + dt) / mu))
    absorbed = np.sum((1 - om) * beam_lost) + np.sum((1 - t) * (1 - om) * (D[1:] + U[:-1]))
    bottom = mu * F0 * math.exp(-dt.sum() / mu)
    out = U[L] + absorbed + (1 - A) * (D[0] + bottom)
    assert out == pytest.approx(mu * F0, rel=1e-12)
    assert D[L] == 0.0 and np.all(U >= 0) and np.all(D >= 0)
    assert np.allclose(Jd, 0.25 * (U[:-1] + U[1:] + D[:-1] + D[1:]), rtol=1e-15)


def test_two_stream_conservative_reflecting():
    """No absorption anywhere and a white lower boundary: the whole beam comes back out of the top."""
    rng = np.random.default_rng(5)
    L = 25
    ts = 10.0 ** rng.uniform(-2, 1, L)
    mu, F0 = 0.6, 3e13
    U, D, Jd = two_stream(np.zeros(L), ts, F0, mu, 1.0)
    assert U[L] == pytest.approx(mu * F0, rel=1e-12)


def test_two_stream_one_layer_closed_form():
    ta, ts, F0, mu, A = 0.3, 0.7, 2.0, 0.5, 0.4
    U, D, Jd = two_stream([ta], [ts], F0, mu, A)
    dt = ta + ts
    om, t = ts / dt, math.exp(-dt / 0.5)
    r, T = (1 - t) * om / 2, t + (1 - t) * om / 2
    P = om * mu * F0 * (1 - math.exp(-dt / mu))
    B = mu * F0 * math.exp(-dt / mu)
    U0 = A * (P / 2 + B) / (1 - A * r)
    D0 = r * U0 + P / 2
    U1 = T * U0 + P / 2
    assert U[0] == pytest.approx(U0, rel=1e-14)
    assert D[0] == pytest.approx(D0, rel=1e-14)
    assert U[1] == pytest.approx(U1, rel=1e-14)
    assert Jd[0] == pytest.approx(0.25 * (U0 + U1 + D0), rel=1e-14)


def test_two_stream_pure_absorption():
    """Without scattering there is no diffuse source; a reflecting bottom sends the beam back up,
    attenuated by exp(-2 dtau) per layer (the hemispheric mean path), and nothing comes down."""
    rng = np.random.default_rng(9)
    L = 12
    ta, _ = _layers(rng, L, scatter=False)
    mu, F0 = 0.5, 1e12
    U, D, Jd = two_stream(ta, np.zeros(L), F0, mu, 0.0)
    assert np.all(U == 0) and np.all(D == 0) and np.all(Jd == 0)
    U, D, Jd = two_stream(ta, np.zeros(L), F0, mu, 0.7)
    B = mu * F0 * math.exp(-ta.sum() / mu)
    expect = 0.7 * B * np.concatenate([[1.0], np.cumprod(np.exp(-ta / 0.5))])
    assert np.allclose(U, expect, rtol=1e-13, atol=0)
    assert np.all(D == 0)


def test_rayleigh_extinction_enters_the_beam():
    """A column whose only extinction is Rayleigh scattering: k_ph follows J0 exp(-tau_s/mu) with
    tau_s = sum sigma_s n dz to the layer midpoint, and adding the diffuse field raises every rate."""
    p = synth.small_column()
    o = Oracle(p)
    n = o.initial_state()
    ngas, z, dz, dzi = o.grid()
    ps = synth.with_scattering(p, diffuse=0).replace(sigma_abs=np.zeros_like(p.sigma_abs))
    kph = Oracle(ps).photolysis(n)
    alpha_s = n @ ps.sigma_s                               # [L, W]
    ext = alpha_s * dz[:, None]
    above = np.concatenate([np.cumsum(ext[::-1], axis=0)[::-1][1:], np.zeros((1, p.W))])
    J = p.J0 * np.exp(-(above + 0.5 * ext) / p.mu)
    ref = p.tf * J @ (p.sigma * p.dlam).T
    np.testing.assert_allclose(kph, ref, rtol=1e-12)
    kd = Oracle(ps.replace(diffuse=1, albedo=0.2)).photolysis(n)
    assert np.all(kd >= kph) and np.any(kd > kph * (1 + 1e-3))


def test_scattering_off_is_the_direct_beam():
    p = synth.small_column()
    o = Oracle(p)
    n = o.initial_state()
    base = o.photolysis(n)
    z = synth.with_scattering(p, diffuse=1).replace(sigma_s=np.zeros((p.S, p.W)))
    assert np.array_equal(Oracle(z).photolysis(n), base)


# ------------------------------------------------ photolysis rates in the Jacobian

def _relaxed_small():
    p = synth.small_column(L=20)
    o = Oracle(p)
    n, info = o.run_to_steady(o.initial_state(), max_steps=300)
    return p, o, n


def _stoich(p):
    nu = np.zeros((p.R, p.S))
    for r in range(p.R):
        for s in p.reac[r]:
            if s >= 0:
                nu[r, s] -= 1
        for s in p.prod[r]:
            if s >= 0:
                nu[r, s] += 1
    return nu


def _full_matrix(p, o, n, dt):
    """I/dt - J with the photolysis rates differentiated, assembled here from the block Jacobian
    and the rate derivative (each pinned on its own)."""
    from tests.helpers import full_matrix
    A, lo, up = o.jacobian(n, dt)
    M = full_matrix(A, lo, up)
    dk = o.photolysis_dn(n)                       # [L*Rph, L*S]
    nu = _stoich(p)
    L, S = p.L, p.S
    for r in np.flatnonzero(p.rtype == synth.RX_PHOTO):
        q, a = p.prow[r], p.reac[r, 0]
        for k in range(L):
            g = n[k, a] * dk[k * p.Rph + q]       # d w_r,k / dn through k_ph
            for y in np.flatnonzero(nu[r]):
                M[k * S + y] -= nu[r, y] * g
    return M


def test_photolysis_rate_derivative_is_the_finite_difference():
    p, o, n = _relaxed_small()
    dk = o.photolysis_dn(n)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(n.shape) * n
        eps = 1e-6
        fd = ((o.photolysis(n + eps * v) - o.photolysis(n - eps * v)) / (2 * eps)).ravel()
        an = dk @ v.ravel()
        assert np.max(np.abs(fd - an)) < 1e-7 * np.max(np.abs(an))
    # a species absorbs only for the layers at and below it
    k = p.L // 2
    row = dk[k * p.Rph].reshape(p.L, p.S)
    assert np.all(row[:k] == 0.0) and np.any(row[k + 1:] != 0.0)


def test_coupled_jacobian_is_the_finite_difference_of_the_residual():
    """(I/dt - M) v with the photolysis coupling equals the central difference of F along v with the
    rates re-evaluated at the perturbed states."""
    p, o, n = _relaxed_small()
    dt = 1.0
    M = _full_matrix(p, o, n, dt)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(n.shape) * n
    eps = 1e-7
    fd = (o.residual(n + eps * v) - o.residual(n - eps * v)).ravel() / (2 * eps)
    Jv = (v.ravel() / dt) - M @ v.ravel()
    scale = np.abs(fd) + np.abs(Jv) + 1e-300
    big = scale > 1e-6 * scale.max()
    assert np.max(np.abs(fd - Jv)[big] / scale[big]) < 1e-4


def test_coupled_step_solves_the_full_system():
    """The oracle's coupled step is the dense solve of the system assembled above (a numpy solve),
    and differs from the lagged step by far more than the solve's error."""
    p, o, n = _relaxed_small()
    ngas = o.grid()[0]
    s = np.maximum(n, 1e-20 * ngas[:, None])
    dt = 1.0
    M = _full_matrix(p, o, n, dt)
    F = o.residual(n).ravel()
    ref = np.linalg.solve(M, F).reshape(n.shape)
    d = o.step_delta_coupled(n, dt)
    assert np.max(np.abs(d - ref) / s) < 1e-8
    lag = o.step_delta(n, dt)
    assert np.max(np.abs(lag - d) / s) > 1e-4
