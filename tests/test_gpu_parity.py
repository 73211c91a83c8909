"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Every row of the implicit step is compared element by element on seeded
inputs: grid, Gibbs energies and ln K_c, rate coefficients, photolysis rates,
transport coefficients, residual, Jacobian blocks, the block-tridiagonal
solve, single linear steps in both precision modes, controlled step
sequences and runs to steady state.

Tolerances (FP64 everywhere except the mixed-precision factorization):
  - quantities computed by the same formula in the same order: 1e-12 relative
    (CUDA exp/log/pow are within 1-2 ulp of the host libm);
  - rate coefficients: 1e-11 relative (exp(-ln K_c) amplifies the ulp error of
    ln K_c, |ln K_c| < 100);
  - residual: 1e-10 of the gross production + loss of each species (F is a
    sum with cancellation);
  - linear steps: 1e-6 of max(n, 1e-20 n_gas) (condition numbers of 1e10 to
    1e16 turn 1e-16 roundoff into this; the two sides pivot differently);
  - end states of runs: 1e-6 relative on species above 1e-20 mixing ratio.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle, default_policy
from paper_2512_06729_gb300 import synth
from tests.helpers import full_matrix, independent_refined_solve, relative_to_state

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import xk  # noqa: E402

xkbuild.build()


def cpu(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


PROBLEMS = {
    "tiny": lambda: synth.tiny_column(),
    "small": lambda: synth.small_column(),
    "chons": lambda: synth.chons_column(),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def pair(request):
    p = PROBLEMS[request.param]()
    return p, Oracle(p), xk.Column(p, "fp64")


def relerr(a, b, floor=0.0):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)) if a.size else 0.0


def test_grid(pair):
    p, o, c = pair
    ng, z, dz, dzi = (cpu(t) for t in c.eval_grid())
    ong, oz, odz, odzi = o.grid()
    assert relerr(ng, ong) < 1e-14
    np.testing.assert_allclose(z, oz, rtol=1e-12, atol=1e-9 * oz.max())
    np.testing.assert_allclose(dz, odz, rtol=1e-11)
    np.testing.assert_allclose(dzi, odzi, rtol=1e-11)


def test_thermo_and_rates(pair):
    p, o, c = pair
    grt, lnkc = (cpu(t) for t in c.eval_thermo())
    ogrt, olnkc = o.thermo()
    assert np.max(np.abs(grt - ogrt) / np.maximum(np.abs(ogrt), 1.0)) < 1e-12
    assert np.max(np.abs(lnkc - olnkc) / np.maximum(np.abs(olnkc), 1.0)) < 1e-12
    kf, kr = (cpu(t) for t in c.eval_rates())
    okf, okr = o.rate_coefficients()
    assert relerr(kf, okf, 1e-300) < 1e-11
    assert relerr(kr, okr, 1e-300) < 1e-11


def test_photolysis(pair):
    p, o, c = pair
    if p.Rph == 0:
        pytest.skip("no photolysis in this network")
    n = o.initial_state()
    kph = cpu(c.eval_photolysis(dev(n)))
    assert relerr(kph, o.photolysis(n), 1e-300) < 1e-12


def test_transport(pair):
    p, o, c = pair
    u, v = (cpu(t) for t in c.eval_transport())
    ou, ov = o.transport()
    assert relerr(u, ou, 1e-300) < 1e-11
    assert relerr(v, ov, 1e-300) < 1e-11


def _gross(p, o, n):
    """Sum over reactions of |nu| (w_f + w_b) per species: the scale of F's cancellation."""
    kf, kr = o.rate_coefficients()
    kph = o.photolysis(n)
    L, S = n.shape
    g = np.zeros((L, S))
    for r in range(p.R):
        if p.rtype[r] == 2:
            f = kph[:, p.prow[r]].copy(); b = np.zeros(L)
        else:
            f = kf[:, r].copy(); b = kr[:, r].copy()
        for s in range(3):
            if p.reac[r, s] >= 0: f = f * n[:, p.reac[r, s]]
            if p.prod[r, s] >= 0: b = b * n[:, p.prod[r, s]]
        for s in range(3):
            for sp in (p.reac[r, s], p.prod[r, s]):
                if sp >= 0: g[:, sp] += np.abs(f) + np.abs(b)
    # transport: the four flux terms of each layer
    if L > 1:
        u, v = o.transport()
        dz = o.grid()[2]
        t = np.zeros((L, S))
        t[:-1] += np.abs(u * n[:-1]) + np.abs(v * n[1:])
        t[1:] += np.abs(u * n[:-1]) + np.abs(v * n[1:])
        g += t / dz[:, None]
    return g


def test_residual(pair):
    p, o, c = pair
    n = o.initial_state()
    F = cpu(c.eval_residual(dev(n)))
    oF = o.residual(n)
    gross = _gross(p, o, n) + np.abs(oF) + 1e-300
    assert np.max(np.abs(F - oF) / gross) < 1e-10


def test_jacobian(pair):
    p, o, c = pair
    n = o.initial_state()
    for dt in (1e-3, 1e6):
        A, lo, up = (cpu(t) for t in c.eval_jacobian(dev(n), dt))
        oA, olo, oup = o.jacobian(n, dt)
        scale = np.abs(oA).max(axis=2, keepdims=True) + 1e-300
        assert np.max(np.abs(A - oA) / scale) < 1e-12
        np.testing.assert_allclose(lo, olo, rtol=1e-11, atol=0)
        np.testing.assert_allclose(up, oup, rtol=1e-11, atol=0)


def test_block_solve_matches_oracle(pair):
    p, o, c = pair
    n = o.initial_state()
    rng = np.random.default_rng(0)
    f = rng.normal(size=n.shape) * n
    for dt in (1e-6, 1e-2):
        oA, olo, oup = o.jacobian(n, dt)
        x = cpu(c.block_solve(dev(oA), dev(olo), dev(oup), dev(f)))
        ox = o.block_solve(oA, olo, oup, f)
        scale = np.abs(ox).max() + 1e-300
        assert np.max(np.abs(x - ox)) / scale < 1e-10


def test_block_solve_late_state_large_dt(pair):
    """Near steady state at dt = dt_max = 1e8 s the block system has condition
    numbers near 1e16, so two FP64 solvers that pivot differently (scaled
    explicit inverses here, unscaled LU in the oracle) can differ by up to
    kappa * eps ~ 1e-4 of the solution in the ill-determined directions; the
    bound below is that.  Trajectory parity over many such steps is checked
    separately (the backward-Euler map contracts those differences)."""
    p, o, c = pair
    if p.L * p.S > 4000:
        pytest.skip("late state is prepared only for the small columns")
    ng = o.grid()[0]
    n, _ = o.run_to_steady(o.initial_state(), max_steps=400)
    oA, olo, oup = o.jacobian(n, 1e8)
    f = o.residual(n)
    x = cpu(c.block_solve(dev(oA), dev(olo), dev(oup), dev(f)))
    ox = o.block_solve(oA, olo, oup, f)
    s = np.maximum(n, 1e-20 * ng[:, None])
    assert np.max(np.abs(x - ox) / s) < 1e-4


@pytest.mark.parametrize("panel,nb,twisted", [(1, 8, 0), (1, 16, 0), (1, 32, 0), (0, 8, 1), (0, 8, 0), (0, 16, 1)])
def test_fp64_factor_variants(panel, nb, twisted):
    """FP64 block inversion with each panel's pivots chosen first and its
    multipliers formed on all CTAs by triangular solves (panel = 1; widths 8,
    16, 32 with ragged last panels on 40 species) and column by column on one
    CTA (panel = 0; top-down, or from both ends on the two halves of the grid
    meeting in the middle layer, with the matching two-cluster sweeps): the
    direct solve against the oracle's LU at moderate dt to 1e-10; and near
    steady state at dt = 1e8 s, where the system's condition number is near
    1e16, the FP64 path's step (FGMRES refinement around each variant's
    factorization) against the oracle's step, every width held to the bound
    that an independent FP64 solve of the same system sets."""
    p = synth.small_column()
    o = Oracle(p)
    c = xk.Column(p, "fp64", fp64_panel=panel, panel_width=nb, twisted=twisted)
    n = o.initial_state()
    rng = np.random.default_rng(4)
    f = rng.normal(size=n.shape) * n
    for dt in (1e-6, 1e-2):
        oA, olo, oup = o.jacobian(n, dt)
        x = cpu(c.block_solve(dev(oA), dev(olo), dev(oup), dev(f)))
        ox = o.block_solve(oA, olo, oup, f)
        assert np.max(np.abs(x - ox)) / (np.abs(ox).max() + 1e-300) < 1e-10, (panel, nb, dt)
    nl, _ = o.run_to_steady(n, max_steps=400)
    d, iters, res = c.step_delta(dev(nl), 1e8)
    bound, errs, spread = _step_parity(o, nl, 1e8, {"fp64": cpu(d)})
    assert errs["fp64"] <= bound, (panel, nb, twisted, errs, bound, spread, iters, res)


def test_fp64_factor_full_size():
    """Both FP64 inversions at 594 species (74 panels of 8 and a ragged one of
    2) on a 4-layer slice of the 7,720-reaction column, against the oracle's
    LU."""
    p = synth.full_column()
    p = p.replace(P_bar=p.P_bar[:4].copy(), T=p.T[:4].copy(), Kzz=p.Kzz[:4].copy(), f0=p.f0[:4].copy())
    o = Oracle(p)
    n = o.initial_state()
    f = np.random.default_rng(5).normal(size=n.shape) * n
    for panel, twisted in ((0, 1), (0, 0), (1, 0)):
        c = xk.Column(p, "fp64", fp64_panel=panel, twisted=twisted)
        for dt in (1e-6, 1e-2):
            oA, olo, oup = o.jacobian(n, dt)
            x = cpu(c.block_solve(dev(oA), dev(olo), dev(oup), dev(f)))
            ox = o.block_solve(oA, olo, oup, f)
            assert np.max(np.abs(x - ox)) / (np.abs(ox).max() + 1e-300) < 1e-10, (panel, twisted, dt)
        c.close()


@pytest.mark.parametrize("pivoting,cluster,nb,twisted,bcr", [(0, 0, 0, 1, 0), (0, 0, 0, 0, 0), (0, 2, 16, 1, 0),
                                                              (0, 3, 16, 1, 0), (0, 4, 8, 0, 0), (0, 1, 8, 1, 0),
                                                              (0, -1, 0, 1, 0), (1, 0, 0, 1, 0), (0, 0, 0, 1, 1)])
def test_fp32_block_solve(pivoting, cluster, nb, twisted, bcr):
    """The FP32 block inversion (the mixed path's preconditioner) on the scaled
    system diag(1/s) A diag(s), against the oracle's FP64 solve of the same
    system: cluster-resident kernel (automatic size and panel width 8, eliminated
    from both ends of the column on two clusters or top-down on one; 2 and 4
    CTAs holding several panels each; 3 CTAs with one 16-wide panel each, the
    last one ragged; one-CTA clusters), the grid-wide kernel without
    pivoting, and with pivoting; and the block cyclic reduction on the tensor
    cores (bcr = 1: leaf blocks pivoted, the rest without pivoting).
    The bound is FP32 rounding (6e-8) times the condition number of the scaled
    system (about 1e3 at dt = 1e-6 s and 1e5 at dt = 1e-2 s on this column),
    with a margin; without pivoting the element growth adds to it at
    dt = 1e-2 s (the same elimination emulated in numpy float32, with exact
    diagonal-block inverses, errs by 1.5e-2 / 1.0e-2 / 1.6e-3 for panels of
    8 / 16 / 32 columns), so the no-pivot variants get 3e-2 there.  An indexing
    error gives O(1); the dt = 1e-6 s case stays at 1e-4.  The reduction's
    products round to about 3 * 2^-22 per step (TF32 head and tail), a dozen
    FP32 units, so its bound at dt = 1e-6 s is 12x that."""
    p = synth.small_column()
    o = Oracle(p)
    c = xk.Column(p, "mixed", fp32_pivoting=pivoting, cluster_size=cluster, panel_width=nb, twisted=twisted,
                  fp32_bcr=bcr)
    ng = o.grid()[0]
    n = o.initial_state()
    s = np.maximum(n, 1e-20 * ng[:, None])
    rng = np.random.default_rng(2)
    for dt, tol in ((1e-6, 1.2e-3 if bcr else 1e-4), (1e-2, 1e-2 if pivoting else 3e-2)):
        A, lo, up = o.jacobian(n, dt)
        As = A * s[:, None, :] / s[:, :, None]
        los = lo * np.vstack([s[:1], s[:-1]]) / s
        ups = up * np.vstack([s[1:], s[-1:]]) / s
        f = rng.normal(size=n.shape)
        x = cpu(c.block_solve32(dev(As), dev(los), dev(ups), dev(f)))
        ox = o.block_solve(As, los, ups, f)
        err = np.max(np.abs(x - ox)) / np.max(np.abs(ox))
        assert err < tol, (pivoting, dt, err)


def test_fp32_cluster_full_size():
    """The cluster-resident FP32 inversion at the full 594-species block size
    (several panels per CTA, ragged last panel of 2 columns) on a 4-layer slice
    of the 7,720-reaction column (eliminated from both ends, meeting in layer
    2, and top-down), against the oracle's FP64 solve; and the grid-wide FP32
    kernel and the block cyclic reduction on the tensor cores on the same
    system (bound 12x the FP32 one: its products round to a dozen FP32
    units)."""
    p = synth.full_column()
    p = p.replace(P_bar=p.P_bar[:4].copy(), T=p.T[:4].copy(), Kzz=p.Kzz[:4].copy(), f0=p.f0[:4].copy())
    o = Oracle(p)
    ng = o.grid()[0]
    n = o.initial_state()
    s = np.maximum(n, 1e-20 * ng[:, None])
    A, lo, up = o.jacobian(n, 1e-6)
    As = A * s[:, None, :] / s[:, :, None]
    los = lo * np.vstack([s[:1], s[:-1]]) / s
    ups = up * np.vstack([s[1:], s[-1:]]) / s
    f = np.random.default_rng(3).normal(size=n.shape)
    ox = o.block_solve(As, los, ups, f)
    errs = {}
    for cluster, twisted, bcr in ((0, 1, 0), (0, 0, 0), (-1, 1, 0), (0, 1, 1)):
        c = xk.Column(p, "mixed", cluster_size=cluster, twisted=twisted, fp32_bcr=bcr)
        x = cpu(c.block_solve32(dev(As), dev(los), dev(ups), dev(f)))
        errs[(cluster, twisted, bcr)] = np.max(np.abs(x - ox)) / np.max(np.abs(ox))
        c.close()
    assert all(e < (1.2e-3 if k[2] else 1e-4) for k, e in errs.items()), errs


@pytest.mark.parametrize("precision,kw", [("fp64", {}), ("mixed", {}), ("mixed", {"fp32_bcr": 0, "twisted": 0}),
                                          ("mixed", {"fp32_bcr": 0, "cluster_size": -1}),
                                          ("mixed", {"fp32_bcr": 0, "fp32_pivoting": 1}), ("mixed", {"fp32_bcr": 0})])
def test_step_delta(precision, kw):
    """One linear step at the initial state (small dt) and at a late state
    (the dt the controller reached there), against the oracle.  In mixed
    precision (block cyclic reduction on the tensor cores, the default; the
    cluster-resident FP32 inversion, top-down or twisted; grid-wide without
    and with pivoting) FGMRES must converge on the FP32 preconditioner at the
    initial state (iters >= 0: no FP64 fallback)."""
    p = synth.small_column()
    o = Oracle(p)
    c = xk.Column(p, precision, **kw)
    ng = o.grid()[0]
    n0 = o.initial_state()
    nl, info = o.run_to_steady(n0, max_steps=500)
    for i, (n, dt) in enumerate(((n0, 1e-6), (n0, 1e-2), (nl, info.dt))):
        d, iters, res = c.step_delta(dev(n), dt)
        d = cpu(d)
        od = o.step_delta(n, dt)
        s = np.maximum(n, 1e-20 * ng[:, None])
        err = np.max(np.abs(d - od) / s)
        assert err < 1e-6, (precision, kw, dt, err, iters, res)
        if precision == "mixed" and i < 2:
            assert iters >= 0, (kw, dt, iters, res)


def test_controlled_steps_follow_the_oracle():
    p = synth.tiny_column()
    o = Oracle(p)
    c = xk.Column(p, "fp64")
    ng = o.grid()[0]
    n = o.initial_state()
    c.set_mixing_ratios(p.f0)
    np.testing.assert_allclose(c.get_state(), n, rtol=1e-15)
    dt = 1e-8
    pol = default_policy()
    for it in range(60):
        info = c.step(dt)
        n, oinfo = o.step(n, dt, pol)
        assert info.accepted == oinfo.accepted
        assert info.dt_next == pytest.approx(oinfo.dt_next, rel=1e-6)
        m = c.get_state()
        s = np.maximum(n, 1e-20 * ng[:, None])
        assert np.max(np.abs(m - n) / s) < 1e-8
        dt = oinfo.dt_next


def _oracle_schedule(o, n, steps):
    """dt of every accepted step of the oracle's own controlled run."""
    dts, dt = [], 1e-8
    for _ in range(steps):
        n, info = o.step(n, dt)
        if info.accepted:
            dts.append(dt)
        dt = info.dt_next
    return dts


def _replay(p, precision, dts, **kw):
    """Replay dts on both sides with every step accepted; per step, the worst
    relative difference over species above 1e-12 and over those between 1e-20
    and 1e-12 mixing ratio."""
    o = Oracle(p)
    ng = o.grid()[0]
    loose = dict(rel_reject=1e300, neg_tol=1e300)
    pol = default_policy(**loose)
    c = xk.Column(p, precision, **loose, **kw)
    c.set_mixing_ratios(p.f0)
    n = o.initial_state()
    out = []
    for dt in dts:
        info = c.step(dt)
        n, oinfo = o.step(n, dt, pol)
        assert info.accepted == 1 and oinfo.accepted == 1
        m = c.get_state()
        rel = np.abs(m - n) / np.maximum(n, 1e-300)
        major = n > 1e-12 * ng[:, None]
        trace = (n > 1e-20 * ng[:, None]) & ~major
        out.append((float(rel[major].max()), float(rel[trace].max()) if trace.any() else 0.0))
    return np.array(out)


@pytest.mark.parametrize("precision,kw", [("fp64", {}), ("mixed", {}), ("mixed", {"fp32_bcr": 0})])
def test_replayed_schedule_small_column(precision, kw):
    """The oracle's own controlled dt sequence on the 40-species, 60-layer
    column (1e-8 s up to dt_max = 1e8 s), replayed by both sides with every
    step accepted: within 1e-6 on every species above 1e-20, every step."""
    p = synth.small_column()
    dts = _oracle_schedule(Oracle(p), Oracle(p).initial_state(), 700)
    assert dts[-1] >= 1e7
    err = _replay(p, precision, dts, **kw)
    assert err.max() <= 1e-6, err.max(axis=0)


def _second_trajectory(p, dts):
    """The oracle's replayed schedule taken a second time on the CPU with the
    linear solves done by independent_refined_solve (the oracle's residual and
    Jacobian, a solver that shares no code with it); per step, the worst
    relative difference from the oracle's own trajectory over species above
    1e-12 and between 1e-20 and 1e-12 mixing ratio: how far FP64 alone lets
    two correct trajectories drift."""
    o = Oracle(p)
    ng = o.grid()[0]
    pol = default_policy(rel_reject=1e300, neg_tol=1e300)
    n = o.initial_state()
    m = n.copy()
    out = []
    for dt in dts:
        n, _ = o.step(n, dt, pol)
        A, lo, up = o.jacobian(m, dt)
        F = o.residual(m)
        s = np.maximum(m, 1e-20 * ng[:, None])
        m = np.maximum(m + independent_refined_solve(A, lo, up, F, s), 0.0)
        rel = np.abs(m - n) / np.maximum(n, 1e-300)
        major = n > 1e-12 * ng[:, None]
        trace = (n > 1e-20 * ng[:, None]) & ~major
        out.append((float(rel[major].max()), float(rel[trace].max()) if trace.any() else 0.0))
    return np.array(out)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_replayed_schedule_tiny_column(precision):
    """The same on the 20-species column, whose late steps (up to dt = 1e8 s)
    have species relaxing on 1e13 s time scales that FP64 no longer pins
    down.  Every step is held to 1e-6 or, where FP64 itself cannot tell two
    correct trajectories apart that closely, to 10x the drift between the
    oracle's trajectory and a second CPU trajectory with an independent
    solver (largest drift so far, per class of species)."""
    p = synth.tiny_column()
    dts = _oracle_schedule(Oracle(p), Oracle(p).initial_state(), 900)
    assert dts[-1] >= 1e8
    err = _replay(p, precision, dts)
    drift = np.maximum.accumulate(_second_trajectory(p, dts), axis=0)
    bound = np.maximum(1e-6, 10.0 * drift)
    worst = np.argmax((err / bound).max(axis=1))
    assert (err <= bound).all(), (worst, dts[worst], err[worst], drift[worst])


@pytest.mark.parametrize("precision,reuse,bcr", [("fp64", 0, 0), ("mixed", 0, 0), ("mixed", 1, 0), ("mixed", 1, 1)])
def test_run_to_steady_matches_oracle(precision, reuse, bcr):
    """Adaptive run to the steady-state test on the 40-species column; both
    sides reach the same state within 1e-6 on species above 1e-20 (also with
    the FP64 factorization reused as FGMRES preconditioner)."""
    p = synth.small_column()
    o = Oracle(p)
    ng = o.grid()[0]
    on, oinfo = o.run_to_steady(o.initial_state(), dt0=1e-8, max_steps=6000)
    assert oinfo.converged
    c = xk.Column(p, precision, reuse_factorization=reuse, fp32_bcr=bcr)
    c.set_mixing_ratios(p.f0)
    info = c.run_to_steady(1e-8, 6000)
    assert info.converged
    n = c.get_state()
    mask = on > 1e-20 * ng[:, None]
    err = np.max(np.abs(n[mask] - on[mask]) / on[mask])
    assert err <= 1e-6, (err, info.steps, oinfo.steps)


def test_single_layer_and_no_photolysis_edge_cases():
    p = synth.tiny_column()
    p1 = p.replace(P_bar=p.P_bar[:1], T=p.T[:1], Kzz=p.Kzz[:1], f0=p.f0[:1])
    o = Oracle(p1)
    c = xk.Column(p1, "fp64")
    n = o.initial_state()
    d, _, _ = c.step_delta(dev(n), 1e-4)
    np.testing.assert_allclose(cpu(d), o.step_delta(n, 1e-4), rtol=1e-9, atol=1e-12 * n.max())
    F = cpu(c.eval_residual(dev(n)))
    oF = o.residual(n)
    assert np.max(np.abs(F - oF) / (_gross(p1, o, n) + 1e-300)) < 1e-10


def test_invalid_inputs_raise():
    p = synth.tiny_column()
    bad = p.replace(reac=p.reac.copy())
    bad.reac[3, 0] = p.S + 5
    with pytest.raises(xk.XkError):
        xk.Column(bad, "fp64")
    bad = p.replace(P_bar=p.P_bar[::-1].copy())
    with pytest.raises(xk.XkError):
        xk.Column(bad, "fp64")


def test_rate_coefficients_evaluated_once():
    """Rate coefficients depend on the atmosphere only: a column that sets them
    explicitly and one that evaluates them lazily in its first step take the
    same steps, bit for bit, and the device values equal a fresh evaluation."""
    p = synth.tiny_column()
    a, b = xk.Column(p, "fp64"), xk.Column(p, "fp64")
    a.set_rate_coefficients()
    for c in (a, b):
        c.set_mixing_ratios(p.f0)
    dt = 1e-8
    for _ in range(10):
        ia, ib = a.step(dt), b.step(dt)
        assert ia.accepted == ib.accepted and ia.dt_next == ib.dt_next
        dt = ia.dt_next
    assert np.array_equal(a.get_state(), b.get_state())
    kf, kr = (cpu(t) for t in a.eval_rates())
    o = Oracle(p)
    okf, okr = o.rate_coefficients()
    assert relerr(kf, okf, 1e-300) < 1e-11 and relerr(kr, okr, 1e-300) < 1e-11


def _step_parity(o, n, dt, deltas):
    """Each delta in `deltas` against the oracle's step, relative to n on the
    species above 1e-20 mixing ratio, with the bound derived here from a
    second FP64 solve of the same system that shares no code with the oracle
    (LAPACK block Thomas in relative variables plus refinement): FP64 itself
    determines the step only to within the disagreement of the two, so a
    result within 10x that of the oracle (and never held to less than 1e-9)
    is as close as FP64 can tell.  Returns (bound, errors, reference spread)."""
    ng = o.grid()[0]
    od = o.step_delta(n, dt)
    A, lo, up = o.jacobian(n, dt)
    F = o.residual(n)
    s = np.maximum(n, 1e-20 * ng[:, None])
    x2 = independent_refined_solve(A, lo, up, F, s)
    spread = relative_to_state(x2, od, n, ng)
    bound = max(10.0 * spread, 1e-9)
    errs = {k: relative_to_state(d, od, n, ng) for k, d in deltas.items()}
    return bound, errs, spread


def test_full_size_column():
    """The 594-species, 7,720-reaction, 150-layer column at the bench's launch
    configuration (library defaults: FP32 block cyclic reduction on the tensor
    cores, twisted FP64 inversion, FGMRES refinement in both paths): rate
    coefficients, photolysis and the residual at the initial state element by
    element against the oracle; Jacobian blocks of three layers; and the
    mixed and FP64 linear steps at dt = 1e-6 s and 1e-2 s element by element
    against the oracle's step, relative to n on every species above 1e-20
    mixing ratio, within the bound that a second, independent FP64 solve of
    the same system sets (see _step_parity)."""
    p = synth.full_column()
    o = Oracle(p)
    n = o.initial_state()
    c = xk.Column(p, "mixed")
    kf, kr = (cpu(t) for t in c.eval_rates())
    okf, okr = o.rate_coefficients()
    assert relerr(kf, okf, 1e-300) < 1e-11 and relerr(kr, okr, 1e-300) < 1e-11
    kph = cpu(c.eval_photolysis(dev(n)))
    assert relerr(kph, o.photolysis(n), 1e-300) < 1e-11
    F = cpu(c.eval_residual(dev(n)))
    oF = o.residual(n)
    gross = _gross(p, o, n) + np.abs(oF) + 1e-300
    assert np.max(np.abs(F - oF) / gross) < 1e-10
    oA = o.jacobian(n, 1e-2)[0]
    A = c.eval_jacobian(dev(n), 1e-2)[0]
    for k in (0, 75, 149):
        Ak = cpu(A[k])
        scale = np.abs(oA[k]).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(Ak - oA[k]) / scale) < 1e-12, k
    del A, oA
    f64 = xk.Column(p, "fp64")
    for dt in (1e-6, 1e-2):
        deltas, info = {}, {}
        for prec, col in (("mixed", c), ("fp64", f64)):
            d, iters, res = col.step_delta(dev(n), dt)
            deltas[prec] = cpu(d)
            info[prec] = (iters, res)
            assert np.isfinite(deltas[prec]).all(), prec
        bound, errs, spread = _step_parity(o, n, dt, deltas)
        print(f"full size dt={dt:g}: errors vs oracle {errs}, independent FP64 spread {spread:.3e}, solver {info}")
        for prec, e in errs.items():
            assert e <= bound, (dt, prec, e, bound, spread, info[prec])
    f64.close()
    c.close()
