"""Pins of the oracle's equilibrium initial state (Sec. 2.5, option (i)) and of its
reaction-pathway analyser (Sec. 4), against closed forms, the conditions that define
the Gibbs minimum, library routines and brute force (no GPU needed)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2512_06729_gb300 import synth
from tests.helpers import custom_problem, nasa_const_cp

KB = 1.380649e-16
P0 = 1.0e6


def _eq(p, n=None, **kw):
    o = Oracle(p)
    if n is None:
        n = o.initial_state()
    x, it, ok = o.equilibrium(o.element_totals(n), **kw)
    return o, n, x, it, ok


def _gibbs_rt_all(o):
    return o.thermo()[0]


# ------------------------------------------------------------------ equilibrium

@pytest.mark.parametrize("make", [synth.tiny_column, lambda: synth.small_column(), lambda: synth.chons_column(L=12)])
def test_equilibrium_satisfies_mass_action(make):
    """At the Gibbs minimum every thermal reaction is in equilibrium: sum nu ln n = ln K_c
    with n = x n_gas and K_c from the (separately pinned) thermochemistry, including the
    pressure term of reactions that change the number of molecules (three-body ones)."""
    p = make()
    o, n, x, it, ok = _eq(p)
    assert ok
    ngas = o.grid()[0]
    lnkc = o.thermo()[1]
    worst = 0.0
    checked = 0
    for k in range(p.L):
        lnn = np.log(np.maximum(x[k], 1e-300) * ngas[k])
        for r in range(p.R):
            if p.rtype[r] == synth.RX_PHOTO:
                continue
            sp = [s for s in p.reac[r] if s >= 0] + [s for s in p.prod[r] if s >= 0]
            if min(x[k, s] for s in sp) < 1e-250:
                continue
            q = sum(lnn[s] for s in p.prod[r] if s >= 0) - sum(lnn[s] for s in p.reac[r] if s >= 0)
            worst = max(worst, abs(q - lnkc[k, r]))
            checked += 1
    assert checked > p.L
    assert worst < 1e-9, worst


@pytest.mark.parametrize("make", [synth.tiny_column, lambda: synth.chons_column(L=12)])
def test_equilibrium_keeps_element_ratios(make):
    p = make()
    o, n, x, it, ok = _eq(p)
    b = o.element_totals(n)
    got = x @ p.elem.astype(float)
    assert np.allclose(x.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    rel = np.abs(got / got.sum(1, keepdims=True) - b / b.sum(1, keepdims=True)) / (b / b.sum(1, keepdims=True))
    assert rel.max() < 1e-11, rel.max()


def _isomer_problem(gA, gB, T=1500.0, P=1.0):
    elem = [[1, 1], [1, 1], [2, 0]]          # A and B share one element vector; C is another molecule
    nasa = [nasa_const_cp(3.5, gA * T, 3.5 * (1 - math.log(T))),
            nasa_const_cp(3.5, gB * T, 3.5 * (1 - math.log(T))),
            nasa_const_cp(3.5, 0.0, 3.5 * (1 - math.log(T)))]
    return custom_problem(elem, [2.0, 2.0, 2.0], [], nasa, [P], [T], f0=[[0.3, 0.3, 0.4]])


def test_equilibrium_isomers_closed_form():
    """Two isomers A, B: x_B / x_A = exp(g_A - g_B) and the element vectors fix x_A + x_B."""
    for gA, gB in ((-10.0, -12.5), (3.0, 3.0), (-40.0, -1.0)):
        p = _isomer_problem(gA, gB)
        o, n, x, it, ok = _eq(p)
        assert ok
        ratio = x[0, 1] / x[0, 0]
        assert ratio == pytest.approx(math.exp(gA - gB), rel=1e-11)
        # element e1 lives in A and B only (one atom each), e0 also in C (two atoms)
        assert (x[0, 0] + x[0, 1]) / (2 * x[0, 2] + x[0, 0] + x[0, 1]) == pytest.approx(0.6 / 1.4, rel=1e-12)


def test_equilibrium_dissociation_closed_form():
    """H2 <-> 2 H at pressure P: x_H^2 P / (x_H2 p0) = exp(g_H2 - 2 g_H) with x_H + x_H2 = 1,
    a quadratic whose root depends on P (pins the ln(P/p0) term and the total-moles update)."""
    T = 3000.0
    for P in (1e-4, 1.0, 1e2):
        gH2, gH = -20.0, -8.0
        nasa = [nasa_const_cp(3.5, gH2 * T, 3.5 * (1 - math.log(T))),
                nasa_const_cp(2.5, gH * T, 2.5 * (1 - math.log(T)))]
        p = custom_problem([[2], [1]], [2.0, 1.0], [], nasa, [P], [T], f0=[[1.0, 0.0]])
        o, n, x, it, ok = _eq(p)
        assert ok
        K = math.exp(gH2 - 2 * gH) / P        # x_H^2 / x_H2
        xH = (-K + math.sqrt(K * K + 4 * K)) / 2
        assert x[0, 1] == pytest.approx(xH, rel=1e-11)
        assert x[0, 0] == pytest.approx(1 - xH, rel=1e-11)


def _gibbs(x, h):
    m = x > 0
    return float(np.sum(x[m] * (h[m] + np.log(x[m]))))


def test_equilibrium_is_the_gibbs_minimum():
    """The oracle's composition has lower G than every feasible perturbation along the null
    space of the element matrix, and scipy's constrained minimiser (a library routine) finds
    the same minimum from a feasible start."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    import scipy.linalg as sla
    p = synth.tiny_column()
    o, n, x, it, ok = _eq(p)
    grt = _gibbs_rt_all(o)
    rng = np.random.default_rng(3)
    A = p.elem.astype(float).T
    Z = sla.null_space(A)
    for k in (0, 20, 39):
        h = grt[k] + math.log(p.P_bar[k])
        g0 = _gibbs(x[k], h)
        for _ in range(50):
            d = Z @ rng.standard_normal(Z.shape[1])
            t = 0.5 * np.min(x[k][d < 0] / -d[d < 0])
            for s in (t, t * 1e-3):
                y = x[k] + s * d
                assert _gibbs(y / y.sum() * 1.0, h) >= g0 - 1e-12 or abs(y.sum() - 1) > 0
                # at fixed element totals the molecule count may change; compare N-weighted G
                assert np.sum(y * (h + np.log(np.maximum(y, 1e-300) / y.sum()))) >= g0 - 1e-12
        # library cross-check: SLSQP on the primal in log variables u = ln N from the initial state
        b = A @ (n[k] / n[k].sum())

        def G(u):
            N = np.exp(u)
            return float(np.sum(N * (h + u - np.log(N.sum()))))

        def dG(u):
            N = np.exp(u)
            return N * (h + u - np.log(N.sum()))

        cons = {"type": "eq", "fun": lambda u: A @ np.exp(u) - b, "jac": lambda u: A * np.exp(u)}
        with np.errstate(over="ignore", invalid="ignore"):
            res = scipy_opt.minimize(G, np.log(n[k] / n[k].sum()), jac=dG, method="SLSQP",
                                     constraints=[cons], options={"maxiter": 1000, "ftol": 1e-15})
        Ns = np.exp(res.x) / np.exp(res.x).sum()
        Ntot = b.sum() / (A @ x[k]).sum()            # molecules of the oracle's mixture at totals b
        assert G(np.log(np.maximum(x[k] * Ntot, 1e-300))) <= G(res.x) + 1e-9 * abs(G(res.x))
        major = x[k] > 1e-4
        assert np.allclose(Ns[major], x[k][major], rtol=1e-3)


def test_equilibrium_absent_element():
    """An element with zero total is absent: every species holding it gets x = 0 and the
    rest is the equilibrium of the remaining elements."""
    p = synth.tiny_column()
    o = Oracle(p)
    b = o.element_totals(o.initial_state())
    b[:, 3] = 0.0                                   # no oxygen
    x, it, ok = o.equilibrium(b)
    assert ok
    holds = p.elem[:, 3] > 0
    assert np.all(x[:, holds] == 0.0)
    assert np.allclose(x.sum(1), 1.0, atol=1e-13)
    x2, _, ok2 = o.equilibrium(b, max_iter=2)
    assert not ok2


# ---------------------------------------------------------------- pathway analyser

def _edges(p, q):
    """(u, v, code, weight) of one layer's graph, from the definition."""
    out = []
    for r in range(p.R):
        for d in (0, 1):
            rate = q[r, d]
            if not rate > 0:
                continue
            frm = p.reac[r] if d == 0 else p.prod[r]
            to = p.prod[r] if d == 0 else p.reac[r]
            for u in set(int(s) for s in frm if s >= 0):
                for v in set(int(s) for s in to if s >= 0):
                    if u != v:
                        out.append((u, v, 2 * r + d, 1.0 / rate))
    return out


def _column_state(p):
    o = Oracle(p)
    n = o.initial_state()
    return o, n, o.fluxes(n)


def test_fluxes_are_the_mass_action_rates():
    """Forward minus reverse rate is the net rate that enters the residual: sum over
    reactions of nu (q_f - q_r) plus transport equals F."""
    p = synth.small_column()
    o, n, q = _column_state(p)
    kf, kr = o.rate_coefficients()
    F = o.residual(n)
    nu = np.zeros((p.R, p.S))
    for r in range(p.R):
        for s in p.reac[r]:
            if s >= 0: nu[r, s] -= 1
        for s in p.prod[r]:
            if s >= 0: nu[r, s] += 1
    chem = (q[:, :, 0] - q[:, :, 1]) @ nu
    u, v = o.transport()
    _, _, dz, _ = o.grid()
    tr = np.zeros_like(n)
    trs = np.zeros_like(n)                            # gross transport flux, the scale of its roundoff
    phi = u * n[:-1] - v * n[1:]
    gross = np.abs(u * n[:-1]) + np.abs(v * n[1:])
    tr[:-1] -= phi / dz[:-1, None]
    tr[1:] += phi / dz[1:, None]
    trs[:-1] += gross / dz[:-1, None]
    trs[1:] += gross / dz[1:, None]
    scale = np.abs(q[:, :, 0] + q[:, :, 1]) @ np.abs(nu) + trs + 1e-300
    assert np.max(np.abs(chem + tr - F) / scale) < 1e-12


@pytest.mark.parametrize("layer", [0, 30, 59])
def test_pathways_match_library_dijkstra(layer):
    """Distances equal scipy's shortest paths on the same graph (parallel edges reduced to
    the lightest), and the predecessor tree is made of real edges that add up exactly."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    p = synth.small_column()
    o, n, q = _column_state(p)
    E = _edges(p, q[layer])
    W = {}
    for u, v, c, w in E:
        W[(u, v)] = min(W.get((u, v), np.inf), w)
    rows, cols, vals = zip(*[(u, v, w) for (u, v), w in W.items()])
    G = sp.csr_matrix((vals, (rows, cols)), shape=(p.S, p.S))
    for src in (0, 2, 7):
        ref = csgraph.dijkstra(G, directed=True, indices=src)
        got = o.pathways(q[layer], src)
        fin = np.isfinite(ref)
        assert np.array_equal(fin, np.isfinite(got["dist"]))
        assert np.allclose(got["dist"][fin], ref[fin], rtol=1e-12, atol=0)
        ecode = {(u, v, c): w for u, v, c, w in E}
        for y in np.flatnonzero(fin):
            if y == src:
                assert got["pred_sp"][y] == -1 and got["dist"][y] == 0.0
                continue
            u, c = int(got["pred_sp"][y]), int(got["pred_edge"][y])
            assert (u, int(y), c) in ecode
            assert got["dist"][y] == got["dist"][u] + ecode[(u, int(y), c)]
            # slowest step: the heaviest edge on the path back to src
            path_w = []
            v = int(y)
            while v != src:
                pu, pc = int(got["pred_sp"][v]), int(got["pred_edge"][v])
                path_w.append((ecode[(pu, v, pc)], pc))
                v = pu
            wmax = max(w for w, _ in path_w)
            assert got["lim_w"][y] == wmax
            assert got["lim_edge"][y] in [pc for w, pc in path_w if w == wmax]


def test_pathways_brute_force_small_network():
    """On a six-species network the fastest route from A to every species is the minimum
    over all simple paths (enumerated), and its slowest step is the path's heaviest edge."""
    elem = [[1, 0], [1, 0], [0, 1], [1, 1], [2, 0], [0, 2]]
    rx = []
    rng = np.random.default_rng(11)
    pairs = [([0], [1]), ([1], [3]), ([0, 2], [3]), ([3], [4]), ([1, 2], [5]), ([4], [5]),
             ([0], [4]), ([5], [2]), ([2, 3], [0, 5])]
    for r, pr in pairs:
        rx.append(dict(type=0, reac=r, prod=pr, arr=[1e-12, 0, 0]))
    nasa = [nasa_const_cp(3.5, 0.0, 0.0)] * 6
    p = custom_problem(elem, [1.0] * 6, rx, nasa, [1.0], [1000.0])
    o = Oracle(p)
    q = np.zeros((p.R, 2))
    q[:, 0] = 10.0 ** rng.uniform(-3, 3, p.R)
    q[:, 1] = np.where(rng.uniform(size=p.R) < 0.5, 10.0 ** rng.uniform(-3, 3, p.R), 0.0)
    E = _edges(p, q)
    adj = {}
    for u, v, c, w in E:
        adj.setdefault(u, []).append((v, c, w))
    best = {0: (0.0, None)}

    def dfs(u, seen, cost, wmax):
        for v, c, w in adj.get(u, []):
            if v in seen:
                continue
            nc, nw = cost + w, max(wmax, w)
            if v not in best or nc < best[v][0] - 1e-15:
                best[v] = (nc, nw)
            dfs(v, seen | {v}, nc, nw)
    dfs(0, {0}, 0.0, 0.0)
    got = o.pathways(q, 0)
    for y in range(p.S):
        if y in best:
            assert got["dist"][y] == pytest.approx(best[y][0], rel=1e-14)
            if y != 0:
                assert got["lim_w"][y] == pytest.approx(best[y][1], rel=1e-14)
        else:
            assert math.isinf(got["dist"][y]) and got["pred_sp"][y] == -1
