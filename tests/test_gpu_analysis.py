"""Parity of the equilibrium initial state (Sec. 2.5) and of the reaction-pathway analyser
(Sec. 4) on the GPU, through the C-ABI, with the FP64 CPU oracle.

Tolerances:
  - equilibrium mole fractions: 1e-9 relative on every species above 1e-250 (the problem has one
    solution; both sides converge it to ~1e-13 in the element potentials, and a species' relative
    error is the potentials' error times its atom count);
  - reaction rates: 1e-11 relative (as the rate coefficients they are made of);
  - pathways on the same rates: bit for bit (IEEE division and addition in the same order on both
    sides, the same tie-breaking rules), distances, predecessor trees and slowest steps alike.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle
from paper_2512_06729_gb300 import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import xk  # noqa: E402

xkbuild.build()


def cpu(t):
    return t.detach().cpu().numpy()


def dev(a, dtype=np.float64):
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


PROBLEMS = {
    "tiny": lambda: synth.tiny_column(),
    "small": lambda: synth.small_column(),
    "chons": lambda: synth.chons_column(),
    "full": lambda: synth.full_column(),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    o = Oracle(p)
    c = xk.Column(p, "fp64")
    n = o.initial_state()
    c.set_state(n)
    yield p, o, c, n
    c.close()


def _rel_eq(x, ref):
    m = ref > 1e-250
    assert np.array_equal(x == 0.0, ref == 0.0)
    return float(np.max(np.abs(x[m] - ref[m]) / ref[m]))


def test_equilibrium_matches_oracle(case):
    p, o, c, n = case
    ref, it_ref, ok = o.equilibrium(o.element_totals(n))
    assert ok
    x, info = c.equilibrium()                       # element totals from the state
    assert info.layers_not_converged == 0 and info.layers_singular == 0
    assert _rel_eq(cpu(x), ref) < 1e-9
    # the same with explicit totals, and the state set to x n_gas
    b = dev(o.element_totals(n))
    x2, _ = c.equilibrium(b, set_state=True)
    assert _rel_eq(cpu(x2), ref) < 1e-9
    ngas = o.grid()[0]
    st = c.get_state()
    assert np.allclose(st, cpu(x2) * ngas[:, None], rtol=1e-15, atol=0)
    c.set_state(n)


def test_equilibrium_absent_element_and_errors():
    p = synth.small_column()
    o = Oracle(p)
    c = xk.Column(p, "fp64")
    n = o.initial_state()
    c.set_state(n)
    b = o.element_totals(n)
    b[:, 4] = 0.0                                    # nitrogen absent
    ref, _, ok = o.equilibrium(b)
    assert ok
    x, info = c.equilibrium(dev(b))
    assert _rel_eq(cpu(x), ref) < 1e-9
    assert np.all(cpu(x)[:, p.elem[:, 4] > 0] == 0.0)
    with pytest.raises(xk.XkError) as e:
        c.equilibrium(dev(b), max_iter=2)
    assert e.value.code == -3
    with pytest.raises(xk.XkError):
        c.equilibrium(dev(b), tol=0.0)
    # the context stays usable
    x3, _ = c.equilibrium(dev(b))
    assert _rel_eq(cpu(x3), ref) < 1e-9
    c.close()


def test_reaction_fluxes_match_oracle(case):
    p, o, c, n = case
    q = cpu(c.reaction_fluxes(dev(n)))
    ref = o.fluxes(n)
    m = ref > 0
    assert np.array_equal(q > 0, m)
    assert np.max(np.abs(q[m] - ref[m]) / ref[m]) < 1e-11


def test_pathways_bitwise_on_the_same_rates(case):
    p, o, c, n = case
    q = o.fluxes(n)
    srcs = [0, 2, p.S - 1] if p.S < 200 else [2, 7]
    layers = range(p.L) if p.S < 200 else [0, 37, 75, 112, 149]
    got = {k: cpu(v) for k, v in c.pathways(dev(q), srcs).items()}
    for j, s in enumerate(srcs):
        for k in layers:
            ref = o.pathways(q[k], s)
            for key in ("dist", "pred_sp", "pred_edge", "lim_edge", "lim_w"):
                assert np.array_equal(got[key][j, k], ref[key]), (s, k, key)


def test_pathways_tree_on_device_rates(case):
    """On the GPU's own rates: every tree edge is a real reaction edge and the distances add
    up exactly along it; unreachable species have no predecessor."""
    p, o, c, n = case
    qd = c.reaction_fluxes(dev(n))
    q = cpu(qd)
    got = {k: cpu(v) for k, v in c.pathways(qd, [2]).items()}
    dist, pred, edge = got["dist"][0], got["pred_sp"][0], got["pred_edge"][0]
    for k in (0, p.L // 2, p.L - 1):
        for y in range(p.S):
            if not np.isfinite(dist[k, y]):
                assert pred[k, y] == -1
                continue
            if y == 2:
                assert dist[k, y] == 0.0
                continue
            u, e = int(pred[k, y]), int(edge[k, y])
            r, d = divmod(e, 2)
            frm = p.reac[r] if d == 0 else p.prod[r]
            to = p.prod[r] if d == 0 else p.reac[r]
            assert u in frm and y in to and q[k, r, d] > 0
            assert dist[k, y] == dist[k, u] + 1.0 / q[k, r, d]


def test_pathways_reject_bad_sources():
    p = synth.tiny_column()
    c = xk.Column(p, "fp64")
    q = torch.zeros((p.L, p.R, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(xk.XkError):
        c.pathways(q, [p.S])
    with pytest.raises(xk.XkError):
        c.pathways(q, list(range(p.S)) + [0])
    out = c.pathways(q, [1])          # no positive rate: only the source is reached
    d = cpu(out["dist"])[0]
    assert np.all(d[:, 1] == 0.0) and np.all(np.isinf(np.delete(d, 1, axis=1)))
    c.close()
