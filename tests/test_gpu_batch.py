"""Batches of columns (continuous batching): each column's result in a
batch equals its result alone, admission respects the HBM budget, and the
serving loop returns the same steady states as solving each request alone.
Tolerance 1e-9 relative on species above 1e-20 mixing ratio: the FP64 path
reproduces bit for bit; the mixed path differs only in the last bits of the
FP32 preconditioner's rounding (7.6e-12 measured)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import serving, synth, xk  # noqa: E402

xkbuild.build()


def _problems():
    return [synth.tiny_column(), synth.small_column(),
            synth.small_column(S=30, L=45, n_two=80, n_three=20, n_photo=6, seed=9, W=120),
            synth.sweep_column(96, 40, 1500.0, 3.0, 0.5, seed=4)]


def _alone(p, precision, steps, initial="user", **kw):
    c = xk.Column(p, precision, **kw)
    c.set_mixing_ratios(p.f0)
    if initial == "equilibrium":
        c.equilibrium(set_state=True)
    info = c.run_to_steady(1e-8, steps)
    return c.get_state(), info


@pytest.mark.parametrize("precision,largest_first", [("fp64", False), ("mixed", False), ("mixed", True),
                                                     ("fp64", True)])
def test_batch_results_equal_alone(precision, largest_first):
    """Columns of 20 to 96 species stepped together; created largest first, the
    last-planned (smallest) column must not shrink the shared-memory limit the
    others' kernels launch with."""
    probs = _problems()
    if largest_first:
        probs = probs[::-1]
    b = xk.Batch(64 << 30, 8)
    cols, slots = [], []
    for p in probs:
        c = xk.Column(p, precision)
        c.set_mixing_ratios(p.f0)
        slots.append(b.add(c, 1e-8))
        cols.append(c)
    assert None not in slots
    for _ in range(400):
        b.step(8)
        if all(b.poll(s)[1] for s in slots):
            break
    for p, c, s in zip(probs, cols, slots):
        info, finished, status = b.poll(s)
        assert finished and status == 0
        n_batch = b.remove(s).get_state()
        n_alone, ainfo = _alone(p, precision, info.steps)
        assert ainfo.steps == info.steps
        ng = n_alone.max(axis=1, keepdims=True)
        mask = n_alone > 1e-20 * ng
        err = np.max(np.abs(n_batch[mask] - n_alone[mask]) / n_alone[mask])
        assert err <= 1e-9, (p.name, err)
    b.close()


def test_batch_admission_by_footprint():
    p = synth.small_column()
    c1 = xk.Column(p, "fp64")
    c2 = xk.Column(p, "fp64", allocate=False)
    assert c2.ws is None and c2.workspace_bytes == c1.workspace_bytes   # footprint known, nothing allocated
    b = xk.Batch(int(c1.workspace_bytes * 1.5), 4)
    assert b.fits(c2.workspace_bytes)
    s1 = b.add(c1)
    assert s1 is not None
    assert not b.fits(c2.workspace_bytes)  # the second footprint does not fit: checked before allocating
    c2.allocate()
    assert b.add(c2) is None
    b.remove(s1)
    assert b.fits(c2.workspace_bytes)
    assert b.add(c2) is not None          # admitted once the first one left
    b.close()


def test_serving_results_equal_alone():
    reqs = [serving.Request(i, 0.002 * i, p) for i, p in enumerate(_problems())]
    srv = serving.Server(64 << 30, 3, precision="mixed", chunk=8, keep_states=True,
                         column_kw=dict(reuse_factorization=1))
    res = srv.run(reqs)
    srv.close()
    for r, q in zip(res, reqs):
        assert r.converged
        n_alone, info = _alone(q.problem, "mixed", r.steps, reuse_factorization=1)
        assert info.steps == r.steps
        ng = n_alone.max(axis=1, keepdims=True)
        mask = n_alone > 1e-20 * ng
        assert np.max(np.abs(r.state[mask] - n_alone[mask]) / n_alone[mask]) <= 1e-9
        assert r.finished >= r.admitted >= r.arrival - 1e-9
    s = serving.summarize(res, max(r.finished for r in res))
    assert s["requests"] == 4 and s["converged"] == 4 and s["p99_s"] >= s["p50_s"] > 0


def test_serving_from_equilibrium_equals_alone():
    """Requests that start from the chemical-equilibrium composition (computed at admission on the
    device) end where the same column started from it alone ends."""
    reqs = [serving.Request(i, 0.002 * i, p, initial="equilibrium") for i, p in enumerate(_problems()[:3])]
    srv = serving.Server(64 << 30, 2, precision="fp64", chunk=8, keep_states=True)
    res = srv.run(reqs)
    srv.close()
    for r, q in zip(res, reqs):
        assert r.converged
        n_alone, info = _alone(q.problem, "fp64", r.steps, initial="equilibrium")
        assert info.steps == r.steps
        ng = n_alone.max(axis=1, keepdims=True)
        mask = n_alone > 1e-20 * ng
        assert np.max(np.abs(r.state[mask] - n_alone[mask]) / n_alone[mask]) <= 1e-9


def test_batch_submit_query():
    """Asynchronous form: a slot's submitted steps run on its own stream; the
    synchronous step refuses while they are in flight; after query reports
    them done, poll shows exactly that many steps."""
    p = synth.tiny_column()
    b = xk.Batch(8 << 30, 2)
    c = xk.Column(p, "fp64")
    c.set_mixing_ratios(p.f0)
    slot = b.add(c, 1e-8)
    b.submit(slot, 4)
    with pytest.raises(xk.XkError):
        b.submit(slot, 1)
    with pytest.raises(xk.XkError):
        b.step(1)
    while not b.query(slot):
        pass
    info, finished, status = b.poll(slot)
    assert info.steps == 4 and status == 0 and not finished
    b.step(2)
    assert b.poll(slot)[0].steps == 6
    b.close()
