"""Controlled steps replayed from CUDA graphs: a captured chunk of steps gives
the same trajectory as the same kernels launched one by one from the host,
run_to_steady replays one graph per chunk, and a batch round of every
unfinished column is one graph launch.  Same kernels, same plans, same inputs:
the trajectories agree to the last bits (1e-12 relative on species above 1e-20
mixing ratio, equal step counts)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import synth, xk  # noqa: E402

xkbuild.build()


def _close(a, b, tol=1e-12):
    ng = np.abs(b).max(axis=1, keepdims=True)
    mask = np.abs(b) > 1e-20 * ng
    return np.max(np.abs(a[mask] - b[mask]) / np.abs(b[mask]))


def _run(p, precision, use_graphs, steps):
    c = xk.Column(p, precision, use_graphs=use_graphs)
    c.set_mixing_ratios(p.f0)
    g0 = xk.Column.graph_launches()
    info = c.run_to_steady(1e-8, steps)
    return c.get_state(), info, xk.Column.graph_launches() - g0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("steps", [16, 37])
def test_graph_steps_equal_launched_steps(precision, steps):
    """37 steps = two 16-step graphs and a 5-step one (unless steady earlier)."""
    p = synth.small_column()
    n_g, info_g, glaunch = _run(p, precision, 1, steps)
    n_h, info_h, hlaunch = _run(p, precision, 0, steps)
    assert hlaunch == 0
    assert glaunch >= 1
    assert info_g.steps == info_h.steps and info_g.accepted == info_h.accepted
    assert info_g.fp64_steps == info_h.fp64_steps
    assert _close(n_g, n_h) <= 1e-12


def test_graph_run_to_steady_same_steps():
    """A full run to steady state on the tiny column through graphs converges in
    the same number of steps as without."""
    p = synth.tiny_column()
    n_g, info_g, glaunch = _run(p, "mixed", 1, 3000)
    n_h, info_h, _ = _run(p, "mixed", 0, 3000)
    assert info_g.converged and info_h.converged
    assert info_g.steps == info_h.steps
    assert glaunch == -(-info_g.steps // 16)     # one replay per 16-step chunk
    assert _close(n_g, n_h) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_round_is_one_graph_launch(precision):
    probs = [synth.tiny_column(), synth.small_column(),
             synth.small_column(S=30, L=45, n_two=80, n_three=20, n_photo=6, seed=9, W=120)]
    states = {}
    for use_graphs in (1, 0):
        b = xk.Batch(32 << 30, 4)
        cols, slots = [], []
        for p in probs:
            c = xk.Column(p, precision, use_graphs=use_graphs)
            c.set_mixing_ratios(p.f0)
            slots.append(b.add(c, 1e-8))
            cols.append(c)
        g0 = xk.Column.graph_launches()
        k0 = xk.Column.lib_launches()
        rounds = 6
        for _ in range(rounds):
            b.step(3)
        g = xk.Column.graph_launches() - g0
        k = xk.Column.lib_launches() - k0
        if use_graphs:
            assert g == rounds              # one graph launch per round, all columns in it
        else:
            assert g == 0
        assert k > 0
        states[use_graphs] = [(b.poll(s)[0].steps, b.remove(s).get_state()) for s in slots]
        b.close()
    for (sg, ng), (sh, nh) in zip(states[1], states[0]):
        assert sg == sh
        assert _close(ng, nh) <= 1e-12


def test_batch_submit_replays_a_graph():
    p = synth.small_column()
    b = xk.Batch(8 << 30, 2)
    c = xk.Column(p, "mixed")
    c.set_mixing_ratios(p.f0)
    slot = b.add(c, 1e-8)
    g0 = xk.Column.graph_launches()
    for _ in range(3):
        b.submit(slot, 4)
        while not b.query(slot):
            pass
    assert xk.Column.graph_launches() - g0 == 3
    info, finished, status = b.poll(slot)
    assert status == 0 and (finished or info.steps == 12)
    b.close()
