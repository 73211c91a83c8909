"""Parity of the variable-order BDF integrator (the DLSODES family of Sec. 2.1) on the GPU,
through the C-ABI, with the oracle's BDF: the same accepted and rejected attempts, orders and
times on the first steps of the tiny and small columns in both precision modes, and the same end
state, and runs to steady state that end at the oracle's end state.

Tolerances: step counts and per-order histograms equal; times 1e-9 relative; states 1e-6 relative
on species above 1e-20 mixing ratio (each step is the linear solve of the backward-Euler parity
tests, with the same 1e-6 bound per step on these columns)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle, default_policy
from paper_2512_06729_gb300 import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import xk  # noqa: E402

xkbuild.build()

CASES = {
    "tiny": (lambda: synth.tiny_column(), 1e4),
    "small": (lambda: synth.small_column(), 1e2),
}


def _rel(a, b, ngas):
    keep = b > 1e-20 * ngas[:, None]
    return float(np.max(np.abs(a[keep] - b[keep]) / b[keep]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_bdf_steps_follow_the_oracle(name, prec):
    make, t_end = CASES[name]
    p = make()
    o = Oracle(p)
    n0 = o.initial_state()
    ngas = o.grid()[0]
    for max_steps in (25, 80):
        ref, ri, rrc = o.bdf_run(n0, h0=1e-8, t_end=t_end, max_steps=max_steps, rtol=1e-3)
        c = xk.Column(p, prec)
        c.set_state(n0)
        gi, grc = c.bdf_run(h0=1e-8, t_end=t_end, max_steps=max_steps, rtol=1e-3)
        assert (gi.steps, gi.accepted, gi.rejected) == (ri.steps, ri.accepted, ri.rejected)
        assert list(gi.order_steps) == list(ri.order_steps)
        assert gi.q == ri.q
        assert gi.t == pytest.approx(ri.t, rel=1e-9)
        assert _rel(c.get_state(), ref, ngas) < 1e-6
        c.close()
    assert max(i for i in range(6) if ri.order_steps[i]) >= 3


def test_bdf_run_to_steady_matches_oracle():
    """A run to a tight steady state ends at a fixed point of the oracle's residual (1e-8 of the
    gross fluxes, as the oracle's own run), and at the oracle's end state within the spread the
    oracle itself shows when its initial state is perturbed by 1e-13 (three draws; the step count
    then changes by thousands, the end state by ~1e-7-1e-6: the fixed point is ill-conditioned),
    times 10, at least 1e-5."""
    from tests.test_oracle_bdf import _relative_residual
    p = synth.tiny_column()
    o = Oracle(p)
    n0 = o.initial_state()
    ngas = o.grid()[0]
    pol = dict(ss_tol=1e-9, ss_dt=1e11, dt_max=1e13)
    ref, ri, rrc = o.bdf_run(n0, h0=1e-8, stop_at_steady=True, max_steps=8000, policy=default_policy(**pol))
    assert ri.converged
    spread = 0.0
    for seed in (3, 4, 5):
        pert = n0 * (1.0 + 1e-13 * np.random.default_rng(seed).standard_normal(n0.shape))
        ref2, ri2, _ = o.bdf_run(pert, h0=1e-8, stop_at_steady=True, max_steps=8000, policy=default_policy(**pol))
        assert ri2.converged
        spread = max(spread, _rel(ref2, ref, ngas))
    bound = max(1e-5, 10.0 * spread)
    c = xk.Column(p, "fp64", **pol)
    c.set_state(n0)
    gi, grc = c.bdf_run(h0=1e-8, stop_at_steady=True, max_steps=8000)
    assert grc == 0 and gi.converged
    g = c.get_state()
    assert _relative_residual(o, p, g) < 1e-8
    assert _rel(g, ref, ngas) < bound
    c.close()


def test_bdf_fixed_order_and_arguments():
    p = synth.tiny_column()
    o = Oracle(p)
    n0 = o.initial_state()
    ngas = o.grid()[0]
    ref, ri, _ = o.bdf_run(n0, h0=1e-6, t_end=2e-5, max_steps=100, fixed_order=3, fixed_step=1, qmax=3)
    c = xk.Column(p, "fp64")
    c.set_state(n0)
    gi, _ = c.bdf_run(h0=1e-6, t_end=2e-5, max_steps=100, fixed_order=3, fixed_step=1, qmax=3)
    assert gi.accepted == ri.accepted == 20 and list(gi.order_steps) == list(ri.order_steps)
    assert _rel(c.get_state(), ref, ngas) < 1e-9
    for bad in (dict(rtol=0.0), dict(qmax=6), dict(grow=0.5)):
        with pytest.raises(xk.XkError):
            c.bdf_run(**bad)
    c.close()
