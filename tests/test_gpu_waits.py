"""Bounded device-side waits: a grid barrier that can never complete (its
arrival count raised from the host, as if a CTA never arrived) makes the FP64
factorization give up after the configured number of polls; the call returns
XK_ETIMEOUT, nothing faults, and the same context then solves normally."""
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


@pytest.mark.parametrize("twisted", [1, 0])
def test_unreachable_barrier_times_out_and_context_recovers(twisted):
    p = synth.small_column()
    o = Oracle(p)
    n = o.initial_state()
    ng = o.grid()[0]
    nd = torch.as_tensor(n, device="cuda")
    col = xk.Column(p, "fp64", twisted=twisted, wait_polls=1 << 14)
    ref = o.step_delta(n, 1e-4)
    s = np.maximum(n, 1e-20 * ng[:, None])
    d0, _, _ = col.step_delta(nd, 1e-4)
    assert np.max(np.abs(d0.cpu().numpy() - ref) / s) < 1e-8
    col.hold_next_barrier()
    with pytest.raises(xk.XkError) as err:
        col.step_delta(nd, 1e-4)
    assert err.value.code == -7            # XK_ETIMEOUT
    for _ in range(2):
        d, _, _ = col.step_delta(nd, 1e-4)
        assert np.max(np.abs(d.cpu().numpy() - ref) / s) < 1e-8
    # a controlled step that meets the held barrier reports the timeout and leaves n untouched
    col.set_mixing_ratios(p.f0)
    before = col.get_state()
    col.hold_next_barrier()
    with pytest.raises(xk.XkError) as err:
        col.step(1e-12)
    assert err.value.code == -7
    np.testing.assert_array_equal(col.get_state(), before)
    # the next step runs as if nothing had happened: the oracle's decision and state
    on, oinfo = o.step(n, 1e-12)
    info = col.step(1e-12)
    assert oinfo.accepted == 1 and info.accepted == 1
    assert info.dt_next == pytest.approx(oinfo.dt_next, rel=1e-6)
    assert np.max(np.abs(col.get_state() - on) / s) < 1e-8
    col.close()
