"""Parity of the extinction and diffuse field (Sec. 2.3.3) on the GPU with the FP64 CPU oracle:
photolysis rates with Rayleigh scattering in the optical depth and the two-stream diffuse field,
on the 1,000-bin grid and the paper's 10,000-bin grid (1-10,000 A), and a linear step with them.

Tolerance: 1e-11 relative on every photolysis rate above 1e-300 s^-1 (the same exponentials and
sums as the direct beam's; the GPU's two-stream recursion and the oracle's banded elimination of
the same system differ by rounding only, each row being diagonally dominant)."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


CASES = {
    "small-albedo0.3": lambda: synth.with_scattering(synth.small_column(), albedo=0.3),
    "chons-1000": lambda: synth.with_scattering(synth.chons_column()),
    "chons-10000": lambda: synth.with_scattering(synth.chons_column(), albedo=0.1, bins=10000),
    "full-10000": lambda: synth.with_scattering(synth.full_column(), bins=10000),
    "small-scatter-no-diffuse": lambda: synth.with_scattering(synth.small_column(), diffuse=0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_photolysis_with_scattering_matches_oracle(name):
    p = CASES[name]()
    o = Oracle(p)
    n = o.initial_state()
    c = xk.Column(p, "fp64")
    kph = cpu(c.eval_photolysis(dev(n)))
    ref = o.photolysis(n)
    m = ref > 1e-300
    assert m.sum() > 0.5 * ref.size
    assert np.max(np.abs(kph[m] - ref[m]) / ref[m]) < 1e-11
    assert np.all(np.abs(kph[~m]) < 1e-290)
    # the diffuse field changes the rates (the test would not see a dropped J_diff otherwise)
    if p.diffuse:
        base = Oracle(p.replace(diffuse=0)).photolysis(n)
        assert np.max(np.abs(ref[m] - base[m]) / ref[m]) > 1e-3
    c.close()


def test_step_with_diffuse_field_matches_oracle():
    p = synth.with_scattering(synth.small_column(), albedo=0.2)
    o = Oracle(p)
    n = o.initial_state()
    ngas = o.grid()[0]
    s = np.maximum(n, 1e-20 * ngas[:, None])
    for prec in ("fp64", "mixed"):
        c = xk.Column(p, prec)
        d, iters, res = c.step_delta(dev(n), 1e-4)
        ref = o.step_delta(n, 1e-4)
        assert np.max(np.abs(cpu(d) - ref) / s) < 1e-7, prec
        c.close()


def test_scattering_inputs_are_checked():
    p = synth.small_column()
    bad = synth.with_scattering(p).replace(albedo=1.5)
    with pytest.raises(xk.XkError):
        xk.Column(bad, "fp64")
    neg = synth.with_scattering(p)
    sig = neg.sigma_s.copy()
    sig[0, 0] = -1.0
    with pytest.raises(xk.XkError):
        xk.Column(neg.replace(sigma_s=sig), "fp64")


def test_step_with_photolysis_jacobian_matches_coupled_oracle():
    """With photo_jacobian the step solves the fully linearised system (dk_ph/dn couples every layer
    to the layers above it) through FGMRES on the exact operator: it matches the oracle's dense
    coupled step, and differs from the lagged step by far more than that tolerance."""
    p = synth.small_column(L=20)
    o = Oracle(p)
    n, _ = o.run_to_steady(o.initial_state(), max_steps=300)
    ngas = o.grid()[0]
    s = np.maximum(n, 1e-20 * ngas[:, None])
    dt = 1.0
    ref = o.step_delta_coupled(n, dt)
    lag = o.step_delta(n, dt)
    assert np.max(np.abs(ref - lag) / s) > 1e-4
    for prec in ("fp64", "mixed"):
        c = xk.Column(p, prec, photo_jacobian=1)
        d, iters, res = c.step_delta(dev(n), dt)
        assert np.max(np.abs(cpu(d) - ref) / s) < 1e-6, (prec, iters, res)
        c.close()


def test_photolysis_jacobian_refuses_the_diffuse_field():
    p = synth.with_scattering(synth.small_column(), diffuse=1)
    with pytest.raises(xk.XkError):
        xk.Column(p, "mixed", photo_jacobian=1)
