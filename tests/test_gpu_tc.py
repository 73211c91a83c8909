"""The tensor-core contraction (tcgen05, TF32 head/tail split, three
products per step) through the C-ABI against an FP64 product of the same FP32
inputs: sizes of one and of several 128 x 128 tiles with ragged last tiles,
long K (several pipeline rounds), alpha/beta accumulation in place, and
operands spanning many orders of magnitude (the scaled Jacobian blocks do).

Bound: the head is x rounded to 10 explicit mantissa bits, so the tail is
at most 2^-11 of |x|; rounding the tail to TF32 and dropping the
tail-by-tail term leave at most 3 * 2^-22 of |a||b| per product, and FP32
accumulation over K terms adds up to K * 2^-24: |C - C_ref| <=
(3 * 2^-22 + K 2^-24) (|A| |B|) per element.  A layout or indexing error
gives O(1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import xk  # noqa: E402

xkbuild.build()


def _check(M, N, K, seed, alpha=1.0, beta=0.0, spread=0.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    if spread:
        A *= np.exp(rng.uniform(-spread, spread, size=(M, 1))).astype(np.float32)
        B *= np.exp(rng.uniform(-spread, spread, size=(1, N))).astype(np.float32)
    C0 = rng.normal(size=(M, N)).astype(np.float32)
    ref = alpha * (A.astype(np.float64) @ B.astype(np.float64)) + beta * C0.astype(np.float64)
    mag = np.abs(alpha) * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)) + abs(beta) * np.abs(C0)
    dA, dB = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
    dC = torch.as_tensor(C0, device="cuda")
    xk.tc_gemm(dA, dB, dC, alpha, beta)
    got = dC.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - ref) / (mag + 1e-30))
    assert np.isfinite(got).all()
    return err / (3 * 2.0 ** -22 + K * 2.0 ** -24)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (32, 32, 32), (160, 96, 64), (256, 384, 608), (608, 608, 608),
                                   (96, 1216, 288)])
def test_tc_gemm_matches_fp64(M, N, K):
    err = _check(M, N, K, seed=M + N + K)
    assert err < 1.0, err


def test_tc_gemm_alpha_beta_and_wide_range():
    assert _check(288, 320, 160, seed=1, alpha=-1.0, beta=1.0) < 1.0
    assert _check(128, 256, 608, seed=2, alpha=0.5, beta=-2.0, spread=20.0) < 1.0
