"""xk_block_solve_noalloc: the block solve for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

Called through the C-ABI and checked against xk_block_solve, the entry point
that works from a caller-provided workspace, on two calls in a row with
different right-hand sides (the shared scratch keeps the previous call's
contents, so the second call also checks that nothing stale leaks in).
This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import synth, xk  # noqa: E402

xkbuild.build()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_solve_matches_workspace_solve_twice():
    p = synth.small_column()
    col = xk.Column(p, "fp64")
    n = torch.as_tensor(p.f0, device="cuda") * col.eval_grid()[0][:, None]
    A, lo, up = col.eval_jacobian(n, 1e-2)
    rng = np.random.default_rng(11)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        f = torch.as_tensor(rng.normal(size=(p.L, p.S)), device="cuda") * n
        ref = col.block_solve(A, lo, up, f)
        x = torch.full_like(f, float("nan"))
        rc = xk.lib().xk_block_solve_noalloc(p.L, p.S, _ptr(A), _ptr(lo), _ptr(up), _ptr(f), _ptr(x), stream)
        assert rc == 0, (call, rc)
        scale = ref.abs().max().item()
        assert torch.isfinite(x).all()
        assert (x - ref).abs().max().item() / scale < 1e-10, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = xk.lib().xk_block_solve_noalloc(12, 594, _ptr(t), _ptr(t), _ptr(t), _ptr(t), _ptr(t), stream)
    assert rc == -2            # XK_ENOMEM: 12 layers of 594 species exceed the 32 MiB scratch
    rc = xk.lib().xk_block_solve_noalloc(0, 594, _ptr(t), _ptr(t), _ptr(t), _ptr(t), _ptr(t), stream)
    assert rc == -1            # XK_EINVAL
