"""xk_block_solve_noalloc: the block solve for callers that cannot allocate
device memory (its scratch is a fixed device array inside the library).

Called through the C-ABI on a system built by the CPU oracle, and checked
against the oracle's own solve and against xk_block_solve (the entry point
that works from a caller-provided workspace), on two calls in a row with
different right-hand sides: the shared scratch keeps the previous call's
contents, so the second call also checks that nothing stale leaks in.  A call
with a host pointer after a good call must be refused, not answered with the
previous call's result.  This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2512_06729_gb300 import build as xkbuild  # noqa: E402
from paper_2512_06729_gb300 import synth, xk  # noqa: E402

xkbuild.build()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def test_noalloc_solve_matches_oracle_and_workspace_solve_twice():
    p = synth.small_column()
    o = Oracle(p)
    n = o.initial_state()
    oA, olo, oup = o.jacobian(n, 1e-2)
    A, lo, up = _dev(oA), _dev(olo), _dev(oup)
    col = xk.Column(p, "fp64")
    rng = np.random.default_rng(11)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        fh = rng.normal(size=(p.L, p.S)) * n
        f = _dev(fh)
        ox = o.block_solve(oA, olo, oup, fh)
        ref = col.block_solve(A, lo, up, f).cpu().numpy()
        x = torch.full_like(f, float("nan"))
        rc = xk.lib().xk_block_solve_noalloc(p.L, p.S, _ptr(A), _ptr(lo), _ptr(up), _ptr(f), _ptr(x), stream)
        assert rc == 0, (call, rc)
        xh = x.cpu().numpy()
        assert np.isfinite(xh).all()
        scale = np.abs(ox).max()
        assert np.max(np.abs(xh - ox)) / scale < 1e-10, call
        assert np.max(np.abs(xh - ref)) / scale < 1e-10, call
    # a host array in place of A after a good call: refused before any work, x left alone
    A_host = np.ascontiguousarray(oA)
    x = torch.full_like(f, 7.0)
    rc = xk.lib().xk_block_solve_noalloc(p.L, p.S, C.c_void_p(A_host.ctypes.data), _ptr(lo), _ptr(up), _ptr(f),
                                         _ptr(x), stream)
    assert rc == -1                        # XK_EINVAL
    torch.cuda.synchronize()
    assert (x == 7.0).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = xk.lib().xk_block_solve_noalloc(12, 594, _ptr(t), _ptr(t), _ptr(t), _ptr(t), _ptr(t), stream)
    assert rc == -2            # XK_ENOMEM: 12 layers of 594 species exceed the 32 MiB scratch
    rc = xk.lib().xk_block_solve_noalloc(0, 594, _ptr(t), _ptr(t), _ptr(t), _ptr(t), _ptr(t), stream)
    assert rc == -1            # XK_EINVAL
