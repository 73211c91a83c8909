"""The C-ABI library builds, loads and exports every entry point the public
header declares (no GPU needed; no compute calls)."""
import ctypes as C
import os
import re

import pytest

from paper_2512_06729_gb300 import build, xk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(xk_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libxk():
    build.build()
    return xk.lib()


def test_every_declared_symbol_is_exported(libxk):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libxk, n), n


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(xk.SIGNATURES)


def test_config_defaults(libxk):
    cfg = xk.Config()
    assert libxk.xk_config_init(C.byref(cfg)) == 0
    assert cfg.precision == 0 and cfg.dt_max == 1e8 and cfg.ss_tol == 1e-3 and cfg.gmres_restart == 30 and cfg.gmres_max_iter == 40
    assert libxk.xk_version() >= 100


def test_bad_arguments_are_rejected_without_a_gpu(libxk):
    assert libxk.xk_config_init(None) == -1
    assert libxk.xk_create(None, None) == -1
    assert libxk.xk_destroy(None) == -1
