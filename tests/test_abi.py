"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point that include/amgpr.h declares, and the calls that
only validate arguments answer without touching a device."""
import ctypes
import os
import re

import pytest

from paper_2108_02054_gb300 import amg as B
from paper_2108_02054_gb300 import build as Bd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "amgpr.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    path = Bd.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == declared


def test_default_params_and_argument_checks_without_gpu():
    p = B.default_params()
    assert p.theta == 0.08 and abs(p.omega - 2 / 3) < 1e-16 and p.smoother == 0
    assert (p.npre, p.npost, p.coarse_enough, p.max_levels, p.maxiter) == (1, 1, 256, 20, 100)
    L = B.lib()
    assert L.amg_poisson_nnz(3, 192) == 49_324_032
    assert L.amg_poisson_nnz(2, 32) == 4992
    assert L.amg_poisson_nnz(4, 8) == -1
    h = ctypes.c_void_p()
    bad = B.default_params(npre=-1)
    assert L.amg_create(ctypes.byref(h), ctypes.byref(bad), None) == B.AMG_ERR_ARG
    bad = B.default_params(precision=7)
    assert L.amg_create(ctypes.byref(h), ctypes.byref(bad), None) == B.AMG_ERR_ARG
    assert L.amg_full_setup(None, 4, 4, None, None, None) == B.AMG_ERR_ARG
    assert L.amg_solve(None, None, None, 1e-8, None) == B.AMG_ERR_ARG
    assert L.amg_poisson_pattern(5, 8, None, None, None) == B.AMG_ERR_ARG
    assert B.lib().amg_last_error(None) == b"null context"


def test_binding_fails_loudly_without_the_library(monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", "/nonexistent/libamgpr.so")
    with pytest.raises(RuntimeError, match="missing"):
        B.lib()
