"""The C-ABI library builds, loads and exports every function of include/rve.h.

CPU only: no compute call is made (argument checks that fail before any CUDA
work are exercised).
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_03297_gb300.build import build_library
    build_library()
    from paper_2105_03297_gb300 import _rve
    return _rve.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "rve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2105_03297_gb300 import _rve
    names = _declared()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
        assert name in _rve.SIGNATURES, f"{name} has no binding"


def test_error_strings(lib):
    for code in range(0, -9, -1):
        assert lib.rve_error_string(code)
    assert b"unknown" in lib.rve_error_string(42)


def test_argument_checks_before_any_device_work(lib):
    h = C.c_void_p()
    n = (C.c_int64 * 2)(30, 32)
    assert lib.rve_create(C.byref(h), 2, n, None, 0, None) == -2       # not a power of two
    n = (C.c_int64 * 2)(2048, 32)
    assert lib.rve_create(C.byref(h), 2, n, None, 0, None) == -2       # beyond the FFT range
    n3 = (C.c_int64 * 3)(512, 16, 16)
    assert lib.rve_create(C.byref(h), 3, n3, None, 0, None) == -2
    assert lib.rve_create(C.byref(h), 4, n3, None, 0, None) == -1      # bad dimension
    assert lib.rve_create(C.byref(h), 2, n, None, 7, None) == -1       # bad precision
    assert lib.rve_destroy(None) == 0
    assert lib.rve_solve(None, None, 1, 1e-8, 10, None) == -1
