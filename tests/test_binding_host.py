"""Argument marshalling of the Python binding (CPU, no device work): caller
buffers of the wrong element type, size or layout are rejected before the
library reads or writes them."""
import ctypes as C

import numpy as np
import pytest

from paper_2105_03297_gb300 import _rve


def test_buffer_accepts_exact_numpy_and_torch_buffers():
    a = np.zeros((3, 5))
    p, flag, keep = _rve._buffer(a, np.float64, 15, "a")
    assert flag == _rve.RVE_PTR_HOST and keep is a and p.value == a.ctypes.data
    torch = pytest.importorskip("torch")
    t = torch.zeros(15, dtype=torch.float32)
    p, flag, keep = _rve._buffer(t, np.float32, 15, "t")
    assert flag == _rve.RVE_PTR_HOST and p.value == t.data_ptr()


@pytest.mark.parametrize("bad,err", [
    (np.zeros(14), ValueError),                      # too small: the library would write past it
    (np.zeros(15, dtype=np.float32), TypeError),     # wrong element type
    (np.zeros((5, 6))[:, ::2], ValueError),          # 15 elements, not contiguous
    ([0.0] * 15, TypeError),                         # not a buffer
])
def test_buffer_rejects_mismatches(bad, err):
    with pytest.raises(err):
        _rve._buffer(bad, np.float64, 15, "out")


def test_buffer_rejects_torch_mismatches():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        _rve._buffer(torch.zeros(15, dtype=torch.float16), np.float64, 15, "E")
    with pytest.raises(ValueError):
        _rve._buffer(torch.zeros(16, dtype=torch.float64), np.float64, 15, "E")
    with pytest.raises(ValueError):
        _rve._buffer(torch.zeros(5, 6, dtype=torch.float64)[:, ::2], np.float64, 15, "E")


def _fake_handle(dim=2, n=(4, 4), precision="mixed"):
    """An RVE object with sizes but a NULL handle: if a check were missing, the
    library would see the NULL handle and return RVE_ERR_ARG, not touch memory."""
    r = object.__new__(_rve.RVE)
    r.n, r.dim, r.precision = n, dim, precision
    r.N = int(np.prod(n)); r.ns = 3 if dim == 2 else 6; r.m = 2 * r.ns if dim == 2 else 6 * r.ns
    r.inner_dtype = np.float32 if precision == "mixed" else np.float64
    r.h = None
    r.L = 0
    return r


def test_methods_check_their_buffers_first():
    r = _fake_handle()
    with pytest.raises(ValueError):
        r.set_material(np.ones(15), 0.3)                       # N = 16
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        r.set_material(torch.ones(16, dtype=torch.float16), 0.3)
    with pytest.raises(ValueError):
        r.solve(np.eye(4))                                      # n_s = 3
    with pytest.raises(ValueError):
        r.adjoint(np.eye(3), out=np.zeros(15))
    with pytest.raises(ValueError):
        r.adjoint(np.eye(2))
    with pytest.raises(ValueError):
        r.get_strain(0, out=np.zeros((r.m, r.N - 1)))
    with pytest.raises(TypeError):
        r.get_strain(0, out=np.zeros((r.m, r.N), dtype=np.float32))
    with pytest.raises(ValueError):
        r.apply_operator(np.zeros((r.m - 1, r.N)))
    with pytest.raises(TypeError):
        r.apply_operator(np.zeros((r.m, r.N)), out=np.zeros((r.m, r.N)))   # out must be FP32 here
    r.h = None


def test_null_handle_is_an_argument_error():
    lib = _rve.load()
    assert lib.rve_solve(None, None, 1, 1e-10, 10, None) == _rve.RVE_ERR_ARG
    assert lib.rve_set_material(None, None, _rve.RVE_F64, 0.3, _rve.RVE_PTR_HOST) == _rve.RVE_ERR_ARG
    assert lib.rve_apply_operator(None, None, None, 1, 0) == _rve.RVE_ERR_ARG
    assert lib.rve_get_strain(None, 0, None, 0) == _rve.RVE_ERR_ARG
    assert isinstance(lib.rve_error_string(_rve.RVE_ERR_ARG), bytes)
    assert C.sizeof(_rve.rve_info) == 32


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the built library every entry point raises."""
    saved = _rve._lib
    _rve._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            _rve.load(str(tmp_path / "librve.so"))
    finally:
        _rve._lib = saved


def _header_constants():
    """Every RVE_* constant of include/rve.h (enum members and #defines)."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rve.h")
    src = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"(RVE_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    for name, val in re.findall(r"#define\s+(RVE_[A-Z0-9_]+)\s+(-?\d+)", src):
        consts[name] = int(val)
    return consts


def test_binding_constants_match_the_header():
    h = _header_constants()
    for name in ("RVE_OK", "RVE_ERR_ARG", "RVE_ERR_UNSUPPORTED_SIZE", "RVE_ERR_CUDA", "RVE_ERR_OOM",
                 "RVE_ERR_NOT_CONVERGED", "RVE_ERR_NONFINITE", "RVE_ERR_TIMEOUT", "RVE_ERR_SCRATCH_LIMIT",
                 "RVE_FP64", "RVE_MIXED", "RVE_F32", "RVE_F64", "RVE_PTR_HOST", "RVE_PTR_DEVICE"):
        assert getattr(_rve, name) == h[name], name
    assert (_rve.RVE.SCHED_PASSES, _rve.RVE.SCHED_VARIANTS) == (h["RVE_SCHED_PASSES"], h["RVE_SCHED_VARIANTS"])
    assert _rve.RVE.FORMS == {"stress": h["RVE_FORM_STRESS"], "factored": h["RVE_FORM_FACTORED"],
                              "nodal": h["RVE_FORM_NODAL"]}
    assert len(_rve.RVE.KINDS) == h["RVE_NKINDS"]
    assert _rve.RVE.DERIVATIVES == {"fe": h["RVE_DERIV_FE"], "fourier": h["RVE_DERIV_FOURIER"],
                                    "central": h["RVE_DERIV_CENTRAL"], "forward": h["RVE_DERIV_FORWARD"],
                                    "lsq": h["RVE_DERIV_LSQ"], "fourier2": h["RVE_DERIV_FOURIER2"]}
