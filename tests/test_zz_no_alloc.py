"""The allocation-free operator entry point against the allocating one.

rve_apply_operator_2d_static serves callers that cannot call cudaMalloc (an
application owning the whole device pool through its own allocator, or a
latency-critical loop).  It must give the same q = G C p (and the bare
projection) as rve_apply_operator on an FP32 (mixed) handle, on consecutive
calls that share its static scratch.  This file is collected last so that a
run stopping at the first failure has run every other test already.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import lognormal, require_gpu

pytestmark = pytest.mark.gpu


def _static_apply(lib, n, E_dev, nu, p_dev, q_dev, material):
    import torch
    nn = (C.c_int64 * 2)(*n)
    code = lib.rve_apply_operator_2d_static(nn, None, C.c_void_p(E_dev.data_ptr()), nu,
                                            C.c_void_p(p_dev.data_ptr()), C.c_void_p(q_dev.data_ptr()),
                                            1 if material else 0,
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code


@pytest.mark.parametrize("n", [(64, 32), (256, 256)])
def test_static_operator_matches_handle_operator(n):
    require_gpu()
    import torch
    from paper_2105_03297_gb300 import RVE, _rve
    lib = _rve.load()
    nu = 0.3
    E = lognormal(n, 41).astype(np.float32)
    rng = np.random.default_rng(42)
    E_dev = torch.from_numpy(E.reshape(-1)).cuda()
    with RVE(n, precision="mixed") as r:
        r.set_material(E, nu)
        for call, material in enumerate((True, False, True)):   # consecutive calls share the scratch
            p = rng.standard_normal((6, E.size)).astype(np.float32)
            ref = r.apply_operator(p, material=material)
            p_dev = torch.from_numpy(p).cuda()
            q_dev = torch.full_like(p_dev, float("nan"))
            assert _static_apply(lib, n, E_dev, nu, p_dev, q_dev, material) == 0
            q = q_dev.cpu().numpy()
            assert np.all(np.isfinite(q)), call
            assert np.abs(q - ref).max() <= 2e-5 * np.abs(ref).max(), call


def test_static_operator_rejects_grids_beyond_its_scratch():
    require_gpu()
    import torch
    from paper_2105_03297_gb300 import _rve
    lib = _rve.load()
    n = (512, 64)
    E_dev = torch.ones(n[0] * n[1], device="cuda")
    p_dev = torch.zeros(6 * n[0] * n[1], device="cuda")
    q_dev = torch.zeros_like(p_dev)
    assert _static_apply(lib, n, E_dev, 0.3, p_dev, q_dev, True) == _rve.RVE_ERR_SCRATCH_LIMIT
    assert b"static scratch" in lib.rve_error_string(_rve.RVE_ERR_SCRATCH_LIMIT)
