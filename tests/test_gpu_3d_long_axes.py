"""GPU parity of the 3D kernels at axis lengths 128 and 256 against the FP64 oracle.

The kernels are compiled per axis length (the x transform of passes A and E,
the y transform of passes B and D, the z transform and projection of pass C,
and the force and update stencils of the factored and nodal forms), and the
256-point instantiations use their own FFT split, launch shapes and shared
memory sizes; these grids put 256 (or 128) points on one axis at a time:

* the projected operator q = G C p (Appendix B, Eqs. small-strain-eq2 and
  small-strain-chi; six Kuhn tetrahedra per voxel, Sec. 2.6) elementwise, FP64
  to 1e-12 and FP32 to 2e-5 of the field maximum, with every row-tile variant
  of passes A and E where n_x = 256;
* a converged solve (stress, factored and nodal forms): mean stress and the
  strain field of the load case against the oracle's, to 1e-9.
"""
import functools

import numpy as np
import pytest

from oracle.fe_projection import Problem
from tests.gpu_util import lognormal, rel_max, require_gpu

pytestmark = pytest.mark.gpu

LONG = [(256, 16, 16), (16, 256, 16), (16, 16, 256), (128, 128, 16)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("n", LONG)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_operator_elementwise_long_axes(n, prec, tol):
    from paper_2105_03297_gb300 import RVE
    E = lognormal(n, 91)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(92).standard_normal((P.m,) + E.shape)
    if prec == "mixed":
        p = p.astype(np.float32).astype(np.float64)
    ref = P.operator(p)
    variants = (0, 1, 2) if n[0] == 256 else (0,)
    with RVE(n, precision=prec) as r:
        r.set_material(E, 0.3)
        for v in variants:
            r.set_schedule(v, v)
            q = r.apply_operator(p.reshape(P.m, -1)).reshape(ref.shape)
            assert np.abs(q - ref).max() <= tol * np.abs(ref).max(), v


@pytest.mark.parametrize("n", [(256, 16, 16), (16, 16, 256)])
def test_bare_projection_long_axes(n):
    from paper_2105_03297_gb300 import RVE
    E = lognormal(n, 93)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(94).standard_normal((P.m,) + E.shape)
    ref = P.project(p)
    with RVE(n, precision="fp64") as r:
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1), material=False).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()


EMAC = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0])


@functools.lru_cache(maxsize=None)
def _oracle(n):
    P = Problem(n, lognormal(n, 95), 0.3)
    eps, _, _ = P.solve(EMAC, tol=1e-13)
    return P.mean_stress(eps), eps


@pytest.mark.parametrize("n", [(256, 16, 16), (16, 256, 16), (16, 16, 256)])
@pytest.mark.parametrize("form,prec", [("stress", "mixed"), ("stress", "fp64"), ("factored", "mixed"),
                                       ("nodal", "mixed")])
def test_solve_long_axis_matches_oracle(n, form, prec):
    from paper_2105_03297_gb300 import RVE
    S_ref, eps_ref = _oracle(n)
    with RVE(n, precision=prec) as r:
        r.set_operator_form(form)
        r.set_material(lognormal(n, 95), 0.3)
        code, info = r.solve(EMAC[None], rel_tol=1e-12, max_iter=4000)
        S = r.mean_stress()[0]
        eps = r.get_strain(0).reshape(eps_ref.shape)
    assert code == 0, info
    assert rel_max(S, S_ref) < 1e-9
    assert np.abs(eps - eps_ref).max() <= 1e-9 * np.abs(eps_ref).max()


@pytest.mark.parametrize("n", [(256, 16, 16), (128, 32, 32)])
def test_pipelined_passes_run_the_same_cg(n):
    """Tile variant 5 of the first pass and variant 3 of the last pass (persistent
    grids whose next tile's rows, and the last pass's spectrum tile, arrive by
    TMA copies on an mbarrier while the current tile is transformed), and
    variants 6 and 4 (the default tiles, each block asking for a later block's
    rows and spectrum tile to be prefetched into L2), run the same CG as
    variants 0: two load cases solved together (per-slot partial sums) give the
    same mean stresses to 1e-10, and the oracle's to 1e-9."""
    from paper_2105_03297_gb300 import RVE
    E = lognormal(n, 95)
    Em = np.eye(6)[[0, 3]]
    S = {}
    for va, ve in ((0, 0), (5, 0), (0, 3), (5, 3), (6, 4), (6, 0), (0, 4)):
        with RVE(n, precision="mixed") as r:
            r.set_schedule(va, ve, 0, 0)
            r.set_material(E, 0.3)
            code, info = r.solve(Em, rel_tol=1e-12, max_iter=4000)
            assert code == 0, info
            assert r.schedule()[0][:2] == [va, ve]
            S[va, ve] = r.mean_stress()
    for key in ((5, 0), (0, 3), (5, 3), (6, 4), (6, 0), (0, 4)):
        assert rel_max(S[key], S[0, 0]) < 1e-10, key
    if n == (256, 16, 16):
        S_ref, _ = _oracle(n)
        assert rel_max(S[5, 3][0], S_ref) < 1e-9


def test_pipelined_wait_that_runs_out_reports_a_timeout():
    """Failure detection without a GPU fault: with the test hook on, the
    pipelined passes issue none of their copies, so their bounded mbarrier waits
    (about two seconds) run out; the solve must return RVE_ERR_TIMEOUT, and the
    same handle must solve correctly once the hook is off (the context stays
    usable)."""
    from paper_2105_03297_gb300 import RVE, _rve
    n = (256, 16, 16)
    E = lognormal(n, 95)
    with RVE(n, precision="mixed") as r:
        r.set_schedule(5, 3, 0, 0)
        r.set_material(E, 0.3)
        r.test_stall_copies(True)
        with pytest.raises(_rve.RveError) as err:
            r.solve(EMAC[None], rel_tol=1e-12, max_iter=4000)
        assert err.value.code == _rve.RVE_ERR_TIMEOUT
        r.test_stall_copies(False)
        code, info = r.solve(EMAC[None], rel_tol=1e-12, max_iter=4000)
        assert code == 0, info
        S_ref, _ = _oracle(n)
        assert rel_max(r.mean_stress()[0], S_ref) < 1e-9
