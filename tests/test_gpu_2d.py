"""GPU parity of the 2D path (two triangles per pixel) against the FP64 oracle.

Every call goes through the C ABI (ctypes binding of librve.so).
Tolerances: FP64 operator 1e-12 of the field maximum (FFT round-off);
FP32 operator 2e-5 (single-precision FFTs of length <= 1024); effective
stiffness 1e-9 relative in the matrix-max norm for both precisions.
"""
import json
import os

import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent
from oracle.fe_projection import Problem
from tests.gpu_util import lognormal, rel_max, require_gpu

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _rve(n, prec):
    from paper_2105_03297_gb300 import RVE
    return RVE(n, precision=prec)


@pytest.mark.parametrize("n", [(16, 16), (32, 64), (128, 16), (256, 256)])
@pytest.mark.parametrize("material", [True, False])
def test_operator_fp64_elementwise(n, material):
    E = lognormal(n, 1)
    P = Problem(n, E, 0.3)
    rng = np.random.default_rng(2)
    p = rng.standard_normal((P.m,) + E.shape)
    ref = P.operator(p) if material else P.project(p)
    with _rve(n, "fp64") as r:
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1), material=material).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [(32, 32), (1024, 64), (64, 1024)])
def test_operator_fp32_elementwise(n):
    E = lognormal(n, 3)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(4).standard_normal((P.m,) + E.shape)
    ref = P.operator(p.astype(np.float32).astype(np.float64))
    with _rve(n, "mixed") as r:
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1).astype(np.float32)).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_disc32_effective_tangent(prec):
    cfg = ms.config_inputs("disc32")
    ref = json.load(open(os.path.join(GOLDEN, "disc32.json")))
    Cref = np.array(ref["C_eff"])
    with _rve(cfg["n"], prec) as r:
        r.set_material(cfg["E"], cfg["nu"])
        code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, Cref) < 1e-9
    assert rel_max(C, np.array(ref["C_eff_fem"])) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 32), (64, 64)])
def test_strain_field_matches_oracle(prec, n):
    E = lognormal(n, 5)
    P = Problem(n, E, 0.3)
    Em = np.array([0.01, -0.004, 0.003])
    eps_ref, _, _ = P.solve(Em, tol=1e-13)
    with _rve(n, prec) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(Em[None], rel_tol=1e-12, max_iter=3000)
        eps = r.get_strain(0).reshape(eps_ref.shape)
        S = r.mean_stress()[0]
    assert code == 0, info
    assert np.abs(eps - eps_ref).max() <= 1e-9 * np.abs(eps_ref).max()
    assert rel_max(S, P.mean_stress(eps_ref)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_homogeneous_material_needs_no_iteration(prec):
    n = (32, 16)
    with _rve(n, prec) as r:
        r.set_material(np.full((16, 32), 3.0), 0.25)
        code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=100)
        C = r.effective_tangent()
    assert code == 0
    assert all(i["iterations"] == 0 for i in info)
    from oracle.fe_projection import stiffness_mandel
    assert rel_max(C, stiffness_mandel(2, 3.0, 0.25)) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_laminate_closed_form(prec):
    n = (64, 16)
    layers = np.exp(2.0 * np.random.default_rng(9).standard_normal(64))
    with _rve(n, prec) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, _ = r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        C = r.effective_tangent()
    assert code == 0
    assert rel_max(C, laminate_tangent(layers, 0.3, 2)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_matches_oracle(prec):
    n = (16, 16)
    E = lognormal(n, 11)
    P = Problem(n, E, 0.3)
    W = np.array([[1.0, 0.2, 0.0], [0.2, 0.5, 0.0], [0.0, 0.0, 0.3]])
    g_ref, C_ref = P.adjoint_gradient(W, tol=1e-13)
    with _rve(n, prec) as r:
        r.set_material(E, 0.3)
        r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        g = r.adjoint(W, rel_tol=1e-12, max_iter=3000).reshape(E.shape)
    assert rel_max(g, g_ref) < 1e-9
    J = float(np.sum(W * C_ref))
    assert abs(np.sum(E * g) - J) < 1e-9 * abs(J)


def test_errors_are_reported():
    from paper_2105_03297_gb300 import RveError
    n = (32, 32)
    E = lognormal(n, 1)
    with _rve(n, "fp64") as r:
        bad = E.copy(); bad[3, 4] = np.nan
        with pytest.raises(RveError):
            r.set_material(bad, 0.3)
        with pytest.raises(RveError):
            r.set_material(E, 0.5)
        r.set_material(E, 0.3)
        code, info = r.solve([[0.01, 0, 0]], rel_tol=1e-12, max_iter=2)
        assert code == -5 and info[0]["status"] == -5
        with pytest.raises(RveError):
            r.effective_tangent()   # L != n_s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gauss1024_golden(prec):
    path = os.path.join(GOLDEN, "gauss1024.json")
    if not os.path.exists(path):
        pytest.skip("golden not generated")
    ref = json.load(open(path))
    cfg = ms.config_inputs("gauss1024")
    with _rve(cfg["n"], prec) as r:
        r.set_material(cfg["E"], cfg["nu"])
        code, info = r.solve(cfg["E_macro"], rel_tol=1e-11, max_iter=5000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, np.array(ref["C_eff"])) < 1e-9


@pytest.mark.parametrize("dim", [2, 3])
def test_every_tile_variant_gives_the_same_solution(dim):
    """The autotuner may pick any tile variant of passes A and E: all must agree."""
    from paper_2105_03297_gb300 import RVE
    n = (64, 64) if dim == 2 else (64, 32, 16)
    E = lognormal(n, 61)
    ns = 3 if dim == 2 else 6
    Cs = []
    for va in range(3):
        for ve in range(3):
            with RVE(n, precision="mixed") as r:
                r.set_schedule(va, ve)
                r.set_material(E, 0.3)
                code, info = r.solve(np.eye(ns), rel_tol=1e-11, max_iter=3000)
                assert code == 0, info
                Cs.append(r.effective_tangent())
                assert r.schedule()[0] == [va, ve, 0, 0]
    for C in Cs[1:]:
        assert rel_max(C, Cs[0]) < 1e-10
    with RVE(n, precision="mixed") as r:
        r.set_material(E, 0.3)
        r.solve(np.eye(ns), rel_tol=1e-11, max_iter=3000)
        var, ms = r.schedule()
        assert var[0] in range(7) and var[1] in range(5) and var[2] in (0, 1) and var[3] in (0, 1)
        # candidate times are those of the last tuning of this handle (zero when the
        # choice came from the per-grid cache of an earlier handle)
        assert len(ms) == 4 and all(len(m) == r.SCHED_VARIANTS and min(m) >= 0 for m in ms)


@pytest.mark.parametrize("n", [(64, 64), (64, 32, 16), (16, 128, 64)])
def test_every_fft_schedule_gives_the_same_operator(n):
    """The autotuner may pick any split of the four-step FFTs (pass C's axis,
    the y axis of passes B / D) and any thread variant of pass A: every
    schedule must apply the same operator q = G C p (FP32, to 2e-5 of the
    oracle's field maximum)."""
    from paper_2105_03297_gb300 import RVE
    dim = len(n)
    E = lognormal(n, 62)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(63).standard_normal((P.m,) + E.shape).astype(np.float32).astype(np.float64)
    ref = P.operator(p)
    scheds = [(a, 0, c, y) for a in range(5 if n[0] >= 64 else 3)
              for c in (0, 1) for y in ((0, 1) if dim == 3 else (0,))]
    with RVE(n, precision="mixed") as r:
        r.set_material(E, 0.3)
        for sch in scheds:
            r.set_schedule(*sch)
            assert r.schedule()[0] == list(sch)
            q = r.apply_operator(p.reshape(P.m, -1)).reshape(ref.shape)
            assert np.abs(q - ref).max() <= 2e-5 * np.abs(ref).max(), sch


@pytest.mark.parametrize("n", [(1024, 32), (512, 64)])
def test_lane_pair_transform_variant(n):
    """Tile variant 5 of the first pass at n_x = 1024 and 512 (each 32-point
    register FFT of the x transform's first step spread over a lane pair)
    applies the same operator as the oracle (FP32, to 2e-5 of the field
    maximum) and runs the same CG as variant 0 (three load cases, C_eff to
    1e-10, and the oracle's to 1e-9)."""
    from paper_2105_03297_gb300 import RVE
    E = lognormal(n, 64)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(65).standard_normal((P.m,) + E.shape).astype(np.float32).astype(np.float64)
    ref = P.operator(p)
    Cs = {}
    for va, ve in ((0, 0), (5, 0)):
        with RVE(n, precision="mixed") as r:
            r.set_schedule(va, ve)
            r.set_material(E, 0.3)
            assert r.schedule()[0][:2] == [va, ve]
            q = r.apply_operator(p.reshape(P.m, -1)).reshape(ref.shape)
            assert np.abs(q - ref).max() <= 2e-5 * np.abs(ref).max(), (va, ve)
            code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=4000)
            assert code == 0, info
            Cs[va, ve] = r.effective_tangent()
    assert rel_max(Cs[5, 0], Cs[0, 0]) < 1e-10
    C_ref, _, _ = P.effective_tangent(np.eye(3), tol=1e-13)
    assert rel_max(Cs[5, 0], C_ref) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_anisotropic_voxels(prec):
    """Cell lengths enter through the voxel sizes h_a = L_a / n_a (Appendix A)."""
    from paper_2105_03297_gb300 import RVE
    n, length = (32, 16), (2.0, 0.5)
    E = lognormal(n, 71)
    C_ref, _, _ = Problem(n, E, 0.3, length=length).effective_tangent(np.eye(3), tol=1e-13)
    with RVE(n, precision=prec, length=length) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9
