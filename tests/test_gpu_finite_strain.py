"""Finite strain (St. Venant-Kirchhoff, Newton-projected CG) on the GPU against
the FP64 finite-strain oracle and its closed forms.

The gradient projection must agree elementwise to FP64 FFT rounding; the mean
first Piola-Kirchhoff stress and the deformation field to 1e-9 of their
largest entry; a laminate under stretch matches its one-dimensional solution.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_stretch
from oracle.finite_strain import FiniteStrainProblem
from tests.gpu_util import lognormal, rel_max, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _rve(n):
    from paper_2105_03297_gb300 import RVE
    r = RVE(n, precision="fp64")
    r.set_kinematics("finite")
    return r


@pytest.mark.parametrize("n", [(32, 64), (16, 32, 16)])
def test_gradient_projection_elementwise(n):
    D = len(n)
    E = lognormal(n, 701)
    P = FiniteStrainProblem(n, E, 0.3)
    A = np.random.default_rng(702).standard_normal((P.nq, D, D) + E.shape)
    ref = P.project(A).reshape(P.nq * D * D, -1)
    with _rve(n) as r:
        field = np.zeros((r.m, E.size))
        field[:P.nq * D * D] = A.reshape(P.nq * D * D, -1)
        q = r.apply_operator(field, material=False)
    assert np.abs(q[:P.nq * D * D] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.all(q[P.nq * D * D:] == 0.0)


@pytest.mark.parametrize("n,Fm", [((64, 64), [[1.1, 0.05], [0.0, 0.95]]),
                                  ((32, 16), [[0.92, -0.08], [0.1, 1.06]]),
                                  ((16, 32, 16), [[1.05, 0.02, 0.0], [0.0, 0.97, 0.04], [-0.03, 0.0, 1.02]])])
def test_solve_matches_oracle(n, Fm):
    E = lognormal(n, 703)
    Fm = np.array(Fm)
    P = FiniteStrainProblem(n, E, 0.3)
    F_ref, steps, _, _ = P.solve(Fm, tol=1e-12)
    Pm_ref = P.mean_stress(F_ref)
    with _rve(n) as r:
        r.set_material(E, 0.3)
        code, info = r.solve_finite(Fm[None], rel_tol=1e-12)
        assert code == 0, info
        Pm = r.mean_piola()[0]
        F = r.get_deformation(0)
    assert rel_max(Pm, Pm_ref) < 1e-9
    Fr = F_ref.reshape(F.shape)
    assert np.abs(F - Fr).max() < 1e-9 * np.abs(Fr).max()
    assert info[0]["refine_steps"] >= 2


@pytest.mark.parametrize("dim", [2, 3])
def test_laminate_stretch(dim):
    n = (32, 16) if dim == 2 else (32, 16, 16)
    layers = np.exp(np.random.default_rng(704).standard_normal(32))
    Fm = np.eye(dim)
    Fm[0, 0] = 1.12
    with _rve(n) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, info = r.solve_finite(Fm[None], rel_tol=1e-12)
        assert code == 0, info
        Pm = r.mean_piola()[0]
    ref = laminate_stretch(layers, 0.3, dim, 1.12)
    assert np.abs(Pm - ref).max() < 1e-9 * np.abs(ref).max()


def test_homogeneous_and_several_load_cases():
    n = (32, 32)
    Fms = np.array([[[1.05, 0.0], [0.0, 1.0]], [[1.0, 0.1], [0.0, 1.0]], [[0.9, 0.0], [0.05, 1.1]]])
    with _rve(n) as r:
        r.set_material(np.full((32, 32), 3.0), 0.3)
        code, info = r.solve_finite(Fms, rel_tol=1e-12)
        assert code == 0 and all(i["refine_steps"] == 0 for i in info)
        Pm = r.mean_piola()
    P = FiniteStrainProblem(n, np.full((32, 32), 3.0), 0.3)
    for l in range(3):
        ref = P.stress(P.broadcast(Fms[l]))[0, :, :, 0, 0]
        assert np.abs(Pm[l] - ref).max() < 1e-13 * np.abs(ref).max()


def test_rules():
    from paper_2105_03297_gb300 import RVE, RveError
    with RVE((32, 32), precision="mixed") as r:
        with pytest.raises(RveError):
            r.set_kinematics("finite")            # FP64 only
    with RVE((16, 16, 256), precision="fp64") as r:
        with pytest.raises(RveError):
            r.set_kinematics("finite")            # n_z <= 128
    with _rve((16, 16)) as r:
        r.set_material(np.ones((16, 16)), 0.3)
        with pytest.raises(RveError):
            r.solve(np.eye(3))                    # small-strain solve refused on a finite handle
        with pytest.raises(RveError):
            r.set_operator_form("nodal")
        r.set_kinematics("small")
        code, _ = r.solve(np.eye(3), rel_tol=1e-10)
        assert code == 0


def test_anisotropic_voxels():
    from paper_2105_03297_gb300 import RVE
    n, length = (32, 16), (2.0, 0.5)
    E = lognormal(n, 705)
    Fm = np.array([[1.07, 0.03], [0.0, 0.96]])
    P = FiniteStrainProblem(n, E, 0.3, length=length)
    F_ref, _, _, _ = P.solve(Fm, tol=1e-12)
    with RVE(n, precision="fp64", length=length) as r:
        r.set_kinematics("finite")
        r.set_material(E, 0.3)
        code, info = r.solve_finite(Fm[None], rel_tol=1e-12)
        assert code == 0, info
        Pm = r.mean_piola()[0]
    assert rel_max(Pm, P.mean_stress(F_ref)) < 1e-9
