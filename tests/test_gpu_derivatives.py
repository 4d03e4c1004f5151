"""The other discrete derivatives (Secs. 2.3-2.5, Appendix C) on the GPU against
the FP64 oracle with the same derivative.

rve_set_derivative changes B(k) and n_q; the solve is the plain projected CG
on the strain fluctuation in FP64, which is exactly the oracle's scheme, so
the operator must agree elementwise to FP64 FFT rounding (1e-12 of the field
maximum) and C_eff / strain fields to 1e-9.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent
from oracle.fe_projection import Problem
from tests.gpu_util import lognormal, rel_max, require_gpu

pytestmark = pytest.mark.gpu

DERIVS_2D = ["fourier", "central", "forward", "lsq", "fourier2"]
DERIVS_3D = ["fourier", "central", "forward", "lsq"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _rve(n, derivative):
    from paper_2105_03297_gb300 import RVE
    r = RVE(n, precision="fp64")
    r.set_derivative(derivative)
    return r


@pytest.mark.parametrize("material", [True, False])
@pytest.mark.parametrize("derivative,n", [(d, (32, 64)) for d in DERIVS_2D] + [(d, (16, 32, 16)) for d in DERIVS_3D])
def test_operator_elementwise(derivative, n, material):
    E = lognormal(n, 601)
    P = Problem(n, E, 0.3, derivative=derivative)
    p = np.random.default_rng(602).standard_normal((P.m,) + E.shape)
    ref = P.operator(p) if material else P.project(p)
    with _rve(n, derivative) as r:
        assert r.derivative() == derivative and r.m == P.m
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1), material=material).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("derivative,n", [(d, (64, 64)) for d in DERIVS_2D] + [(d, (32, 16, 32)) for d in DERIVS_3D])
def test_tangent_and_field_match_oracle(derivative, n):
    E = lognormal(n, 603, sigma=1.2)
    ns = 3 if len(n) == 2 else 6
    P = Problem(n, E, 0.3, derivative=derivative)
    C_ref, fields, _ = P.effective_tangent(np.eye(ns), tol=1e-13)
    with _rve(n, derivative) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(ns), rel_tol=1e-12, max_iter=6000)
        assert code == 0, info
        C = r.effective_tangent()
        eps1 = r.get_strain(1).reshape(fields[1].shape)
    assert rel_max(C, C_ref) < 1e-9
    assert np.abs(eps1 - fields[1]).max() <= 1e-9 * np.abs(fields[1]).max()


@pytest.mark.parametrize("derivative", ["forward", "lsq"])
@pytest.mark.parametrize("dim", [2, 3])
def test_laminate_is_exact(derivative, dim):
    n = (32, 16) if dim == 2 else (32, 16, 16)
    layers = np.exp(np.random.default_rng(604).standard_normal(32))
    ns = 3 if dim == 2 else 6
    with _rve(n, derivative) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, info = r.solve(np.eye(ns), rel_tol=1e-12, max_iter=4000)
        assert code == 0, info
        C = r.effective_tangent()
    assert rel_max(C, laminate_tangent(layers, 0.3, dim)) < 1e-9


def test_rules_and_switching_back():
    from paper_2105_03297_gb300 import RVE, RveError
    n = (32, 32)
    E = lognormal(n, 605)
    with RVE(n, precision="mixed") as r:
        with pytest.raises(RveError):
            r.set_derivative("fourier")          # non-FE derivatives are FP64 only
    with RVE((16, 16, 16), precision="fp64") as r:
        with pytest.raises(RveError):
            r.set_derivative("fourier2")         # two evaluation points: 2D only
    with RVE(n, precision="fp64") as r:
        r.set_material(E, 0.3)
        r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        C_fe = r.effective_tangent()
        r.set_derivative("forward")
        with pytest.raises(RveError):
            r.effective_tangent()                # the solution was dropped
        with pytest.raises(RveError):
            r.set_operator_form("nodal")         # factored/nodal forms need the FE stencil
        r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        with pytest.raises(RveError):
            r.adjoint(np.eye(3), rel_tol=1e-10, max_iter=100)
        r.set_derivative("fe")
        r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        assert rel_max(r.effective_tangent(), C_fe) < 1e-13


@pytest.mark.parametrize("derivative", ["fourier", "lsq"])
def test_anisotropic_voxels(derivative):
    """Cell lengths enter the symbols through h_a = L_a / n_a."""
    from paper_2105_03297_gb300 import RVE
    n, length = (32, 16), (2.0, 0.5)
    E = lognormal(n, 606)
    C_ref, _, _ = Problem(n, E, 0.3, length=length, derivative=derivative).effective_tangent(np.eye(3), tol=1e-13)
    with RVE(n, precision="fp64", length=length) as r:
        r.set_derivative(derivative)
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=4000)
        assert code == 0, info
        C = r.effective_tangent()
    assert rel_max(C, C_ref) < 1e-9
