"""GPU parity of the 3D path (six Kuhn tetrahedra per voxel) against the FP64 oracle.

Every call goes through the C ABI.  Tolerances as in the 2D tests.
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


@pytest.mark.parametrize("n", [(16, 16, 16), (32, 16, 64), (16, 64, 32)])
@pytest.mark.parametrize("material", [True, False])
def test_operator_fp64_elementwise(n, material):
    E = lognormal(n, 21)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(22).standard_normal((P.m,) + E.shape)
    ref = P.operator(p) if material else P.project(p)
    with _rve(n, "fp64") as r:
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1), material=material).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [(16, 16, 16), (64, 32, 16)])
def test_operator_fp32_elementwise(n):
    E = lognormal(n, 23)
    P = Problem(n, E, 0.3)
    p = np.random.default_rng(24).standard_normal((P.m,) + E.shape)
    ref = P.operator(p.astype(np.float32).astype(np.float64))
    with _rve(n, "mixed") as r:
        r.set_material(E, 0.3)
        q = r.apply_operator(p.reshape(P.m, -1).astype(np.float32)).reshape(ref.shape)
    assert np.abs(q - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_effective_tangent_and_field(prec):
    n = (16, 16, 32)
    E = lognormal(n, 25)
    P = Problem(n, E, 0.3)
    C_ref, fields, _ = P.effective_tangent(np.eye(6), tol=1e-13)
    with _rve(n, prec) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-12, max_iter=3000)
        C = r.effective_tangent()
        eps = r.get_strain(2).reshape(fields[2].shape)
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9
    assert np.abs(eps - fields[2]).max() <= 1e-9 * np.abs(fields[2]).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_laminate_closed_form(prec):
    n = (32, 16, 16)
    layers = np.exp(1.0 * np.random.default_rng(26).standard_normal(32))
    with _rve(n, prec) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-10, max_iter=3000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, laminate_tangent(layers, 0.3, 3)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_matches_oracle(prec):
    n = (16, 16, 16)
    E = lognormal(n, 27)
    P = Problem(n, E, 0.3)
    W = np.zeros((6, 6)); W[0, 0] = 1.0; W[3, 3] = 0.5
    g_ref, C_ref = P.adjoint_gradient(W, tol=1e-13)
    with _rve(n, prec) as r:
        r.set_material(E, 0.3)
        r.solve(np.eye(6), rel_tol=1e-12, max_iter=3000)
        g = r.adjoint(W, rel_tol=1e-12, max_iter=3000).reshape(E.shape)
    assert rel_max(g, g_ref) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lognormal64_golden(prec):
    """64^3 log-normal moduli: C_eff and the adjoint gradient of C_1111 at 16
    seeded voxels against the oracle's stored values."""
    path = os.path.join(GOLDEN, "lognormal64.json")
    if not os.path.exists(path):
        pytest.skip("golden not generated")
    ref = json.load(open(path))
    cfg = ms.config_inputs("lognormal64")
    W = np.array(ref["adjoint_W"])
    with _rve(cfg["n"], prec) as r:
        r.set_material(cfg["E"], cfg["nu"])
        code, info = r.solve(np.eye(6), rel_tol=1e-11, max_iter=5000)
        C = r.effective_tangent()
        g = r.adjoint(W, rel_tol=1e-11, max_iter=5000)
    assert code == 0, info
    assert rel_max(C, np.array(ref["C_eff"])) < 1e-9
    gs = g[np.array(ref["adjoint_voxels"])]
    assert rel_max(gs, np.array(ref["adjoint_grad"])) < 1e-9
    assert abs(np.sum(cfg["E"].reshape(-1) * g) - ref["adjoint_euler_sum"]) < 1e-9 * abs(ref["adjoint_euler_sum"])


def test_anisotropic_voxels_3d():
    from paper_2105_03297_gb300 import RVE
    n, length = (16, 32, 16), (1.0, 3.0, 0.25)
    E = lognormal(n, 72)
    C_ref, _, _ = Problem(n, E, 0.3, length=length).effective_tangent(np.eye(6), tol=1e-13)
    with RVE(n, precision="mixed", length=length) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-12, max_iter=3000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9


@pytest.mark.parametrize("form", ["stress", "nodal"])
def test_spheres128_golden(form):
    """128^3 random non-overlapping spheres (r = 6, vf 0.2, contrast 1000), six
    unit load cases: the mean stress of every load case whose oracle solution
    is stored (one file per load case) to 1e-9 of the largest stored entry."""
    parts = {l: os.path.join(GOLDEN, f"spheres128_lc{l}.json") for l in range(6)}
    parts = {l: json.load(open(p)) for l, p in parts.items() if os.path.exists(p)}
    if not parts:
        pytest.skip("golden not generated")
    from paper_2105_03297_gb300 import RVE
    cfg = ms.config_inputs("spheres128")
    with RVE(cfg["n"], precision="mixed") as r:
        r.set_operator_form(form)
        r.set_material(cfg["E"], cfg["nu"])
        code, info = r.solve(np.eye(6), rel_tol=1e-11, max_iter=5000)
        S = r.mean_stress()
    assert code == 0, info
    ref = np.array([parts[l]["mean_stress"] for l in sorted(parts)])
    got = np.array([S[l] for l in sorted(parts)])
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
