"""The factored and nodal-state forms of the projected CG against the FP64 oracle.

RVE_FORM_FACTORED evaluates G C p as B_r K^-1 B_r^T (C p): nodal forces by the
element stencils in real space, FFTs of the D nodal components only, the
inverse normal matrix (B^H B)^-1 per wavevector (Eqs. small-strain-eq2 and
small-strain-chi), strains by the stencils again.  RVE_FORM_NODAL runs the
same CG on nodal fields (x = B xi, r = B rho, p = B pi).  Both are the same
operator and the same CG as the default stress form, so every solve must
reach the oracle's C_eff and strain field to the same 1e-9, and the CG must
take about as many iterations.  Grid sizes cover tiles smaller than the
stencil tile (16 per axis), several tiles per axis and anisotropic voxels.
"""
import json
import os

import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent
from oracle.fe_projection import Problem
from tests.gpu_util import lognormal, oracle_tangent, rel_max, require_gpu

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


FORMS = ["factored", "nodal"]


def _factored(n, prec, form, length=None):
    from paper_2105_03297_gb300 import RVE
    r = RVE(n, precision=prec, length=length)
    r.set_operator_form(form)
    return r


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 16), (64, 32), (512, 64), (1024, 32)])
@pytest.mark.parametrize("form", FORMS)
def test_2d_tangent_matches_oracle(prec, n, form):
    E = lognormal(n, 401, sigma=1.2)
    C_ref = oracle_tangent(n, 401, 1.2)
    with _factored(n, prec, form) as r:
        assert r.operator_form() == form
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(3), rel_tol=1e-12, max_iter=4000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 16, 16), (64, 16, 32), (32, 32, 32)])
@pytest.mark.parametrize("form", FORMS)
def test_3d_tangent_matches_oracle(prec, n, form):
    E = lognormal(n, 402)
    C_ref = oracle_tangent(n, 402)
    with _factored(n, prec, form) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-12, max_iter=4000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", FORMS)
def test_strain_field_matches_oracle(dim, form):
    n = (32, 64) if dim == 2 else (16, 32, 16)
    E = lognormal(n, 403)
    P = Problem(n, E, 0.3)
    Em = np.array([0.01, -0.004, 0.003]) if dim == 2 else np.array([0.01, -0.004, 0.002, 0.003, -0.001, 0.002])
    eps_ref, _, _ = P.solve(Em, tol=1e-13)
    with _factored(n, "mixed", form) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(Em[None], rel_tol=1e-12, max_iter=4000)
        eps = r.get_strain(0).reshape(eps_ref.shape)
    assert code == 0, info
    assert np.abs(eps - eps_ref).max() <= 1e-9 * np.abs(eps_ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_same_iterates_as_stress_form(dim):
    """Same operator, same CG: the tangents agree well below the parity bar and
    the slowest load case takes about as many iterations (at most).  (Per load case the
    totals may differ by a whole inner solve: the FP64 outer residual can land
    on either side of rel_tol after the first one.)"""
    from paper_2105_03297_gb300 import RVE
    n = (128, 64) if dim == 2 else (32, 32, 16)
    ns = 3 if dim == 2 else 6
    E = lognormal(n, 404, sigma=1.5)
    out = {}
    with RVE(n, precision="fp64") as r:
        r.set_material(E, 0.3)
        for form in ("stress", "factored", "nodal", "stress"):
            r.set_operator_form(form)
            code, info = r.solve(np.eye(ns), rel_tol=1e-11, max_iter=4000)
            assert code == 0, info
            out.setdefault(form, []).append((r.effective_tangent(), [i["iterations"] for i in info]))
    (Cs, its) = out["stress"][0]
    for form in FORMS:
        Cf, itf = out[form][0]
        assert rel_max(Cf, Cs) < 1e-10, form
        # never slower than the stress form; the nodal state may need fewer
        # iterations (its iterates stay exactly compatible under rounding)
        assert max(itf) <= 1.05 * max(its) + 8, (form, its, itf)
        if form == "factored":
            assert max(its) <= 1.05 * max(itf) + 8, (form, its, itf)
    # switching back gives the stress form's result again
    assert rel_max(out["stress"][1][0], Cs) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("form", FORMS)
def test_laminate_closed_form_3d(prec, form):
    n = (32, 16, 16)
    layers = np.exp(1.0 * np.random.default_rng(405).standard_normal(32))
    with _factored(n, prec, form) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-10, max_iter=4000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, laminate_tangent(layers, 0.3, 3)) < 1e-9


@pytest.mark.parametrize("form", FORMS)
def test_anisotropic_voxels(form):
    n, length = (32, 16, 16), (2.0, 0.5, 1.0)
    E = lognormal(n, 406)
    C_ref, _, _ = Problem(n, E, 0.3, length=length).effective_tangent(np.eye(6), tol=1e-13)
    with _factored(n, "mixed", form, length=length) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(6), rel_tol=1e-12, max_iter=4000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, C_ref) < 1e-9


@pytest.mark.parametrize("form", FORMS)
def test_adjoint_matches_oracle(form):
    n = (32, 16)
    E = lognormal(n, 407)
    P = Problem(n, E, 0.3)
    W = np.array([[1.0, 0.2, 0.0], [0.2, 0.5, 0.0], [0.0, 0.0, 0.3]])
    g_ref, _ = P.adjoint_gradient(W, tol=1e-13)
    with _factored(n, "mixed", form) as r:
        r.set_material(E, 0.3)
        r.solve(np.eye(3), rel_tol=1e-12, max_iter=3000)
        g = r.adjoint(W, rel_tol=1e-12, max_iter=3000).reshape(E.shape)
    assert rel_max(g, g_ref) < 1e-9


@pytest.mark.parametrize("form", FORMS)
def test_lognormal64_golden(form):
    ref = json.load(open(os.path.join(GOLDEN, "lognormal64.json")))
    cfg = ms.config_inputs("lognormal64")
    with _factored(cfg["n"], "mixed", form) as r:
        r.set_material(cfg["E"], cfg["nu"])
        code, info = r.solve(np.eye(6), rel_tol=1e-11, max_iter=5000)
        C = r.effective_tangent()
    assert code == 0, info
    assert rel_max(C, np.array(ref["C_eff"])) < 1e-9


def test_unknown_form_is_rejected():
    from paper_2105_03297_gb300 import RVE
    from paper_2105_03297_gb300._rve import load
    with RVE((16, 16), precision="mixed") as r:
        assert r.operator_form() == "stress"
        assert load().rve_set_operator_form(r.h, 7) != 0
        with pytest.raises(KeyError):
            r.set_operator_form("spectral")
        assert r.operator_form() == "stress"
