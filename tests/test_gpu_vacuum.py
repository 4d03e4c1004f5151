"""Zero-stiffness (vacuum) voxels on the GPU against the FP64 oracle (Sec. 3.2).

E = 0 is accepted by rve_set_material; the solve must give the oracle's
C_eff to 1e-9 and the same strains on every stiff element (those are unique;
strains of vacuum elements are not), in every operator form and precision.
Two pillars cut apart by vacuum columns must not interact, and a homogeneous
pillar must carry the exact uniaxial plane-strain state.
"""
import functools

import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent
from oracle.fe_projection import Problem, lame
from tests.gpu_util import rel_max, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _rve(n, prec, form):
    from paper_2105_03297_gb300 import RVE
    r = RVE(n, precision=prec)
    r.set_operator_form(form)
    return r


@functools.lru_cache(maxsize=None)
def _porous_oracle(n):
    """Oracle C_eff and strain fields of the porous field (shared by the parametrisations)."""
    E = ms.porous_lognormal(n, void_fraction=0.25, seed=501)
    ns = 3 if len(n) == 2 else 6
    C, fields, _ = Problem(n, E, 0.3).effective_tangent(np.eye(ns), tol=1e-13)
    return C, fields


@pytest.mark.parametrize("form", ["stress", "nodal"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(64, 64), (32, 16, 32)])
def test_porous_matches_oracle(n, prec, form):
    E = ms.porous_lognormal(n, void_fraction=0.25, seed=501)
    ns = 3 if len(n) == 2 else 6
    C_ref, fields = _porous_oracle(n)
    stiff = np.broadcast_to(E > 0, fields[0].shape[1:])
    with _rve(n, prec, form) as r:
        r.set_material(E, 0.3)
        code, info = r.solve(np.eye(ns), rel_tol=1e-12, max_iter=8000)
        assert code == 0, info
        C = r.effective_tangent()
        eps0 = r.get_strain(0).reshape(fields[0].shape)
    assert rel_max(C, C_ref) < 1e-9
    d = np.abs(eps0 - fields[0])[:, stiff]
    assert d.max() <= 1e-9 * np.abs(fields[0]).max()


@pytest.mark.parametrize("form", ["stress", "nodal"])
@pytest.mark.parametrize("dim", [2, 3])
def test_vacuum_laminate_closed_form(dim, form):
    n = (32, 16) if dim == 2 else (32, 16, 16)
    layers = np.exp(np.random.default_rng(502).standard_normal(32))
    layers[[5, 20]] = 0.0
    ns = 3 if dim == 2 else 6
    with _rve(n, "mixed", form) as r:
        r.set_material(ms.laminate(n, layers), 0.3)
        code, info = r.solve(np.eye(ns), rel_tol=1e-11, max_iter=4000)
        assert code == 0, info
        C = r.effective_tangent()
    Cref = laminate_tangent(layers, 0.3, dim)
    assert np.abs(C - Cref).max() < 1e-9 * np.abs(Cref).max()


@pytest.mark.parametrize("form", ["stress", "nodal"])
def test_two_pillars_do_not_interact(form):
    n = (64, 32)
    E, A, B = ms.two_pillars(n, E_hard=2.0)
    E2 = E.copy()
    E2[B] = np.exp(np.random.default_rng(503).standard_normal(int(B.sum())))
    Em = np.array([[0.0, 0.1, 0.0]])
    out = []
    for field in (E, E2):
        with _rve(n, "mixed", form) as r:
            r.set_material(field, 0.33)
            code, info = r.solve(Em, rel_tol=1e-12, max_iter=8000)
            assert code == 0, info
            out.append(r.get_strain(0).reshape((6,) + E.shape))
    a = np.abs(out[0] - out[1])[:, A]
    assert a.max() < 1e-9 * np.abs(out[0]).max()
    lam, mu = lame(2.0, 0.33)
    exx = -lam / (lam + 2 * mu) * 0.1
    for q in range(2):
        e = out[0][3 * q:3 * q + 3][:, B]
        assert np.abs(e[0] - exx).max() < 1e-10
        assert np.abs(e[1] - 0.1).max() < 1e-10
        assert np.abs(e[2]).max() < 1e-10


def test_invalid_moduli_are_rejected():
    from paper_2105_03297_gb300 import RVE, RveError
    with RVE((16, 16), precision="mixed") as r:
        with pytest.raises(RveError):
            r.set_material(np.zeros((16, 16)), 0.3)
        bad = np.ones((16, 16))
        bad[2, 3] = -1.0
        with pytest.raises(RveError):
            r.set_material(bad, 0.3)
        ok = np.ones((16, 16))
        ok[:, 4] = 0.0
        r.set_material(ok, 0.3)
