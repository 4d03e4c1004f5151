"""Pins of the oracle for zero-stiffness (vacuum) voxels (Sec. 3.2).

With E = 0 on some voxels the projected operator is only semi-definite; the
oracle's CG runs on its range.  What fixes the answer without the oracle:
* the laminate closed form with vacuum layers (series averages vanish, the
  in-layer terms survive): exact for linear elements;
* the dense FE minimiser with a pseudo-inverse (brute force on tiny grids);
* two bodies cut apart by vacuum columns do not interact (the energy splits),
  and a homogeneous free-standing pillar under a y strain carries the
  uniaxial plane-strain state sigma_xx = sigma_xy = 0 exactly.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent
from oracle.fe_projection import Problem, lame
from oracle.fem_assembly import AssembledFEM


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_vacuum_laminate_closed_form(dim):
    n = (16, 4) if dim == 2 else (12, 4, 4)
    layers = np.exp(np.random.default_rng(31).standard_normal(n[0]))
    layers[[2, 7]] = 0.0
    ns = 3 if dim == 2 else 6
    C, _, _ = Problem(n, ms.laminate(n, layers), 0.3).effective_tangent(np.eye(ns), tol=1e-13)
    Cref = laminate_tangent(layers, 0.3, dim)
    assert Cref[0, 0] == 0.0 and Cref[1, 1] > 0.0
    assert np.abs(C - Cref).max() < 1e-12 * np.abs(Cref).max()


@pytest.mark.parametrize("n", [(16, 16), (6, 6, 6)])
def test_porous_matches_dense_minimiser(n):
    """O1 (projected CG) against K^+ f of the assembled FE system."""
    E = ms.porous_lognormal(n, void_fraction=0.25, seed=32)
    ns = 3 if len(n) == 2 else 6
    P = Problem(n, E, 0.3)
    C, fields, _ = P.effective_tangent(np.eye(ns), tol=1e-13)
    fem = AssembledFEM(n, E, 0.3)
    Kp = np.linalg.pinv(fem.K.toarray(), rcond=1e-11)
    stiff = np.broadcast_to(E > 0, fields[0].shape[1:])
    for l in range(ns):
        u = Kp @ fem.load_vector(np.eye(ns)[l])
        eps = fem.element_strains(np.eye(ns)[l], u)
        assert _rel(fem.mean_stress(eps), C[:, l]) < 1e-12
        # strains of stiff elements are unique
        d = np.abs(eps - fields[l])[:, stiff]
        assert d.max() < 1e-10 * np.abs(fields[l]).max()


def test_two_pillars_do_not_interact():
    n = (32, 16)
    E, A, B = ms.two_pillars(n, E_hard=2.0)
    Em = np.array([0.0, 0.1, 0.0])
    epsA, _, _ = Problem(n, E, 0.33).solve(Em, tol=1e-13)
    E2 = E.copy()
    E2[B] = np.exp(np.random.default_rng(33).standard_normal(int(B.sum())))
    epsB, _, _ = Problem(n, E2, 0.33).solve(Em, tol=1e-13)
    # pillar A does not see what happens in pillar B
    a = np.abs(epsA - epsB)[:, A]
    assert a.max() < 1e-10 * np.abs(epsA).max()
    # the homogeneous pillar B of the first solve is in uniaxial plane strain
    lam, mu = lame(2.0, 0.33)
    M = lam + 2 * mu
    exx = -lam / M * 0.1
    for q in range(2):
        e = epsA[3 * q:3 * q + 3][:, B]
        assert np.abs(e[0] - exx).max() < 1e-12
        assert np.abs(e[1] - 0.1).max() < 1e-12
        assert np.abs(e[2]).max() < 1e-12


def test_all_vacuum_is_trivial():
    P = Problem((8, 8), np.zeros((8, 8)), 0.3)
    eps, it, res = P.solve([0.01, 0.0, 0.0])
    assert it == 0 and np.all(P.mean_stress(eps) == 0.0)
