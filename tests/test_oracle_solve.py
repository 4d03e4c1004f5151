"""Pins of the oracle's projected-CG solve and homogenisation.

The projected solve (O1) is checked against the assembled periodic FEM (O2),
a dense brute-force minimiser, closed forms (homogeneous material, laminate),
energy bounds and the size-independent convergence the paper states.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent, voigt_reuss
from oracle.fe_projection import Problem, array_shape, stiffness_mandel
from oracle.fem_assembly import AssembledFEM, dense_minimiser


def _lognormal(n, seed):
    return np.exp(np.random.default_rng(seed).standard_normal(array_shape(n)))


@pytest.mark.parametrize("n", [(6, 8), (7, 5), (4, 3, 5)])
def test_projected_cg_equals_assembled_fem(n):
    """Sec. 2.6: the FE projection is identical to conforming linear FE."""
    E = _lognormal(n, 1)
    P = Problem(n, E, 0.3)
    I = np.eye(P.ns)
    C1, f1, _ = P.effective_tangent(I, tol=1e-13)
    fem = AssembledFEM(n, E, 0.3)
    C2, f2 = fem.effective_tangent(I)
    assert np.abs(C1 - C2).max() <= 1e-12 * np.abs(C2).max()
    for a, b in zip(f1, f2):
        assert np.abs(a - b).max() < 1e-11


@pytest.mark.parametrize("n,length", [((6, 8), (2.0, 0.5)), ((5, 4), (0.3, 1.7)), ((4, 3, 5), (1.0, 3.0, 0.7))])
def test_projected_cg_equals_assembled_fem_on_anisotropic_voxels(n, length):
    """Cell lengths enter O1 only through h_a = L_a / n_a in the element symbols
    (Appendix A grid) and O2 only through the vertex coordinates of its
    elements; both must give the same solution on non-cubic voxels."""
    E = _lognormal(n, 3)
    P = Problem(n, E, 0.3, length=length)
    I = np.eye(P.ns)
    C1, f1, _ = P.effective_tangent(I, tol=1e-13)
    fem = AssembledFEM(n, E, 0.3, length=length)
    C2, f2 = fem.effective_tangent(I)
    assert np.abs(C1 - C2).max() <= 1e-12 * np.abs(C2).max()
    for a, b in zip(f1, f2):
        assert np.abs(a - b).max() < 1e-11
    # and the voxel shape matters: the unit-cell answer is different
    C0, _, _ = Problem(n, E, 0.3).effective_tangent(I, tol=1e-13)
    assert np.abs(C0 - C1).max() > 1e-3 * np.abs(C1).max()


@pytest.mark.parametrize("n", [(3, 4), (2, 3, 2)])
def test_fem_equals_dense_minimiser(n):
    E = _lognormal(n, 2)
    fem = AssembledFEM(n, E, 0.25)
    Em = np.linspace(0.3, -0.2, fem.ns)
    u = fem.solve(Em)
    assert np.abs(fem.element_strains(Em, u) - dense_minimiser(n, E, 0.25, Em)).max() < 1e-11
    # the solution minimises the energy: random perturbations raise it
    rng = np.random.default_rng(0)
    e0 = fem.energy(Em, u)
    for _ in range(3):
        assert fem.energy(Em, u + 1e-3 * rng.standard_normal(u.shape)) > e0


@pytest.mark.parametrize("n", [(8, 8), (4, 4, 4)])
def test_homogeneous_material_is_exact(n):
    """k = 0 carries E (Sec. 2.3): a homogeneous cell needs no iteration."""
    P = Problem(n, np.full(array_shape(n), 2.5), 0.3)
    Em = np.arange(1, P.ns + 1) * 0.01
    eps, it, _ = P.solve(Em)
    assert it == 0
    assert np.abs(eps - P.broadcast_macro(Em)).max() == 0.0
    C, _, _ = P.effective_tangent(np.eye(P.ns))
    assert np.abs(C - stiffness_mandel(P.dim, 2.5, 0.3)).max() < 1e-14 * 10


@pytest.mark.parametrize("n", [(8, 4), (16, 6), (8, 2, 3), (6, 3, 2)])
def test_laminate_closed_form(n):
    """A grid-aligned laminate is represented exactly by linear elements."""
    rng = np.random.default_rng(n[0] + len(n))
    layers = np.exp(2.0 * rng.standard_normal(n[0]))
    P = Problem(n, ms.laminate(n, layers), 0.3)
    C, _, _ = P.effective_tangent(np.eye(P.ns), tol=1e-14)
    ref = laminate_tangent(layers, 0.3, P.dim)
    assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [(16, 16), (6, 5, 4)])
def test_bounds_symmetry_homogeneity(n):
    E = _lognormal(n, 5)
    P = Problem(n, E, 0.3)
    C, _, _ = P.effective_tangent(np.eye(P.ns), tol=1e-13)
    V, R = voigt_reuss(E, 0.3, P.dim)
    assert np.linalg.eigvalsh(V - C).min() > -1e-12
    assert np.linalg.eigvalsh(C - R).min() > -1e-12
    assert np.abs(C - C.T).max() < 1e-10 * np.abs(C).max()
    P2 = Problem(n, 3.0 * E, 0.3)
    C2, _, _ = P2.effective_tangent(np.eye(P.ns), tol=1e-13)
    assert np.abs(C2 - 3.0 * C).max() < 1e-10 * np.abs(C2).max()
    # energy form equals the mean-stress form at the converged solution
    _, fields, _ = P.effective_tangent(np.eye(P.ns), tol=1e-13)
    Ce = np.array([[P.energy_form(fields[a], fields[b]) for b in range(P.ns)] for a in range(P.ns)])
    assert np.abs(Ce - C).max() < 1e-10 * np.abs(C).max()


def test_iteration_count_independent_of_grid_size():
    """Sec. 2.6: the condition number does not grow with the system size."""
    its = []
    for s in (16, 32, 64):
        n = (s, s)
        P = Problem(n, ms.circular_inclusion(n, 0.25, 10.0, 1.0), 0.3)
        _, it, _ = P.solve([0.01, 0.0, 0.0], tol=1e-10)
        its.append(it)
    assert max(its) - min(its) <= 4, its


def test_disc32_matches_fem():
    """The 32x32 disc workload: O1 and O2 agree on C_eff."""
    cfg = ms.config_inputs("disc32")
    P = Problem(cfg["n"], cfg["E"], cfg["nu"])
    C1, _, _ = P.effective_tangent(np.eye(3), tol=1e-13)
    C2, _ = AssembledFEM(cfg["n"], cfg["E"], cfg["nu"]).effective_tangent(np.eye(3))
    assert np.abs(C1 - C2).max() <= 1e-12 * np.abs(C2).max()


def test_residual_history_records_each_iteration():
    """The history a solve records is ||r_k|| / ||r_0||: it starts at 1, has one
    entry per iteration, ends at the returned residual, and only its last entry
    is at or below the tolerance.  A residual history recomputed from the
    iterate (r_k = -A(E + eps~_k)) after k steps agrees with it."""
    n = (8, 6)
    E = _lognormal(n, 7)
    P = Problem(n, E, 0.3)
    Em = np.array([1.0, 0.0, 0.0])
    hist = []
    eps, it, res = P.solve(Em, tol=1e-10, history=hist)
    assert len(hist) == it + 1 and hist[0] == 1.0 and hist[-1] == res
    assert hist[-1] <= 1e-10 and min(hist[:-1]) > 1e-10
    k = it // 2
    h2 = []
    eps_k, _, _ = P.solve(Em, tol=0.0, maxit=k, history=h2)
    assert h2 == hist[:k + 1]
    r0 = P.operator(P.broadcast_macro(Em))
    rk = P.operator(eps_k)
    assert abs(np.linalg.norm(rk) / np.linalg.norm(r0) - hist[k]) < 1e-8
