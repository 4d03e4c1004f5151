"""Pins of the finite-strain oracle (O3, St. Venant-Kirchhoff; Eqs. def-grad,
original-G, discrete_projection_op, stat-mech-equi-FFT-homogenization).

What fixes it without O3 itself:
* the projection is, row by row of F, the least-squares gradient part for the
  element gradients of O2's real-space shape functions (dense lstsq);
* the law: tangent = central differences of the stress; frame indifference
  P(R F) = R P(F);
* a homogeneous cell is exact with no iteration; at strains of 1e-6 the mean
  stress is O1's small-strain C_eff applied to the strain;
* a grid-aligned laminate stretched along x matches its one-dimensional
  solution (closed_forms.laminate_stretch); rotating F_macro rotates the mean
  stress of a heterogeneous cell;
* the whole solve equals a Newton solve of the periodic finite-strain FE
  problem assembled in real space (fem_assembly.finite_strain_fem).
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_stretch
from oracle.fe_projection import Problem, array_shape, voxel_size
from oracle.fem_assembly import element_vertices, shape_function_gradients
from oracle.finite_strain import FiniteStrainProblem


def _rot(dim, t):
    if dim == 2:
        return np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    a = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K


def _scalar_gradient_operator(n):
    """Dense map from nodal scalars to element gradients (n_q * D * N) x N,
    rows ordered (element, component a, voxel) with x fastest; periodic nodes."""
    D = len(n)
    h = np.array(voxel_size(n))
    N = int(np.prod(n))
    idx = np.array(np.unravel_index(np.arange(N), array_shape(n))[::-1]).T   # (N, D) as (x, y[, z])
    strides = np.array([int(np.prod(n[:a])) for a in range(D)])
    rows = []
    for verts in element_vertices(D):
        grads, _ = shape_function_gradients(verts * h)                        # (D+1, D)
        G = np.zeros((D, N, N))
        for v, off in enumerate(verts):
            nodes = ((idx + off[None, :]) % np.array(n)[None, :]) @ strides
            for a in range(D):
                G[a, np.arange(N), nodes] += grads[v, a]
        rows.append(G.reshape(D * N, N))
    return np.vstack(rows)


@pytest.mark.parametrize("n", [(6, 5), (4, 3, 5)])
def test_projection_is_least_squares_gradient_part(n):
    D = len(n)
    P = FiniteStrainProblem(n, np.ones(array_shape(n)), 0.3)
    A = np.random.default_rng(51).standard_normal((P.nq, D, D) + array_shape(n))
    GA = P.project(A)
    Bs = _scalar_gradient_operator(n)
    for i in range(D):
        f = A[:, i].reshape(-1)                       # (element, a, voxel) order
        ref = Bs @ np.linalg.lstsq(Bs, f, rcond=1e-10)[0]
        assert np.abs(GA[:, i].reshape(-1) - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_law_tangent_and_frame_indifference(dim):
    n = (4, 4) if dim == 2 else (3, 3, 3)
    rng = np.random.default_rng(52)
    P = FiniteStrainProblem(n, np.exp(rng.standard_normal(array_shape(n))), 0.3)
    shape = (P.nq, dim, dim) + array_shape(n)
    F = np.eye(dim)[None, :, :, *([None] * dim)] + 0.2 * rng.standard_normal(shape)
    dF = rng.standard_normal(shape)
    h = 1e-6
    fd = (P.stress(F + h * dF) - P.stress(F - h * dF)) / (2 * h)
    assert np.abs(P.tangent(F, dF) - fd).max() < 1e-7 * np.abs(fd).max()
    R = _rot(dim, 0.7)
    RF = np.einsum("ij,qjk...->qik...", R, F)
    assert np.abs(P.stress(RF) - np.einsum("ij,qjk...->qik...", R, P.stress(F))).max() < 1e-12


def test_homogeneous_cell_and_small_strain_limit():
    n = (8, 8)
    Fm = np.array([[1.08, 0.03], [-0.02, 0.97]])
    P = FiniteStrainProblem(n, np.full(array_shape(n), 2.0), 0.3)
    F, steps, its, _ = P.solve(Fm)
    assert steps == 0 and np.abs(F - P.broadcast(Fm)).max() == 0.0
    E = np.exp(np.random.default_rng(53).standard_normal(array_shape(n)))
    C, _, _ = Problem(n, E, 0.3).effective_tangent(np.eye(3), tol=1e-13)
    Pf = FiniteStrainProblem(n, E, 0.3)
    eps = 1e-6
    H = np.array([[0.3, 0.4], [0.4, -0.2]])        # symmetric small strain
    Fs, _, _, _ = Pf.solve(np.eye(2) + eps * H, tol=1e-12)
    Pm = Pf.mean_stress(Fs) / eps
    sig = C @ np.array([H[0, 0], H[1, 1], np.sqrt(2) * H[0, 1]])
    assert np.abs(np.array([Pm[0, 0], Pm[1, 1], np.sqrt(2) * Pm[0, 1]]) - sig).max() < 1e-5 * np.abs(sig).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_laminate_stretch(dim):
    n = (8, 4) if dim == 2 else (8, 4, 4)
    layers = np.exp(np.random.default_rng(54).standard_normal(8))
    Fm = np.eye(dim)
    Fm[0, 0] = 1.12
    P = FiniteStrainProblem(n, ms.laminate(n, layers), 0.3)
    F, steps, _, res = P.solve(Fm, tol=1e-12)
    ref = laminate_stretch(layers, 0.3, dim, 1.12)
    assert np.abs(P.mean_stress(F) - ref).max() < 1e-10 * np.abs(ref).max()


def test_rotated_load_rotates_mean_stress():
    n = (8, 8)
    E = np.exp(np.random.default_rng(55).standard_normal(array_shape(n)))
    P = FiniteStrainProblem(n, E, 0.3)
    Fm = np.array([[1.1, 0.05], [0.0, 0.95]])
    R = _rot(2, 0.4)
    F1, _, _, _ = P.solve(Fm, tol=1e-12)
    F2, _, _, _ = P.solve(R @ Fm, tol=1e-12)
    assert np.abs(P.mean_stress(F2) - R @ P.mean_stress(F1)).max() < 1e-9 * np.abs(P.mean_stress(F1)).max()


@pytest.mark.parametrize("n,Fm,length", [((6, 5), [[1.1, 0.05], [-0.02, 0.95]], None),
                                         ((6, 5), [[1.1, 0.05], [-0.02, 0.95]], (2.0, 0.6)),
                                         ((3, 4, 3), [[1.06, 0.02, 0.0], [0.0, 0.97, 0.03], [-0.02, 0.0, 1.03]],
                                          None)])
def test_equals_real_space_finite_strain_fem(n, Fm, length):
    """O3 (projection, Fourier space) against a Newton solve of the assembled
    periodic finite-strain FE problem in real space (O2's shape functions),
    on cubic and on non-cubic voxels."""
    from oracle.fem_assembly import finite_strain_fem
    E = np.exp(np.random.default_rng(56).standard_normal(array_shape(n)))
    P = FiniteStrainProblem(n, E, 0.3, length=length)
    F, _, _, _ = P.solve(np.array(Fm), tol=1e-13)
    F_fem, P_fem, steps = finite_strain_fem(n, E, 0.3, Fm, length=length)
    assert steps >= 2
    assert np.abs(P.mean_stress(F) - P_fem).max() < 1e-11 * np.abs(P_fem).max()
    assert np.abs(F.reshape(F_fem.shape) - F_fem).max() < 1e-10
