"""Pins of the oracle's projection operator G(k) against what the paper fixes.

Each check is independent of the formula it tests: algebraic identities of a
projection, the literal index form of Appendix B, the textbook Fourier
small-strain projection it reduces to, and the real-space FE strains of O2.
"""
import numpy as np
import pytest

from oracle.closed_forms import appendix_b_projection, textbook_strain_projection
from oracle.fe_projection import (Problem, array_shape, mandel_to_tensor, projection_matrices,
                                  tensor_to_mandel)
from oracle.fem_assembly import AssembledFEM

GRIDS = [(6, 8), (5, 7), (4, 3, 5), (4, 4, 4)]


def _problem(n, seed=0):
    rng = np.random.default_rng(seed)
    return Problem(n, np.exp(rng.standard_normal(array_shape(n))), 0.3)


@pytest.mark.parametrize("n", GRIDS)
def test_projection_algebra(n):
    """G idempotent (Sec. 2.3), self-adjoint (Eq. stat-mech-equi2), rank D, G B = B."""
    P = _problem(n)
    G = projection_matrices(P.B)
    GH = np.conj(np.swapaxes(G, -1, -2))
    assert np.abs(G @ G - G).max() < 1e-13
    assert np.abs(G - GH).max() < 1e-13
    tr = np.trace(G, axis1=-2, axis2=-1)
    k0 = (0,) * P.dim
    assert abs(tr[k0]) == 0.0
    tr = tr.copy()
    tr[k0] = P.dim
    assert np.abs(tr - P.dim).max() < 1e-12
    GB = G @ P.B
    GB[k0] = P.B[k0]
    assert np.abs(GB - P.B).max() < 1e-12 * np.abs(P.B).max()


@pytest.mark.parametrize("n", GRIDS)
def test_hermitian_symmetry_in_k(n):
    """G(-k) = conj G(k) on every wavevector, Nyquist planes included (Sec. 2.7)."""
    P = _problem(n)
    G = projection_matrices(P.B)
    Gm = G
    for ax in range(P.dim):
        Gm = np.roll(np.flip(Gm, axis=ax), 1, axis=ax)   # index -k
    assert np.abs(Gm - np.conj(G)).max() < 1e-13


@pytest.mark.parametrize("n", GRIDS)
def test_appendix_b_index_form(n):
    """The B-form equals the literal small-strain projection of Appendix B."""
    P = _problem(n)
    G = projection_matrices(P.B)
    rng = np.random.default_rng(3)
    D, nq, ns = P.dim, P.nq, P.ns
    ks = [tuple(rng.integers(0, s) for s in array_shape(n)) for _ in range(6)]
    ks = [k for k in ks if any(k)] + [tuple(s // 2 for s in array_shape(n))]
    for k in ks:
        GB = appendix_b_projection(P.g[(slice(None), slice(None)) + k])
        e = rng.standard_normal((nq, D, D)) + 1j * rng.standard_normal((nq, D, D))
        e = 0.5 * (e + np.swapaxes(e, 1, 2))
        out_b = np.einsum("tijLlm,Lml->tij", GB, e)
        out_m = G[k] @ tensor_to_mandel(e).reshape(-1)
        assert np.abs(out_b - mandel_to_tensor(out_m.reshape(nq, ns), D)).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_single_point_fourier_derivative_is_textbook(dim):
    """One evaluation point with D = ik: Appendix B gives the classical projection,
    and h = 1 - g_11/2 (the closed form stated in Appendix B)."""
    rng = np.random.default_rng(dim)
    for _ in range(5):
        kv = rng.standard_normal(dim)
        Dk = (1j * kv)[None, :]
        assert np.abs(appendix_b_projection(Dk)[0, :, :, 0] - textbook_strain_projection(kv)).max() < 1e-14
        g11 = np.outer(Dk[0], np.conj(Dk[0])) / np.sum(np.abs(Dk) ** 2)
        assert np.abs(np.linalg.inv(np.eye(dim) + g11) - (np.eye(dim) - 0.5 * g11)).max() < 1e-14


@pytest.mark.parametrize("n", [(6, 8), (4, 3, 5)])
def test_projection_fixes_real_space_fe_strains(n):
    """Strains of any periodic nodal displacement (O2's shape functions) are
    compatible and mean-free, so G returns them unchanged; G maps a random
    field onto such strains (the idea of Fig. effect_of_G)."""
    P = _problem(n)
    fem = AssembledFEM(n, P.E, P.nu)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(fem.ndof)
    eps = fem.element_strains(np.zeros(P.ns), u)
    assert np.abs(P.project(eps) - eps).max() < 1e-12 * np.abs(eps).max()
    f = rng.standard_normal(eps.shape)
    pf = P.project(f)
    assert np.abs(P.project(pf) - pf).max() < 1e-12
    # the projected field is the least-squares compatible part: f - Gf is
    # orthogonal to every compatible field
    assert abs(np.sum((f - pf) * eps)) < 1e-10 * np.sum(np.abs(f * eps))


def test_mandel_sqrt2_is_required():
    """Dropping the Mandel sqrt2 breaks self-adjointness in the sigma:eps pairing:
    the result must differ from the correct G (guards against that mistake)."""
    n = (6, 8)
    P = _problem(n)
    Bw = P.B.copy()
    Bw[..., 2, :] /= np.sqrt(2.0)
    Bw[..., 5, :] /= np.sqrt(2.0)
    Gw = projection_matrices(Bw)
    G = projection_matrices(P.B)
    assert np.abs(Gw - G).max() > 1e-3
