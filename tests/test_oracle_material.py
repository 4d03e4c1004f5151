"""Pins of the oracle's material law and Mandel notation against textbook
elasticity written in the engineering constants (E, nu), not through the
Lame constants the oracle (and the laminate closed form) use.

Sec. 3.3 gives E and nu only; the reading is isotropic linear elasticity, plane
strain in 2D.  A slip in lame() or stiffness_mandel() (plane stress instead of
plane strain, a missing factor 2 on mu, a Voigt instead of a Mandel shear)
would cancel between the oracle and the laminate closed form; these checks
fix it from outside.
"""
import numpy as np
import pytest

from oracle.fe_projection import (apply_material, mandel_pairs, mandel_to_tensor, stiffness_mandel,
                                  tensor_to_mandel)


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (210.0, 0.25), (3.5, 0.0), (0.7, 0.45)])
def test_3d_compliance_is_textbook(E, nu):
    S = np.linalg.inv(stiffness_mandel(3, E, nu))
    for i in range(3):
        for j in range(3):
            assert S[i, j] == pytest.approx(1.0 / E if i == j else -nu / E, rel=1e-13, abs=1e-15)
    # Mandel shear components: eps_m = sqrt2 eps_ij, sig_m = sqrt2 sig_ij and eps_ij = (1 + nu) / E sig_ij
    for s in range(3, 6):
        assert S[s, s] == pytest.approx((1.0 + nu) / E, rel=1e-13)
    assert np.abs(S[:3, 3:]).max() == 0.0 and np.abs(S[3:, 3:] - np.diag(np.diag(S[3:, 3:]))).max() == 0.0


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (210.0, 0.25), (0.7, 0.45)])
def test_2d_is_plane_strain(E, nu):
    C2 = stiffness_mandel(2, E, nu)
    S2 = np.linalg.inv(C2)
    # in-plane compliance of plane strain (eps_zz = 0)
    assert S2[0, 0] == pytest.approx((1.0 - nu ** 2) / E, rel=1e-13)
    assert S2[1, 1] == pytest.approx((1.0 - nu ** 2) / E, rel=1e-13)
    assert S2[0, 1] == pytest.approx(-nu * (1.0 + nu) / E, rel=1e-13)
    assert S2[2, 2] == pytest.approx((1.0 + nu) / E, rel=1e-13)
    # the in-plane block (xx, yy, xy) of the 3D stiffness
    C3 = stiffness_mandel(3, E, nu)
    idx = [0, 1, 5]
    assert np.abs(C2 - C3[np.ix_(idx, idx)]).max() <= 1e-14 * np.abs(C3).max()
    # and not plane stress, whose S_xx would be 1/E
    if nu > 0:
        assert abs(S2[0, 0] - 1.0 / E) > 1e-3 / E


@pytest.mark.parametrize("nu", [0.1, 0.3, 0.45])
def test_moduli_of_special_strains(nu):
    E = 2.0
    C = stiffness_mandel(3, E, nu)
    # uniaxial strain: P-wave modulus; hydrostatic strain: 3 K
    assert C[0, 0] == pytest.approx(E * (1 - nu) / ((1 + nu) * (1 - 2 * nu)), rel=1e-13)
    sig = C @ np.array([1.0, 1.0, 1.0, 0, 0, 0])
    assert np.allclose(sig[:3], 3.0 * E / (3.0 * (1 - 2 * nu)), rtol=1e-13) and np.all(sig[3:] == 0)
    # pure shear eps_xy = g: sig_xy = 2 mu g with mu = E / (2 (1 + nu))
    g = 0.01
    sig = C @ tensor_to_mandel(np.array([[0, g, 0], [g, 0, 0], [0, 0, 0.0]]))
    assert mandel_to_tensor(sig, 3)[0, 1] == pytest.approx(E / (1 + nu) * g, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_mandel_pairing_is_frobenius(dim):
    rng = np.random.default_rng(40 + dim)
    A = rng.standard_normal((5, dim, dim)); A = A + np.swapaxes(A, 1, 2)
    B = rng.standard_normal((5, dim, dim)); B = B + np.swapaxes(B, 1, 2)
    a, b = tensor_to_mandel(A), tensor_to_mandel(B)
    assert np.allclose(np.sum(a * b, axis=-1), np.einsum("kij,kij->k", A, B), rtol=1e-14)
    assert np.allclose(mandel_to_tensor(a, dim), A, rtol=0, atol=1e-15)
    assert len(mandel_pairs(dim)) == (3 if dim == 2 else 6)


@pytest.mark.parametrize("n", [(3, 4), (2, 3, 2)])
def test_apply_material_is_per_element(n):
    """sigma = E_v Cbar : eps, element by element (every element of a voxel
    shares the voxel's modulus), against a plain loop over elements and voxels."""
    dim = len(n)
    ns = 3 if dim == 2 else 6
    nq = 2 if dim == 2 else 6
    shape = tuple(reversed(n))
    rng = np.random.default_rng(7)
    E = np.exp(rng.standard_normal(shape))
    eps = rng.standard_normal((nq * ns,) + shape)
    sig = apply_material(eps, E, 0.3)
    Cbar = stiffness_mandel(dim, 1.0, 0.3)
    for q in range(nq):
        for v in np.ndindex(*shape):
            e = eps[q * ns:(q + 1) * ns][(slice(None),) + v]
            assert np.allclose(sig[q * ns:(q + 1) * ns][(slice(None),) + v], E[v] * (Cbar @ e), rtol=1e-14)
