"""Pins of the oracle's adjoint gradient dJ/dE_v for J = W : C_eff.

Checked against central finite differences of C_eff computed by the
independent assembled FEM (O2), and against Euler's identity: C_eff is
homogeneous of degree one in the moduli at fixed nu, so
sum_v E_v dJ/dE_v = J exactly.
"""
import numpy as np
import pytest

from oracle.fe_projection import Problem, array_shape
from oracle.fem_assembly import AssembledFEM


@pytest.mark.parametrize("n", [(6, 6), (3, 4, 3)])
def test_adjoint_vs_finite_differences(n):
    rng = np.random.default_rng(7)
    E = np.exp(rng.standard_normal(array_shape(n)))
    P = Problem(n, E, 0.3)
    ns = P.ns
    W = np.zeros((ns, ns))
    W[0, 0] = 1.0
    W[1, 0] = W[0, 1] = 0.5
    grad, C = P.adjoint_gradient(W, tol=1e-14)
    # Euler identity
    J = float(np.sum(W * C))
    assert abs(np.sum(E * grad) - J) < 1e-11 * abs(J)
    # central differences with O2, relative step h = 1e-6
    h = 1e-6
    flat = E.reshape(-1)
    for v in rng.choice(flat.size, size=4, replace=False):
        Ep = flat.copy(); Ep[v] *= 1 + h
        Em = flat.copy(); Em[v] *= 1 - h
        Cp, _ = AssembledFEM(n, Ep.reshape(E.shape), 0.3).effective_tangent(np.eye(ns))
        Cm, _ = AssembledFEM(n, Em.reshape(E.shape), 0.3).effective_tangent(np.eye(ns))
        fd = (np.sum(W * Cp) - np.sum(W * Cm)) / (2 * h * flat[v])
        # FD rounding ~ 1e-16 * J / (2h E_v); truncation O(h^2)
        assert abs(fd - grad.reshape(-1)[v]) < 1e-5 * abs(fd) + 1e-9


def test_adjoint_c1111_gradient_is_positive():
    """Stiffening any voxel cannot soften C_1111 (energy minimisation)."""
    n = (4, 4, 4)
    E = np.exp(np.random.default_rng(3).standard_normal(array_shape(n)))
    P = Problem(n, E, 0.3)
    W = np.zeros((6, 6)); W[0, 0] = 1.0
    grad, C = P.adjoint_gradient(W, tol=1e-13)
    assert grad.min() > 0.0
    assert abs(np.sum(E * grad) - C[0, 0]) < 1e-11 * C[0, 0]
