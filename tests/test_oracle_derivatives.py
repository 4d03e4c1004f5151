"""Pins of the oracle's other discrete derivatives (Secs. 2.3-2.5, Appendix C).

Each derivative only changes B(k); what fixes it without the oracle:
* the projection is the least-squares compatible part for the real-space
  derivative written out from its stencil (Eqs. central-difference-derivative-
  real and the forward / least-squares stencils of Secs. 2.4-2.5), or, for the
  Fourier derivative on odd grids, from the trigonometric (Dirichlet-kernel)
  interpolant, evaluated at the voxel centre or, for the two evaluation points
  of Appendix C, shifted by -+(h_x, h_y)/6; dense least squares on tiny grids;
* structural properties of a projection (idempotent, self-adjoint, real);
* forward differences and least squares reproduce the laminate closed form
  exactly (u depends on x only, and both stencils then give the exact
  per-voxel strain), homogeneous material needs no iteration, Voigt/Reuss.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import laminate_tangent, voigt_reuss
from oracle.fe_projection import DERIVATIVES, Problem, array_shape

SQ2 = np.sqrt(2.0)


def _shift(nn, s):
    """Periodic shift matrix: (S u)_i = u_{i+s}."""
    return np.roll(np.eye(nn), s, axis=1)


def _dirichlet(nn, x):
    """Trigonometric interpolation kernel of an odd grid of nn points on [0, 2 pi)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = np.abs(np.sin(x / 2)) > 1e-15
    out[nz] = np.sin(nn * x[nz] / 2) / (nn * np.sin(x[nz] / 2))
    return out


def _dirichlet_prime(nn, x):
    x = np.asarray(x, dtype=np.float64)
    s, c = np.sin(x / 2), np.cos(x / 2)
    out = np.zeros_like(x)
    nz = np.abs(s) > 1e-15
    xs = x[nz]
    out[nz] = ((nn / 2) * np.cos(nn * xs / 2) * s[nz] - 0.5 * np.sin(nn * xs / 2) * c[nz]) / (nn * s[nz] ** 2)
    return out


def _axis_ops(derivative, nn, h, delta=0.0):
    """(derivative matrix, interpolation matrix) along one axis, real space."""
    I = np.eye(nn)
    if derivative == "forward":
        return (_shift(nn, 1) - I) / h, I
    if derivative == "central":
        return (_shift(nn, 1) - _shift(nn, -1)) / (2 * h), I
    if derivative in ("fourier", "fourier2"):
        assert nn % 2 == 1
        i = np.arange(nn)
        x = 2 * np.pi * ((i[:, None] - i[None, :]) + delta) / nn    # grid coordinate differences
        return _dirichlet_prime(nn, x) * (2 * np.pi / (nn * h)), _dirichlet(nn, x)
    raise ValueError(derivative)


def _kron(mats):
    """Operator on x-fastest flattened fields from per-axis matrices [x, y(, z)]."""
    out = mats[-1]
    for M in reversed(mats[:-1]):
        out = np.kron(out, M)
    return out


def _gradient_ops(derivative, n, delta=0.0, length=None):
    """Dense d/dx_a, a < D, on x-fastest flattened grids (cell edge lengths
    ``length``, unit cell by default; voxel size h_a = L_a / n_a)."""
    D = len(n)
    length = length or (1.0,) * D
    h = [L / v for L, v in zip(length, n)]
    ops = []
    for a in range(D):
        mats = []
        for b in range(D):
            if derivative == "lsq":
                I = np.eye(n[b])
                mats.append((_shift(n[b], 1) - I) / h[b] if b == a else 0.5 * (I + _shift(n[b], 1)))
            else:
                Dm, Tm = _axis_ops(derivative, n[b], h[b], delta)
                mats.append(Dm if b == a else Tm)
        ops.append(_kron(mats))
    return ops


def _strain_operator(ops):
    """Dense Mandel sym-gradient B_r: (n_s N) x (D N), component-major."""
    D = len(ops)
    N = ops[0].shape[0]
    Z = np.zeros((N, N))
    rows = []
    pairs = [(0, 0), (1, 1), (0, 1)] if D == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for (a, b) in pairs:
        blocks = [Z] * D
        if a == b:
            blocks = [ops[a] if j == a else Z for j in range(D)]
        else:
            blocks = [ops[b] / SQ2 if j == a else (ops[a] / SQ2 if j == b else Z) for j in range(D)]
        rows.append(np.hstack(blocks))
    return np.vstack(rows)


@pytest.mark.parametrize("derivative,n", [("forward", (6, 5)), ("central", (5, 7)), ("lsq", (6, 4)),
                                          ("fourier", (5, 7)), ("forward", (4, 3, 5)), ("central", (3, 5, 3)),
                                          ("lsq", (4, 4, 3)), ("fourier", (3, 5, 3))])
def test_projection_is_least_squares_compatible_part(derivative, n):
    ops = _gradient_ops(derivative, n)
    Br = _strain_operator(ops)
    P = Problem(n, np.ones(array_shape(n)), 0.3, derivative=derivative)
    f = np.random.default_rng(41).standard_normal((P.m,) + array_shape(n))
    ref = Br @ np.linalg.lstsq(Br, f.reshape(-1), rcond=1e-10)[0]
    assert np.abs(P.project(f).reshape(-1) - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("derivative,n,length", [("forward", (6, 5), (2.0, 0.5)), ("central", (5, 7), (0.4, 1.3)),
                                                 ("lsq", (6, 4), (3.0, 1.0)), ("fourier", (5, 7), (1.5, 0.25)),
                                                 ("lsq", (4, 4, 3), (1.0, 2.0, 0.5)),
                                                 ("fourier", (3, 5, 3), (0.5, 1.0, 2.5))])
def test_projection_on_anisotropic_voxels(derivative, n, length):
    """The same least-squares characterisation with non-cubic voxels: the cell
    lengths enter only through h_a in every stencil."""
    Br = _strain_operator(_gradient_ops(derivative, n, length=length))
    P = Problem(n, np.ones(array_shape(n)), 0.3, length=length, derivative=derivative)
    f = np.random.default_rng(43).standard_normal((P.m,) + array_shape(n))
    ref = Br @ np.linalg.lstsq(Br, f.reshape(-1), rcond=1e-10)[0]
    assert np.abs(P.project(f).reshape(-1) - ref).max() < 1e-11 * np.abs(ref).max()


def test_two_point_fourier_is_least_squares_compatible_part():
    """Appendix C: element 1 (lower triangle) samples the Fourier derivative at
    the voxel centre - (h_x, h_y)/6, element 2 at + (h_x, h_y)/6 (odd grid)."""
    n = (5, 7)
    B1 = _strain_operator(_gradient_ops("fourier2", n, -1.0 / 6.0))
    B2 = _strain_operator(_gradient_ops("fourier2", n, +1.0 / 6.0))
    Br = np.vstack([B1, B2])   # element-major rows: element 1 Mandel comps, then element 2
    P = Problem(n, np.ones(array_shape(n)), 0.3, derivative="fourier2")
    f = np.random.default_rng(42).standard_normal((P.m,) + array_shape(n))
    ref = Br @ np.linalg.lstsq(Br, f.reshape(-1), rcond=1e-10)[0]
    assert np.abs(P.project(f).reshape(-1) - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("derivative", DERIVATIVES)
@pytest.mark.parametrize("n", [(6, 8), (5, 7)])
def test_projection_structure(derivative, n):
    P = Problem(n, np.ones(array_shape(n)), 0.3, derivative=derivative)
    rng = np.random.default_rng(43)
    f = rng.standard_normal((P.m,) + array_shape(n))
    g = rng.standard_normal((P.m,) + array_shape(n))
    Pf = P.project(f)
    assert np.abs(P.project(Pf) - Pf).max() < 1e-12 * np.abs(Pf).max()           # idempotent
    assert abs(np.sum(Pf * g) - np.sum(f * P.project(g))) < 1e-11 * np.abs(Pf).max() * f.size   # self-adjoint
    fh = np.fft.fftn(f, axes=P.axes)
    assert np.abs(np.fft.ifftn(P.project_hat(fh), axes=P.axes).imag).max() < 1e-12    # maps real to real


@pytest.mark.parametrize("derivative", ["forward", "lsq"])
@pytest.mark.parametrize("dim", [2, 3])
def test_laminate_is_exact(derivative, dim):
    n = (8, 4) if dim == 2 else (8, 4, 4)
    layers = np.exp(np.random.default_rng(44).standard_normal(8))
    ns = 3 if dim == 2 else 6
    C, _, _ = Problem(n, ms.laminate(n, layers), 0.3, derivative=derivative).effective_tangent(np.eye(ns), tol=1e-13)
    Cref = laminate_tangent(layers, 0.3, dim)
    assert np.abs(C - Cref).max() < 1e-12 * np.abs(Cref).max()


@pytest.mark.parametrize("derivative", DERIVATIVES)
def test_homogeneous_and_bounds(derivative):
    n = (8, 6)
    P = Problem(n, np.full(array_shape(n), 2.5), 0.3, derivative=derivative)
    _, it, _ = P.solve([0.01, -0.02, 0.005])
    assert it == 0
    E = np.exp(np.random.default_rng(45).standard_normal(array_shape(n)))
    C, _, _ = Problem(n, E, 0.3, derivative=derivative).effective_tangent(np.eye(3), tol=1e-13)
    voigt, reuss = voigt_reuss(E, 0.3, 2)
    assert np.abs(C - C.T).max() < 1e-10 * np.abs(C).max()
    assert np.linalg.eigvalsh(voigt - C).min() > -1e-12
    assert np.linalg.eigvalsh(C - reuss).min() > -1e-12
