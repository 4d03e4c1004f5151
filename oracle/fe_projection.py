"""O1: the finite-element compatibility projection and projected CG, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain, unfused numpy;
the DFT (a matrix product per axis, or ``scipy.fft``) and small batched
linear solves are the only library steps.  The projection is applied one
slab of wavevectors at a time (G(k) acts on each wavevector on its own), so
that the symbols of a 256^3 grid never have to be held at once.

Conventions (fixed once, used by every function):

* grid sizes ``n = (n_x, n_y[, n_z])``; cell lengths ``length`` (default 1),
  voxel size ``h_a = length_a / n_a`` (Appendix A);
* per-voxel arrays are C-ordered with x fastest: shape ``(n_y, n_x)`` or
  ``(n_z, n_y, n_x)``; a field of ``m`` scalars per voxel has shape
  ``(m, *array_shape)``;
* a strain/stress field has ``m = n_q * n_s`` scalars per voxel, element
  major: scalar ``Theta * n_s + s`` is Mandel component ``s`` of element
  ``Theta`` of that voxel; Mandel order 2D (xx, yy, sqrt2 xy), 3D (xx, yy, zz,
  sqrt2 yz, sqrt2 xz, sqrt2 xy);
* elements per voxel (Sec. 2.6, "Linear finite elements"): 2D two triangles,
  element 0 on the nodes {00, 10, 01} (the forward-difference stencil) and
  element 1 on {11, 01, 10} (the same stencil taken backwards from node 11);
  3D six Kuhn tetrahedra {0, e_a, e_a+e_b, e_a+e_b+e_c} for the permutations
  (a, b, c) of (x, y, z) in lexicographic order (the paper only calls the 3D
  generalisation straightforward; this split is our reading);
* DFT: forward ``sum_r f(r) exp(-i k.r)``, inverse with ``1/N`` (Appendix A,
  Eqs. discrete-fourier-trafo and inverse-discrete-fourier-trafo).  Two
  interchangeable evaluations: ``dft="direct"`` writes the sum out as one
  matrix product per axis (the exponential of k.r factorises over the axes),
  ``dft="fft"`` (default) calls ``scipy.fft.fftn``/``ifftn`` on all host
  cores; ``tests/test_oracle_dft.py`` pins both to the definition (sign and
  1/N) and to each other;
* 2D material: isotropic small-strain Hooke's law in plane strain.

Pinned by: ``tests/test_oracle_dft.py`` (both DFT evaluations equal the
sums of Appendix A written out as loops on a small non-square grid, the
projected solve is the same with either), ``tests/test_oracle_projection.py`` (G idempotent, Hermitian,
rank D, G B = B, Hermitian symmetry in k, agreement with the literal
Appendix-B index form and with the textbook Fourier projection),
``tests/test_oracle_solve.py`` (equality with the assembled FEM of O2,
homogeneous material, laminate closed form, Voigt/Reuss bounds, iteration
count flat in N) and ``tests/test_oracle_adjoint.py`` (central finite
differences, Euler identity).
"""
from __future__ import annotations

import itertools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft
import scipy.linalg.blas

SQRT2 = np.sqrt(2.0)


# --------------------------------------------------------------------------
# Index bookkeeping
# --------------------------------------------------------------------------

def n_strain(dim):
    """Number of independent symmetric strain components n_s (the small-strain tensor of
    Eq. small-strain, Appendix B)."""
    return 3 if dim == 2 else 6


def n_elements(dim):
    """Elements (= quadrature points) per voxel n_q: two triangles in 2D, six Kuhn
    tetrahedra in 3D (Sec. 2.6)."""
    return 2 if dim == 2 else 6


def mandel_pairs(dim):
    """Tensor index pair (i, j) of each Mandel component.  Mandel's sqrt2 on the shear
    components makes the Euclidean product of Mandel vectors the double contraction
    of the weak form (Eq. stat-mech-equi-weak-form), so G stays self-adjoint."""
    if dim == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def mandel_weight(i, j):
    """sqrt2 on off-diagonal pairs, 1 on the diagonal (see mandel_pairs)."""
    return 1.0 if i == j else SQRT2


def array_shape(n):
    """Array shape of a per-voxel field on the grid of Appendix A (x fastest)."""
    return tuple(int(v) for v in reversed(tuple(n)))


def voxel_size(n, length=None):
    """Voxel edge lengths h_a = L_a / n_a of the grid of Appendix A (unit cell by default)."""
    if length is None:
        length = (1.0,) * len(n)
    return tuple(float(L) / int(na) for L, na in zip(length, n))


def tensor_to_mandel(T):
    """Symmetric tensors ``T[..., i, j]`` to Mandel vectors ``[..., s]`` (see mandel_pairs)."""
    dim = T.shape[-1]
    return np.stack([mandel_weight(i, j) * T[..., i, j] for i, j in mandel_pairs(dim)], axis=-1)


def mandel_to_tensor(v, dim):
    """Mandel vectors ``v[..., s]`` to symmetric tensors ``[..., i, j]`` (see mandel_pairs)."""
    T = np.zeros(v.shape[:-1] + (dim, dim), dtype=v.dtype)
    for s, (i, j) in enumerate(mandel_pairs(dim)):
        T[..., i, j] = v[..., s] / mandel_weight(i, j)
        T[..., j, i] = v[..., s] / mandel_weight(i, j)
    return T


# --------------------------------------------------------------------------
# Material (small-strain isotropic linear elasticity; Sec. 3.3 uses E and nu)
# --------------------------------------------------------------------------

def lame(E, nu):
    """Lame constants (lambda, mu) from Young's modulus and Poisson's ratio, the two
    constants the examples give (Sec. 3.3)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def stiffness_mandel(dim, E=1.0, nu=0.3):
    """Isotropic stiffness ``lambda 1(x)1 + 2 mu I`` as an n_s x n_s Mandel matrix.

    Isotropic linear elasticity in the constants of Sec. 3.3.  In 2D this is plane
    strain (the paper does not say; our reading): the in-plane block of the 3D tensor.
    """
    lam, mu = lame(E, nu)
    ns = n_strain(dim)
    C = np.zeros((ns, ns))
    for s in range(dim):
        for t in range(dim):
            C[s, t] = lam
        C[s, s] += 2.0 * mu
    for s in range(dim, ns):
        C[s, s] = 2.0 * mu
    return C


def apply_material(field, E, nu):
    """sigma_Theta = E_v * Cbar(nu) : eps_Theta for every element of every voxel
    (one constant strain per element, Sec. 2.6; every element of a voxel has its modulus).

    ``field``: (m, *array_shape) Mandel strains; ``E``: (*array_shape) moduli.
    """
    dim = E.ndim
    ns = n_strain(dim)
    nq = field.shape[0] // ns
    Cbar = stiffness_mandel(dim, 1.0, nu)
    f = field.reshape((nq, ns) + E.shape)
    if field.size < (1 << 20):
        sig = np.einsum("st,qt...->qs...", Cbar, f) * E[None, None]
    else:
        sig = np.moveaxis(np.tensordot(Cbar, f, axes=([1], [1])), 0, 1) * E[None, None]   # Cbar_st f_qt
    return sig.reshape(field.shape)


# --------------------------------------------------------------------------
# Fourier symbols of the element gradients (Eq. genfourderiv)
# --------------------------------------------------------------------------

def wave_indices(n, rows=None, nkx=None):
    """Integer wavevector components m_a per axis; ``rows`` (optional) keeps only
    those indices of the slowest axis (z in 3D, y in 2D), ``nkx`` only the first
    nkx indices of the x axis (the half spectrum of a real field)."""
    idx = [np.arange(int(na)) for na in n]
    if rows is not None:
        idx[-1] = np.arange(int(n[-1]))[rows]
    if nkx is not None:
        idx[0] = np.arange(int(nkx))
    return idx


def symbol_shape(n, rows=None, nkx=None):
    """Array shape of the wavevectors selected by ``rows`` and ``nkx`` (see wave_indices)."""
    return tuple(len(i) for i in reversed(wave_indices(n, rows, nkx)))


def phase_factors(n, rows=None, nkx=None):
    """exp(i k_a h_a) = exp(2 pi i m_a / n_a) on the full FFT grid, per axis: the wave
    vectors of Eq. Fourier_wave_vectors for the forward DFT of Eq. discrete-fourier-trafo.
    ``rows`` and ``nkx`` select wavevectors (see wave_indices)."""
    D = len(n)
    out = []
    for a, (na, ma) in enumerate(zip(n, wave_indices(n, rows, nkx))):
        e = np.exp(2j * np.pi * ma / na)
        sh = [1] * D
        sh[D - 1 - a] = len(ma)
        out.append(e.reshape(sh))
    return out


def element_gradient_symbols(n, length=None, rows=None, nkx=None):
    """g[Theta][a](k): symbol of d/dx_a on element Theta.

    From Eq. genfourderiv with the stencils of the linear-FE elements: a node
    at +e_a relative to the voxel's lower corner contributes exp(i k_a h_a).
    Returns an array of shape (n_q, D, *array_shape), complex128 (with ``rows``,
    only those wavevectors of the slowest axis, see wave_indices).
    """
    D = len(n)
    h = voxel_size(n, length)
    e = phase_factors(n, rows, nkx)
    shp = symbol_shape(n, rows, nkx)
    one = np.ones(shp)
    if D == 2:
        # element 0 = nodes {00, 10, 01}: forward differences
        g0 = [(e[0] - 1.0) / h[0] * one, (e[1] - 1.0) / h[1] * one]
        # element 1 = nodes {11, 01, 10}: d/dx along the top edge 01->11,
        # d/dy along the right edge 10->11
        g1 = [e[1] * (e[0] - 1.0) / h[0] * one, e[0] * (e[1] - 1.0) / h[1] * one]
        return np.array([g0, g1])
    tets = []
    for (a, b, c) in itertools.permutations(range(3)):
        g = [None] * 3
        g[a] = (e[a] - 1.0) / h[a] * one
        g[b] = e[a] * (e[b] - 1.0) / h[b] * one
        g[c] = e[a] * e[b] * (e[c] - 1.0) / h[c] * one
        tets.append(g)
    return np.array(tets)


# Other discrete derivatives of Secs. 2.3-2.5 and Appendix C, each with n_q
# evaluation points per voxel; only B(k) changes.
DERIVATIVES = ("fe", "fourier", "central", "forward", "lsq", "fourier2")


def wrapped_angles(n, rows=None, nkx=None):
    """theta_a = k_a h_a in (-pi, pi) per axis (broadcast shapes as phase_factors);
    the Nyquist index of an even axis gets theta = 0 (our reading of the
    ambiguity discussed in Sec. 2.7: the average of the two grid choices)."""
    D = len(n)
    out = []
    for a, (na, m) in enumerate(zip(n, wave_indices(n, rows, nkx))):
        w = np.where(m < (na + 1) // 2, m, m - na).astype(np.float64)
        if na % 2 == 0:
            w[m == na // 2] = 0.0
        sh = [1] * D
        sh[D - 1 - a] = len(m)
        out.append((2.0 * np.pi * w / na).reshape(sh))
    return out


def derivative_symbols(n, length=None, derivative="fe", rows=None, nkx=None):
    """g[Theta][a](k) for the derivative ``derivative`` (shape (n_q, D, *array_shape)).

    fe:       the linear finite elements (``element_gradient_symbols``), n_q = 2 / 6;
    forward:  Eq. forward-difference-derivative-fourier, (exp(i theta_a) - 1)/h_a;
    central:  Eq. central-difference-derivative-fourier, i sin(theta_a)/h_a;
    lsq:      the least-squares voxel gradient of Sec. 2.5 (forward difference
              along a averaged over the voxel edges parallel to a);
    fourier:  i k_a = i theta_a / h_a (Eq. original-G's derivative);
    fourier2: Appendix C, two evaluation points (2D), i k_a exp(-+ i sum_b theta_b / 6).
    ``rows`` and ``nkx`` select wavevectors (see wave_indices).
    """
    if derivative == "fe":
        return element_gradient_symbols(n, length, rows, nkx)
    D = len(n)
    h = voxel_size(n, length)
    # phases with the exact values at theta = 0, pi/2, pi, 3pi/2, so that the
    # derivatives that vanish there (central differences, least squares) vanish
    # exactly rather than at the rounding level of sin(pi)
    e = []
    for ea in phase_factors(n, rows, nkx):
        ea = ea.copy()
        ea.real[np.abs(ea.real) < 1e-14] = 0.0
        ea.imag[np.abs(ea.imag) < 1e-14] = 0.0
        e.append(ea)
    th = wrapped_angles(n, rows, nkx)
    shp = symbol_shape(n, rows, nkx)
    one = np.ones(shp)
    if derivative == "forward":
        return np.array([[(e[a] - 1.0) / h[a] * one for a in range(D)]])
    if derivative == "central":
        # (u(x + h) - u(x - h)) / 2h -> (e - 1/e) / 2h = i sin(theta) / h
        return np.array([[0.5 * (e[a] - 1.0 / e[a]) / h[a] * one for a in range(D)]])
    if derivative == "lsq":
        g = []
        for a in range(D):
            v = (e[a] - 1.0) / h[a] * one
            for b in range(D):
                if b != a:
                    v = v * 0.5 * (1.0 + e[b])
            g.append(v)
        return np.array([g])
    if derivative == "fourier":
        return np.array([[1j * th[a] / h[a] * one for a in range(D)]])
    if derivative == "fourier2":
        assert D == 2, "two evaluation points are defined for 2D"
        phi = (th[0] + th[1]) / 6.0 * one
        ik = [1j * th[a] / h[a] * one for a in range(D)]
        return np.array([[ik[a] * np.exp(-1j * phi) for a in range(D)],
                         [ik[a] * np.exp(+1j * phi) for a in range(D)]])
    raise ValueError(derivative)


def strain_symbol_components(g):
    """B(k) stored component-major, shape (m, D, *array_shape): the Fourier symbol of
    u -> sym(grad_Theta u), the element strain of Eq. small-strain with the element
    derivatives g_Theta(k).

    Row Theta*n_s + s, column j is Mandel component s of sym(g_Theta (x) e_j).
    """
    nq, D = g.shape[0], g.shape[1]
    pairs = mandel_pairs(D)
    ns = len(pairs)
    B = np.zeros((nq * ns, D) + g.shape[2:], dtype=np.complex128)
    for q in range(nq):
        for s, (a, b) in enumerate(pairs):
            for j in range(D):
                # sym(g (x) e_j)_{ab} = (g_a delta_bj + g_b delta_aj) / 2
                if b == j:
                    B[q * ns + s, j] += 0.5 * mandel_weight(a, b) * g[q, a]
                if a == j:
                    B[q * ns + s, j] += 0.5 * mandel_weight(a, b) * g[q, b]
    return B


def strain_symbol(g):
    """B(k) as one m x D matrix per wavevector: shape (*array_shape, m, D) (see
    strain_symbol_components)."""
    return np.ascontiguousarray(np.moveaxis(strain_symbol_components(g), (0, 1), (-2, -1)))


def projection_matrices(B):
    """G(k) = B (B^H B)^-1 B^H for k != 0 and G(0) = 0 (Sec. 2.3, k = 0 rule).

    Explicit m x m matrices per wavevector; for small grids and pins only.
    """
    BH = np.conj(np.swapaxes(B, -1, -2))
    M = BH @ B
    zero = (slice(0, 1),) * (B.ndim - 2)
    M[zero] = np.eye(B.shape[-1])  # placeholder to keep the solve regular
    G = B @ np.linalg.solve(M, BH)
    G[zero] = 0.0
    return G


# --------------------------------------------------------------------------
# The DFT pair of Appendix A (Eqs. discrete-fourier-trafo and
# inverse-discrete-fourier-trafo)
# --------------------------------------------------------------------------

def dft_direct(f, inverse=False):
    """Forward ``F(k) = sum_r f(r) exp(-2 pi i sum_a k_a r_a / n_a)`` over every axis
    of ``f`` (inverse: ``+`` sign and a factor 1/n_a per axis), evaluated as written.

    exp(-2 pi i k.r) is a product of one factor per axis, so the D-dimensional
    sum is D one-dimensional sums, each a product with the n_a x n_a matrix
    W_a[k, r] = exp(-+2 pi i (k r mod n_a) / n_a)."""
    out = np.asarray(f, dtype=np.complex128)
    sign = 1.0 if inverse else -1.0
    for ax in range(out.ndim):
        na = out.shape[ax]
        k = np.arange(na)
        W = np.exp(sign * 2j * np.pi * (np.outer(k, k) % na) / na)
        out = np.moveaxis(np.tensordot(W, out, axes=([1], [ax])), 0, ax)
        if inverse:
            out = out / na
    return out


def _workers(f):
    """Host threads for one transform: all cores for large arrays, one for small
    ones (where starting threads costs more than it saves)."""
    return (os.cpu_count() or 1) if np.size(f) >= (1 << 18) else 1


def dft_fast(f, inverse=False, axes=None):
    """The same transform pair by scipy's FFT on all host cores (over ``axes``,
    default all)."""
    fn = scipy.fft.ifftn if inverse else scipy.fft.fftn
    return fn(np.asarray(f), axes=axes, workers=_workers(f))


def rdft_fast(f, axes=None):
    """The forward DFT of a real field at k_x = 0..n_x/2 only (scipy, all host cores;
    x is the last of ``axes``): for real f, F(-k) = conj F(k), so these hold every
    independent value."""
    return scipy.fft.rfftn(np.asarray(f), axes=axes, workers=_workers(f))


def irdft_fast(F, shape, axes=None):
    """The inverse DFT (with 1/N) of a spectrum with F(-k) = conj F(k), given at
    k_x = 0..n_x/2 (see rdft_fast); returns the real field with spatial shape
    ``shape``."""
    return scipy.fft.irfftn(F, s=shape, axes=axes, workers=_workers(F))


DFTS = ("direct", "fft")


# --------------------------------------------------------------------------
# Vector operations of the CG (library BLAS on whole fields)
# --------------------------------------------------------------------------

# Fields at least this large use the (multi-threaded) BLAS routines; smaller
# ones plain numpy, where starting the BLAS threads would cost more.
BLAS_MIN = 1 << 20


def inner(a, b):
    """<a, b> = sum_i a_i b_i over every entry of two real fields."""
    if a.size < BLAS_MIN:
        return float(np.sum(a * b))
    return float(np.vdot(a, b))


def axpy(alpha, x, y):
    """y += alpha * x in place (y a C-contiguous float64 field)."""
    assert y.flags.c_contiguous and y.dtype == np.float64
    if y.size < BLAS_MIN:
        y += alpha * x
        return
    out = scipy.linalg.blas.daxpy(np.ascontiguousarray(x).reshape(-1), y.reshape(-1), a=alpha)
    assert np.shares_memory(out, y)


class Problem:
    """A periodic RVE (Sec. 2.1): grid of Appendix A, cell lengths, per-voxel moduli
    and Poisson ratio, with the discrete derivative that defines B(k) (Sec. 2.3)."""

    def __init__(self, n, E, nu, length=None, derivative="fe", dft="fft"):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.E = np.asarray(E, dtype=np.float64)
        assert self.E.shape == array_shape(self.n)
        self.nu = float(nu)
        self.length = length
        self.derivative = derivative
        assert dft in DFTS
        self.dft = dft
        self.ns = n_strain(self.dim)
        self.nq = derivative_symbols((2,) * self.dim, None, derivative).shape[0]
        self.m = self.ns * self.nq
        self.axes = tuple(range(1, self.dim + 1))   # spatial axes of an (m, *shape) field
        self.slab_entries = 1 << 23   # entries of B per slab of wavevectors in project_hat
        self.symbol_cache_bytes = 2 << 30   # keep every slab's symbols when they fit in this
        self._full = None
        self._slabs = {}

    def symbols(self, rows=None, nkx=None):
        """(g, B, B^H B, singular) at the wavevectors selected by ``rows`` and ``nkx``
        (see wave_indices), component-major: element derivatives g (n_q, D, *shape),
        B(k) (m, D, *shape), B^H B (D, D, *shape) with identity blocks where G is
        zero, and that mask (*shape).

        G = 0 where B vanishes: k = 0 (Sec. 2.3) and, for derivatives that vanish
        at other wavevectors (central differences, least squares, the zeroed
        Nyquist of the Fourier derivative), those wavevectors too."""
        g = derivative_symbols(self.n, self.length, self.derivative, rows, nkx)
        B = strain_symbol_components(g)
        M = np.einsum("cj...,ck...->jk...", np.conj(B), B)
        singular = np.all(B == 0.0, axis=(0, 1))
        hit = np.flatnonzero(wave_indices(self.n, rows)[-1] == 0)     # the k = 0 wavevector
        if hit.size:
            singular[(int(hit[0]),) + (0,) * (self.dim - 1)] = True
        for j in range(self.dim):
            for k in range(self.dim):
                M[j, k][singular] = 1.0 if j == k else 0.0
        return g, B, M, singular

    def _all_symbols(self):
        if self._full is None:
            self._full = self.symbols()
        return self._full

    # whole-grid symbols as one matrix per wavevector, for the pins on small grids
    g = property(lambda self: self._all_symbols()[0])
    B = property(lambda self: np.ascontiguousarray(np.moveaxis(self._all_symbols()[1], (0, 1), (-2, -1))))
    BHB = property(lambda self: np.ascontiguousarray(np.moveaxis(self._all_symbols()[2], (0, 1), (-2, -1))))
    singular = property(lambda self: self._all_symbols()[3])

    # -- the projection, applied in the factored form B (B^H B)^-1 B^H ----
    def project_hat(self, fh):
        """Apply G(k) to a spectrum ``fh`` of shape (m, *shape), in place; G(0) = 0
        (Sec. 2.3).  ``fh`` holds either every wavevector or (real fields) only
        k_x = 0..n_x/2, as its last axis says.

        G = B (B^H B)^-1 B^H is the small-strain projection of Appendix B
        (Eqs. small-strain-eq2, small-strain-chi) in matrix form.  G(k) acts on
        each wavevector alone; the wavevectors are taken a slab of the slowest
        axis at a time (so that B need not be held for the whole grid; it is kept
        between calls only when it is small), and the slabs, which share
        nothing, on all host cores at once."""
        nkx = fh.shape[-1]
        assert nkx in (self.n[0], self.n[0] // 2 + 1)
        per_row = int(np.prod(fh.shape[2:])) * self.m * self.dim
        step = max(1, self.slab_entries // per_row)

        keep = per_row * self.n[-1] * 16 <= self.symbol_cache_bytes

        def one_slab(r0):
            rows = slice(r0, min(r0 + step, self.n[-1]))
            key = (r0, step, nkx)
            if key in self._slabs:
                B, M, singular = self._slabs[key]
            else:
                _, B, M, singular = self.symbols(rows, nkx)
                if keep:
                    self._slabs[key] = (B, M, singular)
            t = np.einsum("cj...,c...->j...", np.conj(B), fh[:, rows])      # B^H f
            u = np.linalg.solve(np.moveaxis(M, (0, 1), (-2, -1)),
                                np.moveaxis(t, 0, -1)[..., None])[..., 0]  # (B^H B)^-1 B^H f
            y = np.einsum("cj...,...j->c...", B, u)                        # B (...)
            y[:, singular] = 0.0
            fh[:, rows] = y

        starts = range(0, self.n[-1], step)
        if len(starts) == 1:
            one_slab(0)
        else:
            with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
                list(ex.map(one_slab, starts))
        return fh

    def project(self, f):
        """Real-space projection F^-1[ G(k) F[f](k) ] of an (m, *shape) real field, with
        the DFT pair of Eqs. discrete-fourier-trafo and inverse-discrete-fourier-trafo
        (one component at a time).  ``dft="direct"`` transforms every wavevector;
        ``dft="fft"`` keeps k_x = 0..n_x/2, which hold every independent value of the
        spectrum of a real field: G(-k) = conj G(k), so the projected spectrum keeps
        F(-k) = conj F(k) and its inverse is the same real field."""
        shape = f.shape[1:]
        if self.dft == "direct":
            fh = np.empty(f.shape, dtype=np.complex128)
            for c in range(f.shape[0]):
                fh[c] = dft_direct(f[c])
            self.project_hat(fh)
            out = np.empty(f.shape)
            for c in range(f.shape[0]):
                out[c] = np.real(dft_direct(fh[c], inverse=True))
            return out
        if f.size < (1 << 24):          # small fields: all components in one call
            fh = rdft_fast(f, axes=self.axes)
            self.project_hat(fh)
            return irdft_fast(fh, shape, axes=self.axes)
        fh = np.empty(f.shape[:-1] + (self.n[0] // 2 + 1,), dtype=np.complex128)
        for c in range(f.shape[0]):
            fh[c] = rdft_fast(f[c])
        self.project_hat(fh)
        out = np.empty(f.shape)
        for c in range(f.shape[0]):
            out[c] = irdft_fast(fh[c], shape)
        return out

    def material(self, f):
        """Stress of every element, see apply_material."""
        return apply_material(f, self.E, self.nu)

    def operator(self, v):
        """A(v) = F^-1[ G(k) F[C v](k) ] (the projected stress of Eq. stat-mech-equi2)."""
        return self.project(self.material(v))

    def broadcast_macro(self, Emac):
        """The homogeneous field holding the Mandel strain Emac on every element (the
        macroscopic strain is the k = 0 mode, Sec. 2.3)."""
        Emac = np.asarray(Emac, dtype=np.float64)
        f = np.empty((self.m,) + self.E.shape)
        for q in range(self.nq):
            for s in range(self.ns):
                f[q * self.ns + s] = Emac[s]
        return f

    # -- the projected conjugate gradient (Sec. 2.1: gradient-based solver
    #    whose iterates stay compatible) ----------------------------------
    def cg(self, Emac):
        """The projected CG for G C (E + eps~) = 0 (Eq. stat-mech-equi2), one
        iteration per step of the generator.

        Start eps~ = 0, r = -A(E), p = r; each iteration: q = A(p),
        alpha = <r, r> / <p, q>, eps~ += alpha p, r -= alpha q,
        beta = <r', r'> / <r, r>, p = r' + beta p.  <., .> is the plain sum over
        every Mandel scalar of every element.  Yields (eps~, <r, r>, <r0, r0>)
        before the first iteration and after each one."""
        x = np.zeros((self.m,) + self.E.shape)
        r = -self.operator(self.broadcast_macro(Emac))
        rr0 = inner(r, r)
        rr = rr0
        yield x, rr, rr0
        if rr0 == 0.0:
            return
        p = r.copy()
        while True:
            q = self.operator(p)
            alpha = rr / inner(p, q)
            axpy(alpha, p, x)        # x += alpha p
            axpy(-alpha, q, r)       # r -= alpha q
            del q
            rr_new = inner(r, r)
            p *= rr_new / rr         # p = r + beta p
            axpy(1.0, r, p)
            rr = rr_new
            yield x, rr, rr0

    def solve(self, Emac, tol=1e-12, maxit=10000, history=None):
        """Solve G C (E + eps~) = 0 (Eq. stat-mech-equi2) for the compatible fluctuation
        eps~ by the projected CG (see cg); stop when ||r|| <= tol ||r_0|| (at once
        when r_0 = 0, a homogeneous cell).  Returns (eps_total, iterations,
        relative residual).  A list passed as history receives ||r_k|| / ||r_0||
        for k = 0, 1, ... (bookkeeping only)."""
        it = -1
        for x, rr, rr0 in self.cg(Emac):
            it += 1
            if history is not None:
                history.append(0.0 if rr0 == 0.0 else float(np.sqrt(rr / rr0)))
            if rr0 == 0.0 or it >= maxit or rr <= tol * tol * rr0:
                break
        rel = 0.0 if rr0 == 0.0 else np.sqrt(rr / rr0)
        x += self.broadcast_macro(Emac)
        return x, it, rel

    # -- homogenisation ----------------------------------------------------
    def mean_stress(self, eps):
        """Volume average of C eps over all N * n_q (equal-volume) elements: the
        homogenised stress of Sec. 2.1."""
        sig = self.material(eps).reshape((self.nq, self.ns) + self.E.shape)
        return sig.mean(axis=tuple([0] + list(range(2, 2 + self.dim))))

    def energy_form(self, eps_a, eps_b):
        """Volume average of eps_a : C : eps_b (the energy of the weak form,
        Eq. stat-mech-equi-weak-form, evaluated on two solutions)."""
        return float(np.sum(eps_a * self.material(eps_b)) / (self.E.size * self.nq))

    def effective_tangent(self, Emacs, tol=1e-12, maxit=10000):
        """C_eff from L = n_s linearly independent load cases (rows of Emacs); each
        load case prescribes the mean strain (Sec. 2.1).

        Column l of S is the mean stress of load case l; C_eff = S M^-1 with
        M[:, l] = E_l.  Returns (C_eff, fields, iteration counts).
        """
        Emacs = np.asarray(Emacs, dtype=np.float64)
        fields, its = [], []
        S = np.zeros((self.ns, len(Emacs)))
        for l, Em in enumerate(Emacs):
            eps, it, _ = self.solve(Em, tol, maxit)
            fields.append(eps)
            its.append(it)
            S[:, l] = self.mean_stress(eps)
        C = S @ np.linalg.inv(Emacs.T)
        return C, fields, its

    # -- adjoint gradient of J = W : C_eff w.r.t. the voxel moduli ---------
    def adjoint_gradient(self, W, tol=1e-12, maxit=10000):
        """dJ/dE_v for J = sum_ab W_ab C_eff[a, b], C_eff from unit load cases.  The
        paper has no gradient; this is the adjoint of the discrete equilibrium
        G C eps = 0 (Eq. stat-mech-equi2).

        The adjoint of the mean-stress functional for row a is the projected
        problem with macroscopic strain e_a (the operator is self-adjoint), so
        dJ/dE_v = (1/(N n_q)) sum_{Theta in v} sum_ab W_ab
                  (e_a + lam_a)_Theta : Cbar : eps^b_Theta.
        Returns (grad, C_eff).
        """
        W = np.asarray(W, dtype=np.float64)
        I = np.eye(self.ns)
        C, fields, _ = self.effective_tangent(I, tol, maxit)
        # adjoint solves: same projected operator, right-hand side -A(e_a)
        adj = {}
        for a in range(self.ns):
            if np.any(W[a] != 0.0):
                adj[a], _, _ = self.solve(I[a], tol, maxit)
        Cbar = stiffness_mandel(self.dim, 1.0, self.nu)
        grad = np.zeros(self.E.shape)
        for a in adj:
            la = adj[a].reshape((self.nq, self.ns) + self.E.shape)
            for b in range(self.ns):
                if W[a, b] == 0.0:
                    continue
                eb = fields[b].reshape((self.nq, self.ns) + self.E.shape)
                ceb = np.einsum("st,qt...->qs...", Cbar, eb)
                grad += W[a, b] * np.sum(la * ceb, axis=(0, 1))
        grad /= self.E.size * self.nq
        return grad, C
