"""O1: the finite-element compatibility projection and projected CG, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain, unblocked,
unfused numpy; an FFT (``numpy.fft``) and small batched linear solves are the
only library steps.

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
  Eqs. discrete-fourier-trafo and inverse-discrete-fourier-trafo), which is
  numpy's ``fftn``/``ifftn`` over the spatial axes;
* 2D material: isotropic small-strain Hooke's law in plane strain.

Pinned by: ``tests/test_oracle_projection.py`` (G idempotent, Hermitian,
rank D, G B = B, Hermitian symmetry in k, agreement with the literal
Appendix-B index form and with the textbook Fourier projection),
``tests/test_oracle_solve.py`` (equality with the assembled FEM of O2,
homogeneous material, laminate closed form, Voigt/Reuss bounds, iteration
count flat in N) and ``tests/test_oracle_adjoint.py`` (central finite
differences, Euler identity).
"""
from __future__ import annotations

import itertools

import numpy as np

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
    sig = np.einsum("st,qt...->qs...", Cbar, f) * E[None, None]
    return sig.reshape(field.shape)


# --------------------------------------------------------------------------
# Fourier symbols of the element gradients (Eq. genfourderiv)
# --------------------------------------------------------------------------

def phase_factors(n):
    """exp(i k_a h_a) = exp(2 pi i m_a / n_a) on the full FFT grid, per axis: the wave
    vectors of Eq. Fourier_wave_vectors for the forward DFT of Eq. discrete-fourier-trafo."""
    D = len(n)
    out = []
    for a, na in enumerate(n):
        e = np.exp(2j * np.pi * np.arange(na) / na)
        sh = [1] * D
        sh[D - 1 - a] = na
        out.append(e.reshape(sh))
    return out


def element_gradient_symbols(n, length=None):
    """g[Theta][a](k): symbol of d/dx_a on element Theta.

    From Eq. genfourderiv with the stencils of the linear-FE elements: a node
    at +e_a relative to the voxel's lower corner contributes exp(i k_a h_a).
    Returns an array of shape (n_q, D, *array_shape), complex128.
    """
    D = len(n)
    h = voxel_size(n, length)
    e = phase_factors(n)
    shp = array_shape(n)
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


def wrapped_angles(n):
    """theta_a = k_a h_a in (-pi, pi) per axis (broadcast shapes as phase_factors);
    the Nyquist index of an even axis gets theta = 0 (our reading of the
    ambiguity discussed in Sec. 2.7: the average of the two grid choices)."""
    D = len(n)
    out = []
    for a, na in enumerate(n):
        m = np.arange(na)
        w = np.where(m < (na + 1) // 2, m, m - na).astype(np.float64)
        if na % 2 == 0:
            w[na // 2] = 0.0
        sh = [1] * D
        sh[D - 1 - a] = na
        out.append((2.0 * np.pi * w / na).reshape(sh))
    return out


def derivative_symbols(n, length=None, derivative="fe"):
    """g[Theta][a](k) for the derivative ``derivative`` (shape (n_q, D, *array_shape)).

    fe:       the linear finite elements (``element_gradient_symbols``), n_q = 2 / 6;
    forward:  Eq. forward-difference-derivative-fourier, (exp(i theta_a) - 1)/h_a;
    central:  Eq. central-difference-derivative-fourier, i sin(theta_a)/h_a;
    lsq:      the least-squares voxel gradient of Sec. 2.5 (forward difference
              along a averaged over the voxel edges parallel to a);
    fourier:  i k_a = i theta_a / h_a (Eq. original-G's derivative);
    fourier2: Appendix C, two evaluation points (2D), i k_a exp(-+ i sum_b theta_b / 6).
    """
    if derivative == "fe":
        return element_gradient_symbols(n, length)
    D = len(n)
    h = voxel_size(n, length)
    # phases with the exact values at theta = 0, pi/2, pi, 3pi/2, so that the
    # derivatives that vanish there (central differences, least squares) vanish
    # exactly rather than at the rounding level of sin(pi)
    e = []
    for ea in phase_factors(n):
        ea = ea.copy()
        ea.real[np.abs(ea.real) < 1e-14] = 0.0
        ea.imag[np.abs(ea.imag) < 1e-14] = 0.0
        e.append(ea)
    th = wrapped_angles(n)
    shp = array_shape(n)
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


def strain_symbol(g):
    """B(k): (*array_shape, m, D) complex, Fourier symbol of u -> sym(grad_Theta u),
    the element strain of Eq. small-strain with the element derivatives g_Theta(k).

    Row Theta*n_s + s, column j is Mandel component s of sym(g_Theta (x) e_j).
    """
    nq, D = g.shape[0], g.shape[1]
    pairs = mandel_pairs(D)
    ns = len(pairs)
    shp = g.shape[2:]
    B = np.zeros(shp + (nq * ns, D), dtype=np.complex128)
    for q in range(nq):
        for s, (a, b) in enumerate(pairs):
            for j in range(D):
                # sym(g (x) e_j)_{ab} = (g_a delta_bj + g_b delta_aj) / 2
                val = 0.5 * ((g[q, a] if b == j else 0.0) + (g[q, b] if a == j else 0.0))
                B[..., q * ns + s, j] = mandel_weight(a, b) * val
    return B


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


class Problem:
    """A periodic RVE (Sec. 2.1): grid of Appendix A, cell lengths, per-voxel moduli
    and Poisson ratio, with the discrete derivative that defines B(k) (Sec. 2.3)."""

    def __init__(self, n, E, nu, length=None, derivative="fe"):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.E = np.asarray(E, dtype=np.float64)
        assert self.E.shape == array_shape(self.n)
        self.nu = float(nu)
        self.length = length
        self.derivative = derivative
        self.ns = n_strain(self.dim)
        self.g = derivative_symbols(self.n, length, derivative)
        self.nq = self.g.shape[0]
        self.m = self.ns * self.nq
        self.B = strain_symbol(self.g)  # (*shape, m, D)
        BH = np.conj(np.swapaxes(self.B, -1, -2))
        M = BH @ self.B
        # G = 0 where B vanishes: k = 0 (Sec. 2.3) and, for derivatives that
        # vanish at other wavevectors (central differences, least squares, the
        # zeroed Nyquist of the Fourier derivative), those wavevectors too
        self.singular = np.all(np.abs(self.B) == 0.0, axis=(-2, -1))
        self.singular[(0,) * self.dim] = True
        M[self.singular] = np.eye(self.dim)
        self.BHB = M  # B^H B with the singular blocks replaced by I (never used there)
        self.axes = tuple(range(1, self.dim + 1))

    # -- the projection, applied in the factored form B (B^H B)^-1 B^H ----
    def project_hat(self, fh):
        """Apply G(k) to a spectrum ``fh`` of shape (m, *shape); G(0) = 0 (Sec. 2.3).

        G = B (B^H B)^-1 B^H is the small-strain projection of Appendix B
        (Eqs. small-strain-eq2, small-strain-chi) in matrix form."""
        x = np.moveaxis(fh, 0, -1)[..., None]            # (*shape, m, 1)
        t = np.conj(np.swapaxes(self.B, -1, -2)) @ x      # B^H f
        u = np.linalg.solve(self.BHB, t)                  # (B^H B)^-1 B^H f
        y = (self.B @ u)[..., 0]                          # B (...)
        y[self.singular] = 0.0
        return np.moveaxis(y, -1, 0)

    def project(self, f):
        """Real-space projection F^-1[ G(k) F[f](k) ] of an (m, *shape) field, with the
        DFT pair of Eqs. discrete-fourier-trafo and inverse-discrete-fourier-trafo."""
        fh = np.fft.fftn(f, axes=self.axes)
        return np.real(np.fft.ifftn(self.project_hat(fh), axes=self.axes))

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
    def solve(self, Emac, tol=1e-12, maxit=10000):
        """Solve G C (E + eps~) = 0 (Eq. stat-mech-equi2) for the compatible fluctuation eps~.

        Start eps~ = 0, r = -A(E); plain CG with Euclidean inner products on
        the Mandel scalars; stop when ||r|| <= tol ||r_0||.  Returns
        (eps_total, iterations, relative residual).
        """
        Ef = self.broadcast_macro(Emac)
        x = np.zeros_like(Ef)
        r = -self.operator(Ef)
        rr0 = float(np.sum(r * r))
        if rr0 == 0.0:
            return Ef + x, 0, 0.0
        p = r.copy()
        rr = rr0
        it = 0
        while it < maxit and rr > tol * tol * rr0:
            q = self.operator(p)
            alpha = rr / float(np.sum(p * q))
            x += alpha * p
            r -= alpha * q
            rr_new = float(np.sum(r * r))
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
        return Ef + x, it, np.sqrt(rr / rr0)

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
