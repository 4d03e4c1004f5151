"""O3: finite-strain compatibility projection with a Newton-projected-CG solve (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain numpy: FFTs and
elementwise tensor algebra only.

The unknown is the deformation gradient F_Theta = F_macro + H_Theta per
element, F_ia = d chi_i / d r_a (Eq. def-grad).  Compatibility is enforced by
the projection of Eq. original-G, G_i a b j = delta_ij g_ab, with the
discrete derivative of the element stencils (Eq. discrete_projection_op with
n_q evaluation points): for row i of F,

    (G H)_{Theta,i,a} = D_Theta,a(k) sum_{Lambda,b} conj(D_Lambda,b(k)) H_{Lambda,i,b} / S(k),
    S(k) = sum_{Lambda,b} |D_Lambda,b(k)|^2,           G = 0 where S = 0 (k = 0).

Equilibrium is G P(F) = 0 (Eq. stat-mech-equi-FFT-homogenization) with the
first Piola-Kirchhoff stress P.  The law is not stated in the paper beyond
"isotropic finite-strain linear elastic" (Sec. 3.1): we read it as the
St. Venant-Kirchhoff law,

    E = (F^T F - I) / 2,   S = lambda tr(E) I + 2 mu E,   P = F S,

with lambda, mu from the voxel's Young's modulus and the Poisson ratio (plane
strain in 2D), and its tangent dP = dF S + F (lambda tr(dE) I + 2 mu dE),
dE = sym(F^T dF).  The solve is Newton on G P(F) = 0 with each correction
from plain projected CG on G K(F) dH = -G P(F) (K symmetric, so G K G is
self-adjoint and CG applies), as in the gradient-based scheme of Sec. 2.1.

Fields have shape (n_q, D, D, *array_shape): F[Theta, i, a].

Pinned by ``tests/test_oracle_finite_strain.py``: the projection equals the
least-squares compatible part built from O2's real-space shape-function
gradients, the law against central differences and frame indifference, the
homogeneous cell (exact, no iteration), the small-strain limit (O1's C_eff),
a grid-aligned laminate under stretch against its one-dimensional solution,
frame indifference of the whole cell solution, and equality with the
periodic finite-strain FE problem assembled and solved in real space
(``fem_assembly.finite_strain_fem``).
"""
from __future__ import annotations

import numpy as np

from .fe_projection import array_shape, derivative_symbols, lame


class FiniteStrainProblem:
    """A periodic cell under finite strain (St. Venant-Kirchhoff per voxel; Sec. 3.1
    names an isotropic finite-strain linear elastic law, this is our reading of it)."""

    def __init__(self, n, E, nu, length=None, derivative="fe"):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.E = np.asarray(E, dtype=np.float64)
        assert self.E.shape == array_shape(self.n)
        self.nu = float(nu)
        self.g = derivative_symbols(self.n, length, derivative)    # (nq, D, *shape)
        self.nq = self.g.shape[0]
        self.S = np.sum(np.abs(self.g) ** 2, axis=(0, 1))
        self.singular = self.S == 0.0
        self.singular[(0,) * self.dim] = True
        self.axes = tuple(range(3, 3 + self.dim))
        lam1, mu1 = lame(1.0, self.nu)
        self.lam = lam1 * self.E
        self.mu = mu1 * self.E

    # -- the projection -----------------------------------------------------
    def project(self, A):
        """G applied to a gradient field A (n_q, D, D, *shape), real: the gradient
        projection G_iabj = delta_ij g_ab of Eq. original-G with the element derivatives
        of Eq. discrete_projection_op, row by row of F (Eq. def-grad)."""
        Ah = np.fft.fftn(A, axes=self.axes)
        t = np.einsum("qa...,qia...->i...", np.conj(self.g), Ah)      # B^H A per row i
        S = np.where(self.singular, 1.0, self.S)
        w = np.where(self.singular[None], 0.0, t / S[None])
        out = np.einsum("qa...,i...->qia...", self.g, w)
        return np.real(np.fft.ifftn(out, axes=self.axes))

    # -- the law ------------------------------------------------------------
    def _pk2(self, F):
        """Green-Lagrange strain and second Piola-Kirchhoff stress of every element
        (St. Venant-Kirchhoff in the constants of Sec. 3.3, plane strain in 2D)."""
        D = self.dim
        C = np.einsum("qki...,qkj...->qij...", F, F)
        Eg = 0.5 * (C - np.eye(D)[None, :, :, *([None] * self.dim)])
        tr = np.einsum("qii...->q...", Eg)
        S = 2.0 * self.mu[None, None, None] * Eg
        for i in range(D):
            S[:, i, i] += self.lam[None] * tr
        return Eg, S

    def stress(self, F):
        """First Piola-Kirchhoff stress P = F S of every element (the stress of the
        equilibrium G P(F) = 0, Eq. stat-mech-equi-FFT-homogenization)."""
        _, S = self._pk2(F)
        return np.einsum("qik...,qkj...->qij...", F, S)

    def tangent(self, F, dF):
        """dP = dF S(F) + F (lambda tr(dE) I + 2 mu dE), dE = sym(F^T dF): the
        linearisation of stress() that Newton's method solves with."""
        _, S = self._pk2(F)
        FtdF = np.einsum("qki...,qkj...->qij...", F, dF)
        dE = 0.5 * (FtdF + np.swapaxes(FtdF, 1, 2))
        dtr = np.einsum("qii...->q...", dE)
        dS = 2.0 * self.mu[None, None, None] * dE
        for i in range(self.dim):
            dS[:, i, i] += self.lam[None] * dtr
        return np.einsum("qik...,qkj...->qij...", dF, S) + np.einsum("qik...,qkj...->qij...", F, dS)

    # -- the solve ----------------------------------------------------------
    def broadcast(self, Fmac):
        """The homogeneous deformation gradient Fmac on every element (the k = 0 mode
        of F, Sec. 2.3)."""
        Fmac = np.asarray(Fmac, dtype=np.float64).reshape(self.dim, self.dim)
        return np.broadcast_to(Fmac[None, :, :, *([None] * self.dim)],
                               (self.nq, self.dim, self.dim) + self.E.shape).copy()

    def solve(self, Fmac, tol=1e-10, cg_tol=1e-12, max_newton=30, maxit=20000):
        """Newton-projected-CG on G P(F) = 0 (Eq. stat-mech-equi-FFT-homogenization);
        each correction is a projected CG solve of G K(F) dF = -G P(F).  Stops when
        ||G P(F)|| <= tol ||G P(F_macro)||.

        Returns (F, Newton steps, total CG iterations, relative residual)."""
        F = self.broadcast(Fmac)
        P0 = self.stress(F)
        r = -self.project(P0)
        r0 = float(np.sqrt(np.sum(r * r)))
        # a homogeneous cell is in equilibrium: its residual is FFT round-off
        if r0 <= 1e-13 * float(np.sqrt(np.sum(P0 * P0))):
            return F, 0, 0, 0.0
        steps = its = 0
        rn = r0
        while rn > tol * r0 and steps < max_newton:
            # projected CG on G K(F) dH = r, dH compatible, start 0
            x = np.zeros_like(F)
            rr0 = float(np.sum(r * r))
            p = r.copy()
            rr = rr0
            rc = r.copy()
            k = 0
            while k < maxit and rr > cg_tol * cg_tol * rr0:
                q = self.project(self.tangent(F, p))
                alpha = rr / float(np.sum(p * q))
                x += alpha * p
                rc -= alpha * q
                rr_new = float(np.sum(rc * rc))
                p = rc + (rr_new / rr) * p
                rr = rr_new
                k += 1
            F = F + x
            its += k
            steps += 1
            r = -self.project(self.stress(F))
            rn = float(np.sqrt(np.sum(r * r)))
        return F, steps, its, rn / r0

    def mean_stress(self, F):
        """Volume average of P over all (equal-volume) elements, (D, D): the
        homogenised first Piola-Kirchhoff stress."""
        return self.stress(F).mean(axis=(0,) + self.axes)
