"""O2: the conforming periodic linear-FE problem, assembled in real space (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Independent of O1: no
Fourier symbols, no projection.  The paper states that the FE projection is
identical to traditional linear finite elements on the structured grid
(Sec. 2.6, "Linear finite elements"); this module is that traditional
formulation, built from the simplex shape functions:

    minimise  sum_e |e| (E + eps_e(u)) : C_e : (E + eps_e(u))
    over periodic nodal displacement fluctuations u (one node pinned),

i.e. K u = -sum_e |e| B_e^T C_e E with K = sum_e |e| B_e^T C_e B_e.

Nodes sit at voxel corners (Appendix A grid), node (i_x, i_y[, i_z]) is the
lower corner of voxel (i_x, i_y[, i_z]), indices periodic.  Element order per
voxel and the Mandel convention match ``fe_projection``.  Its element strains
are therefore directly comparable with O1's strain fields.

Pinned by: brute-force dense minimisation on tiny grids and the laminate
closed form (``tests/test_oracle_solve.py``).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe_projection import (array_shape, mandel_pairs, mandel_weight, n_strain,
                            stiffness_mandel, voxel_size)


def element_vertices(dim):
    """Vertex offsets (in voxel units) of the elements of one voxel: the two triangles
    of Sec. 2.6 in 2D, the six Kuhn tetrahedra (our reading of the 3D split) in 3D."""
    if dim == 2:
        return [np.array([[0, 0], [1, 0], [0, 1]]),
                np.array([[1, 1], [0, 1], [1, 0]])]
    tets = []
    for (a, b, c) in itertools.permutations(range(3)):
        v0 = np.zeros(3, dtype=int)
        v1 = v0.copy(); v1[a] = 1
        v2 = v1.copy(); v2[b] = 1
        v3 = v2.copy(); v3[c] = 1
        tets.append(np.array([v0, v1, v2, v3]))
    return tets


def shape_function_gradients(X):
    """Gradients of the linear shape functions of a simplex with vertices X (the
    linear elements of Sec. 2.6).

    N_i(x) = a_i + b_i . x with N_i(X_j) = delta_ij; returns b as (D+1, D)
    and the simplex volume.
    """
    D = X.shape[1]
    P = np.hstack([np.ones((D + 1, 1)), X])
    coef = np.linalg.inv(P)          # column i holds (a_i, b_i)
    vol = abs(np.linalg.det(P)) / float(np.prod(np.arange(1, D + 1)))
    return coef[1:, :].T.copy(), vol


def element_strain_matrix(grads):
    """B_e: Mandel strain (Eq. small-strain) of an element from its (D+1) nodal
    displacement vectors."""
    npts, D = grads.shape
    pairs = mandel_pairs(D)
    Be = np.zeros((len(pairs), npts * D))
    for s, (a, b) in enumerate(pairs):
        w = mandel_weight(a, b)
        for i in range(npts):
            for j in range(D):
                # sym(grad N_i (x) e_j)_{ab}
                val = 0.5 * ((grads[i, a] if b == j else 0.0) + (grads[i, b] if a == j else 0.0))
                Be[s, i * D + j] = w * val
    return Be


class AssembledFEM:
    """Periodic linear-FE stiffness of a voxel grid with per-voxel moduli: the
    traditional finite-element problem that Sec. 2.6 says the FE projection reproduces."""

    def __init__(self, n, E, nu, length=None):
        self.n = tuple(int(v) for v in n)
        self.dim = D = len(self.n)
        self.E = np.asarray(E, dtype=np.float64)
        assert self.E.shape == array_shape(self.n)
        self.nu = float(nu)
        self.ns = n_strain(D)
        h = np.array(voxel_size(self.n, length))
        self.Cbar = stiffness_mandel(D, 1.0, nu)
        self.elems = []
        for verts in element_vertices(D):
            grads, vol = shape_function_gradients(verts * h)
            self.elems.append((verts, element_strain_matrix(grads), vol))
        self.nq = len(self.elems)
        N = self.E.size
        self.N = N
        # voxel multi-index (x fastest) and node numbering
        self.idx = np.array(np.unravel_index(np.arange(N), array_shape(self.n))[::-1]).T  # (N, D) as (x, y[, z])
        self.nn = np.array(self.n)
        self.strides = np.array([int(np.prod(self.n[:a])) for a in range(D)])
        self._assemble()

    def _node(self, offs):
        """Node numbers of voxel corner ``offs`` for every voxel (periodic)."""
        p = (self.idx + offs[None, :]) % self.nn[None, :]
        return p @ self.strides

    def _assemble(self):
        """K = sum_e |e| B_e^T C_e B_e over all elements, periodic node numbering."""
        D, N = self.dim, self.N
        Ev = self.E.reshape(-1)  # voxel numbering = x fastest, matches idx rows
        rows, cols, vals = [], [], []
        self.elem_dofs = []
        for verts, Be, vol in self.elems:
            nodes = np.stack([self._node(v) for v in verts], axis=1)    # (N, D+1)
            dofs = (nodes[:, :, None] * D + np.arange(D)[None, None, :]).reshape(N, -1)
            self.elem_dofs.append(dofs)
            Ke = vol * Be.T @ self.Cbar @ Be                              # per unit modulus
            nd = dofs.shape[1]
            rows.append(np.repeat(dofs, nd, axis=1).reshape(-1))
            cols.append(np.tile(dofs, (1, nd)).reshape(-1))
            vals.append((Ev[:, None, None] * Ke[None]).reshape(-1))
        ndof = N * D
        self.K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(ndof, ndof)).tocsr()
        self.ndof = ndof

    def load_vector(self, Emac):
        """f = -sum_e |e| B_e^T C_e E (the load of the prescribed mean strain, Sec. 2.1)."""
        Emac = np.asarray(Emac, dtype=np.float64)
        Ev = self.E.reshape(-1)
        f = np.zeros(self.ndof)
        for (verts, Be, vol), dofs in zip(self.elems, self.elem_dofs):
            fe = -vol * (Be.T @ (self.Cbar @ Emac))                      # (nd,)
            np.add.at(f, dofs.reshape(-1), (Ev[:, None] * fe[None, :]).reshape(-1))
        return f

    def solve(self, Emac, direct=True, tol=1e-14):
        """Nodal fluctuation u (node 0 pinned) for macroscopic strain Emac: K u = f,
        the FE equilibrium of Sec. 2.6."""
        D = self.dim
        f = self.load_vector(Emac)
        free = np.arange(D, self.ndof)
        Kff = self.K[free][:, free].tocsc()
        u = np.zeros(self.ndof)
        if direct:
            u[free] = spla.spsolve(Kff, f[free])
        else:
            d = Kff.diagonal()
            Mpre = spla.LinearOperator(Kff.shape, matvec=lambda x: x / d)
            sol, info = spla.cg(Kff, f[free], rtol=tol, atol=0.0, maxiter=200000, M=Mpre)
            if info != 0:
                raise RuntimeError("FEM CG did not converge")
            u[free] = sol
        return u

    def element_strains(self, Emac, u):
        """Total strain E + B_e u_e per element, as an (m, *array_shape) field."""
        Emac = np.asarray(Emac, dtype=np.float64)
        out = []
        for (verts, Be, vol), dofs in zip(self.elems, self.elem_dofs):
            eps = Emac[None, :] + u[dofs] @ Be.T                          # (N, ns)
            out.append(eps.T.reshape((self.ns,) + self.E.shape))
        return np.concatenate(out, axis=0)

    def energy(self, Emac, u):
        """sum_e |e| eps_e : C_e : eps_e (the minimised functional, the energy of
        Eq. stat-mech-equi-weak-form)."""
        eps = self.element_strains(Emac, u).reshape((self.nq, self.ns, -1))
        Ev = self.E.reshape(-1)
        tot = 0.0
        for q, (verts, Be, vol) in enumerate(self.elems):
            tot += vol * np.sum(Ev * np.einsum("sn,st,tn->n", eps[q], self.Cbar, eps[q]))
        return tot

    def mean_stress(self, eps):
        """Volume average of C eps over all (equal-volume) elements (Sec. 2.1)."""
        Ev = self.E.reshape(-1)
        e = eps.reshape((self.nq, self.ns, -1))
        sig = np.einsum("st,qtn->qsn", self.Cbar, e) * Ev[None, None, :]
        return sig.mean(axis=(0, 2))

    def effective_tangent(self, Emacs, direct=True):
        """C_eff from n_s independent load cases, as Problem.effective_tangent (Sec. 2.1)."""
        Emacs = np.asarray(Emacs, dtype=np.float64)
        S = np.zeros((self.ns, len(Emacs)))
        fields = []
        for l, Em in enumerate(Emacs):
            u = self.solve(Em, direct=direct)
            eps = self.element_strains(Em, u)
            fields.append(eps)
            S[:, l] = self.mean_stress(eps)
        return S @ np.linalg.inv(Emacs.T), fields


def dense_minimiser(n, E, nu, Emac, length=None):
    """Brute force for tiny grids: minimise the FE energy with a dense pseudo-inverse.

    Builds K densely and solves K u = f in the least-squares sense (no node
    pinned, the constant null space is removed by the pseudo-inverse).
    """
    fem = AssembledFEM(n, E, nu, length)
    K = fem.K.toarray()
    f = fem.load_vector(Emac)
    u = np.linalg.pinv(K, rcond=1e-12) @ f
    return fem.element_strains(Emac, u)


def finite_strain_fem(n, E, nu, Fmac, length=None, tol=1e-13, max_newton=50):
    """Periodic finite-strain linear-FE problem in real space (dense; tiny grids).

    The same St. Venant-Kirchhoff law as ``finite_strain`` but no Fourier
    symbols and no projection: nodal displacement fluctuations u (D per node),
    F_e = F_macro + sum_v u_v (x) grad N_v on every simplex, and Newton on the
    stationarity of sum_e |e| W(F_e), W = lambda/2 tr(E)^2 + mu E : E, with the
    consistent tangent assembled densely; the constant null space is removed
    by a least-squares solve.  Returns (F per element [n_q, D, D, N], mean
    first Piola-Kirchhoff stress [D, D], Newton steps).
    """
    n = tuple(int(v) for v in n)
    D = len(n)
    Ev = np.asarray(E, dtype=np.float64).reshape(-1)
    N = Ev.size
    lam1 = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu1 = 1.0 / (2.0 * (1.0 + nu))
    h = np.array(voxel_size(n, length))
    idx = np.array(np.unravel_index(np.arange(N), array_shape(n))[::-1]).T
    strides = np.array([int(np.prod(n[:a])) for a in range(D)])
    elems = []
    for verts in element_vertices(D):
        grads, vol = shape_function_gradients(verts * h)
        nodes = np.stack([((idx + v[None, :]) % np.array(n)[None, :]) @ strides for v in verts], axis=1)
        elems.append((grads, vol, nodes))
    Fm = np.asarray(Fmac, dtype=np.float64).reshape(D, D)
    ndof = N * D
    I = np.eye(D)

    def element_F(u):
        """F = I + grad u per element (Eq. def-grad) from the nodal displacement."""
        out = []
        for grads, vol, nodes in elems:
            U = u.reshape(N, D)[nodes]                           # (N, D+1, D): u_v,i
            H = np.einsum("evi,va->eia", U, grads)
            out.append(Fm[None] + H)
        return out

    def pk(F, e):
        """St. Venant-Kirchhoff first Piola-Kirchhoff stress (as FiniteStrainProblem)."""
        C = np.einsum("eki,ekj->eij", F, F)
        Eg = 0.5 * (C - I[None])
        tr = np.trace(Eg, axis1=1, axis2=2)
        S = e[:, None, None] * (lam1 * tr[:, None, None] * I[None] + 2.0 * mu1 * Eg)
        return S

    def assemble(u):
        """Nodal force vector and dense tangent stiffness of the finite-strain problem."""
        g = np.zeros(ndof)
        K = np.zeros((ndof, ndof))
        for (grads, vol, nodes), F in zip(elems, element_F(u)):
            S = pk(F, Ev)
            P = np.einsum("eik,ekj->eij", F, S)
            # internal force on dof (v, i): sum_a P_ia dN_v/dx_a
            fe = vol * np.einsum("eia,va->evi", P, grads)
            dofs = (nodes[:, :, None] * D + np.arange(D)[None, None, :])   # (N, D+1, D)
            np.add.at(g, dofs.reshape(-1), fe.reshape(-1))
            # tangent dP/dF contracted with the shape-function gradients
            A = np.zeros((N, D, D, D, D))
            for j in range(D):
                for b in range(D):
                    dF = np.zeros((N, D, D))
                    dF[:, j, b] = 1.0
                    FtdF = np.einsum("eki,ekj->eij", F, dF)
                    dE = 0.5 * (FtdF + np.swapaxes(FtdF, 1, 2))
                    dtr = np.trace(dE, axis1=1, axis2=2)
                    dS = Ev[:, None, None] * (lam1 * dtr[:, None, None] * I[None] + 2.0 * mu1 * dE)
                    A[:, :, :, j, b] = np.einsum("eik,ekj->eij", dF, S) + np.einsum("eik,ekj->eij", F, dS)
            Ke = vol * np.einsum("ua,eiajb,vb->euivj", grads, A, grads)           # (N, D+1, D, D+1, D)
            d = dofs.reshape(N, -1)
            m = d.shape[1]
            np.add.at(K, (np.repeat(d, m, axis=1).reshape(-1), np.tile(d, (1, m)).reshape(-1)),
                      Ke.reshape(N, m * m).reshape(-1))
        return g, K

    u = np.zeros(ndof)
    g0 = None
    steps = 0
    while steps < max_newton:
        g, K = assemble(u)
        gn = np.linalg.norm(g)
        if g0 is None:
            g0 = gn
        if gn <= tol * max(g0, 1e-300):
            break
        u -= np.linalg.lstsq(K, g, rcond=1e-12)[0]
        steps += 1
    Fs = element_F(u)
    Pbar = np.zeros((D, D))
    for F in Fs:
        Pbar += np.einsum("eik,ekj->ij", F, pk(F, Ev)) / (N * len(Fs))
    Farr = np.stack([F.transpose(1, 2, 0) for F in Fs])                 # (n_q, D, D, N)
    return Farr, Pbar, steps
