"""Analytic pins for the oracle (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``laminate_tangent``: effective stiffness of a grid-aligned laminate (phase
  depends on the x index only).  The exact displacement is piecewise linear
  in x with kinks on grid planes, which linear elements represent exactly
  (Sec. 2.6), so the discrete solution must reproduce this closed form.
* ``voigt_reuss``: the arithmetic and harmonic means of the element
  stiffnesses, which bound any effective stiffness that minimises the
  elastic energy (Eq. stat-mech-equi2 is its stationarity condition).
* ``textbook_strain_projection``: the small-strain projection of Appendix B
  evaluated with the Fourier derivative ik and one evaluation point, in the
  classical closed form in n = k/|k| (Appendix B points to Milton 1988).
* ``appendix_b_projection``: the index form of Appendix B written out
  literally with (potentially discrete) element derivatives D_Theta(k):
  D^-1 = D*/(sum_L D_L . D_L*), g_TL = D_T (x) D_L^-1,
  h = (1 + sum_T g_TT)^-1, and
  G_TL,ijlm = (g_TL,il h_jm + g_TL,im h_jl + g_TL,jl h_im + g_TL,jm h_il)/2.
"""
from __future__ import annotations

import numpy as np

from .fe_projection import lame, mandel_pairs, n_strain, stiffness_mandel


def laminate_tangent(layer_E, nu, dim):
    """Closed-form Mandel C_eff of layers normal to x with moduli ``layer_E`` (equal thickness).

    Continuity across the layers keeps the in-plane strains and the traction
    (sigma_xx, sigma_xy, sigma_xz) uniform; averaging gives, with M = lambda + 2 mu:
    C_xxxx = <1/M>^-1, C_xxyy = <lambda/M><1/M>^-1,
    C_yyyy = <M - lambda^2/M> + <lambda/M>^2 <1/M>^-1,
    C_yyzz = <lambda - lambda^2/M> + <lambda/M>^2 <1/M>^-1,
    x-shears (Mandel) 2 <1/mu>^-1, the in-layer shear 2 <mu>.
    Zero-modulus layers are allowed (the series averages then vanish).
    """
    E = np.asarray(layer_E, dtype=np.float64)
    # every modulus is E times its unit-modulus value, so the ratios lambda/M
    # and lambda^2/M = E lambda1^2/M1 stay finite for zero-stiffness layers
    # (vacuum, Sec. 3.2), where the series averages <1/M>^-1, <1/mu>^-1 -> 0
    lam1, mu1 = lame(1.0, nu)
    M1 = lam1 + 2.0 * mu1
    lam, mu, M = E * lam1, E * mu1, E * M1
    any_void = bool(np.any(E == 0.0))
    inv_iM = 0.0 if any_void else 1.0 / np.mean(1.0 / M)
    inv_imu = 0.0 if any_void else 1.0 / np.mean(1.0 / mu)
    lM = lam1 / M1                       # lambda/M of every layer
    l2M = E * lam1 ** 2 / M1             # lambda^2/M of every layer
    ns = n_strain(dim)
    C = np.zeros((ns, ns))
    C[0, 0] = inv_iM
    for t in range(1, dim):
        C[0, t] = C[t, 0] = lM * inv_iM
    for s in range(1, dim):
        for t in range(1, dim):
            if s == t:
                C[s, t] = np.mean(M - l2M) + lM ** 2 * inv_iM
            else:
                C[s, t] = np.mean(lam - l2M) + lM ** 2 * inv_iM
    pairs = mandel_pairs(dim)
    for s in range(dim, ns):
        i, j = pairs[s]
        if i == 0 or j == 0:
            C[s, s] = 2.0 * inv_imu
        else:
            C[s, s] = 2.0 * np.mean(mu)
    return C


def voigt_reuss(E_field, nu, dim):
    """(Voigt, Reuss) Mandel bounds of a per-voxel isotropic field: any minimiser of
    the energy of Eq. stat-mech-equi-weak-form lies between them."""
    Cbar = stiffness_mandel(dim, 1.0, nu)
    Ev = np.asarray(E_field).reshape(-1)
    voigt = Cbar * np.mean(Ev)
    reuss = np.linalg.inv(np.linalg.inv(Cbar) * np.mean(1.0 / Ev))
    return voigt, reuss


def textbook_strain_projection(kvec):
    """Classical small-strain compatibility projection for one wavevector, k != 0.

    G_ijlm = (n_i n_l d_jm + n_i n_m d_jl + n_j n_l d_im + n_j n_m d_il)/2 - n_i n_j n_l n_m,
    n = k/|k|.  Returned as a full (D, D, D, D) real tensor.
    """
    k = np.asarray(kvec, dtype=np.float64)
    nvec = k / np.linalg.norm(k)
    D = len(k)
    d = np.eye(D)
    G = np.zeros((D, D, D, D))
    for i in range(D):
        for j in range(D):
            for l in range(D):
                for m in range(D):
                    G[i, j, l, m] = 0.5 * (nvec[i] * nvec[l] * d[j, m] + nvec[i] * nvec[m] * d[j, l]
                                           + nvec[j] * nvec[l] * d[i, m] + nvec[j] * nvec[m] * d[i, l]) \
                        - nvec[i] * nvec[j] * nvec[l] * nvec[m]
    return G


def appendix_b_projection(Dsym):
    """Literal Appendix-B small-strain projection for one wavevector.

    ``Dsym``: (n_q, D) complex element derivatives D_Theta(k), not all zero.
    Returns G[T, i, j, L, l, m] with projected strain
    e'_T,ij = sum_L,l,m G[T, i, j, L, l, m] e_L,ml.
    """
    Dsym = np.asarray(Dsym, dtype=np.complex128)
    nq, D = Dsym.shape
    S = np.sum(Dsym * np.conj(Dsym)).real
    Dinv = np.conj(Dsym) / S
    g = np.einsum("ti,lj->tlij", Dsym, Dinv)          # g_TL,ij = D_T,i D^-1_L,j
    h = np.linalg.inv(np.eye(D) + sum(g[t, t] for t in range(nq)))
    G = np.zeros((nq, D, D, nq, D, D), dtype=np.complex128)
    for t in range(nq):
        for L in range(nq):
            gt = g[t, L]
            G[t, :, :, L, :, :] = 0.5 * (np.einsum("il,jm->ijlm", gt, h) + np.einsum("im,jl->ijlm", gt, h)
                                         + np.einsum("jl,im->ijlm", gt, h) + np.einsum("jm,il->ijlm", gt, h))
    return G


def laminate_stretch(layer_E, nu, dim, stretch):
    """Mean first Piola-Kirchhoff stress of a grid-aligned laminate (layers
    normal to x, equal thickness) under F_macro = diag(stretch, 1, ...), for
    the St. Venant-Kirchhoff law (the finite-strain reading of Sec. 3.1); the
    linear elements of Sec. 2.6 represent its exact solution.

    The exact solution keeps F = diag(f_k, 1, ...) in layer k (a piecewise
    linear u_x(x), which linear elements represent exactly); equilibrium makes
    P_xx = E_k M1 f_k (f_k^2 - 1) / 2 the same in every layer and
    compatibility makes the mean of f_k equal to the stretch (M1 = lambda + 2 mu
    at unit modulus).  The transverse components are P_yy = P_zz =
    <E_k lambda1 (f_k^2 - 1) / 2>; the shear components vanish.  Solved by
    bisection on P_xx with a Newton solve per layer (f_k on the branch
    f > 1/sqrt3, where P_xx(f) increases).
    """
    E = np.asarray(layer_E, dtype=np.float64)
    lam1, mu1 = lame(1.0, nu)
    M1 = lam1 + 2.0 * mu1

    def f_of(P):
        """Stretch f_k of every layer that carries the traction P_xx (Newton)."""
        f = np.full_like(E, 1.0)
        for _ in range(100):
            g = E * M1 * f * (f * f - 1.0) / 2.0 - P
            dg = E * M1 * (3.0 * f * f - 1.0) / 2.0
            f = np.maximum(f - g / dg, 1.0 / np.sqrt(3.0) + 1e-12)
        return f

    lo, hi = -1.0, 1.0
    while np.mean(f_of(lo)) > stretch:
        lo *= 2.0
    while np.mean(f_of(hi)) < stretch:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.mean(f_of(mid)) < stretch:
            lo = mid
        else:
            hi = mid
    P = 0.5 * (lo + hi)
    f = f_of(P)
    out = np.zeros((dim, dim))
    out[0, 0] = P
    for a in range(1, dim):
        out[a, a] = np.mean(E * lam1 * (f * f - 1.0) / 2.0)
    return out

