"""Seeded synthetic microstructures and load cases.

This module produces INPUT DATA only (per-voxel Young's moduli, macroscopic
strains).  It holds none of the homogenization arithmetic: both the FP64
oracle and the CUDA path import it, and nothing else is shared between them.

Array convention: a per-voxel field of a grid with ``n = (n_x, n_y[, n_z])``
voxels is a C-ordered float64 array of shape ``(n_y, n_x)`` in 2D and
``(n_z, n_y, n_x)`` in 3D, i.e. x is the fastest-varying index.  Voxel
(i_x, i_y[, i_z]) has its lower corner at ``(i_x, i_y[, i_z]) * L/n`` (the
paper's Appendix A grid) and its centre at ``(i + 1/2) * L/n``.

Macroscopic strains are Mandel vectors: 2D ``(xx, yy, sqrt2*xy)``, 3D
``(xx, yy, zz, sqrt2*yz, sqrt2*xz, sqrt2*xy)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "array_shape", "circular_inclusion", "thresholded_gaussian", "random_spheres",
    "lognormal_field", "laminate", "uneven_batch_2d", "unit_load_cases",
    "config_inputs",
]


def array_shape(n):
    """Array shape of a per-voxel field for grid sizes ``n = (n_x, n_y[, n_z])``."""
    return tuple(int(v) for v in reversed(tuple(n)))


def _centres(n):
    """Voxel-centre coordinates in a unit cell, one broadcastable array per axis."""
    D = len(n)
    out = []
    for a, na in enumerate(n):
        c = (np.arange(na) + 0.5) / na
        sh = [1] * D
        sh[D - 1 - a] = na
        out.append(c.reshape(sh))
    return out


def circular_inclusion(n=(32, 32), radius=0.25, E_incl=10.0, E_matrix=1.0):
    """Centred disc (2D) or ball (3D) of radius ``radius*L`` in a unit cell.

    A voxel belongs to the inclusion when its centre lies strictly inside the
    radius around the cell centre.
    """
    c = _centres(n)
    r2 = sum((ci - 0.5) ** 2 for ci in c)
    inside = r2 < radius ** 2
    return np.where(inside, E_incl, E_matrix).astype(np.float64)


def _periodic_gaussian_filter(field, sigma_px):
    """Periodic Gaussian blur (circular convolution through the FFT)."""
    D = field.ndim
    kernel_hat = np.ones(field.shape)
    for ax in range(D):
        n = field.shape[ax]
        f = np.fft.fftfreq(n)  # cycles per pixel
        g = np.exp(-2.0 * (np.pi * f * sigma_px) ** 2)
        sh = [1] * D
        sh[ax] = n
        kernel_hat = kernel_hat * g.reshape(sh)
    return np.real(np.fft.ifftn(np.fft.fftn(field) * kernel_hat))


def thresholded_gaussian(n, sigma_px=8.0, vf=0.5, E_hi=100.0, E_lo=1.0, seed=1002):
    """Two-phase field: white noise -> periodic Gaussian filter -> threshold.

    The stiff phase (``E_hi``) occupies the voxels above the ``1 - vf``
    quantile of the filtered field, so its volume fraction is ``vf`` up to ties.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(array_shape(n))
    smooth = _periodic_gaussian_filter(noise, sigma_px)
    thr = np.quantile(smooth, 1.0 - vf)
    return np.where(smooth > thr, E_hi, E_lo).astype(np.float64)


def random_spheres(n=(128, 128, 128), radius=6.0, vf=0.20, E_incl=1000.0, E_matrix=1.0,
                   seed=1003, max_tries=200000):
    """Random sequential addition of non-overlapping periodic spheres.

    Centres are uniform in the cell (voxel units); a candidate is accepted
    when its periodic minimum-image distance to every accepted centre is at
    least ``2*radius``.  Spheres are added until the voxel fraction inside
    (voxel centre strictly within ``radius``) reaches ``vf``.
    """
    rng = np.random.default_rng(seed)
    nn = np.array(n, dtype=np.float64)
    centres = []
    inside = np.zeros(array_shape(n), dtype=bool)
    cx = [np.arange(na) + 0.5 for na in n]
    tries = 0
    while inside.mean() < vf:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_spheres: could not reach the volume fraction")
        c = rng.uniform(0.0, 1.0, size=3) * nn
        if centres:
            d = np.abs(np.array(centres) - c)
            d = np.minimum(d, nn - d)
            if np.min(np.sum(d * d, axis=1)) < (2.0 * radius) ** 2:
                continue
        centres.append(c)
        # mark voxels of this sphere (periodic minimum image per axis)
        dd = []
        for a in range(3):
            t = np.abs(cx[a] - c[a])
            dd.append(np.minimum(t, nn[a] - t))
        r2 = (dd[2][:, None, None] ** 2 + dd[1][None, :, None] ** 2
              + dd[0][None, None, :] ** 2)
        inside |= r2 < radius ** 2
    return np.where(inside, E_incl, E_matrix).astype(np.float64)


def lognormal_field(n, mu=0.0, sigma=1.0, seed=1005):
    """Independent log-normal Young's modulus per voxel, ``exp(N(mu, sigma^2))``."""
    rng = np.random.default_rng(seed)
    return np.exp(mu + sigma * rng.standard_normal(array_shape(n)))


def laminate(n, layer_moduli):
    """Field whose modulus depends on the x index only: ``E[..., i_x] = layer_moduli[i_x]``."""
    layer_moduli = np.asarray(layer_moduli, dtype=np.float64)
    assert layer_moduli.shape == (n[0],)
    return np.broadcast_to(layer_moduli, array_shape(n)).copy()


def porous_lognormal(n, void_fraction=0.25, sigma=1.0, seed=1008):
    """Log-normal moduli with a random set of zero-stiffness (vacuum) voxels.

    Every voxel is independently void with probability ``void_fraction``
    (E = 0); the others get ``exp(N(0, sigma^2))``.
    """
    rng = np.random.default_rng(seed)
    E = np.exp(sigma * rng.standard_normal(array_shape(n)))
    E[rng.random(array_shape(n)) < void_fraction] = 0.0
    return E


def two_pillars(n, gaps=(None, None), E_hard=1.0, soft_ratio=0.1, inclusion=3):
    """Two stiff pillars (bands normal to x) separated by two single-voxel
    zero-stiffness columns, in the spirit of the vacuum example (Sec. 3.2).

    Columns ``gaps`` (default n_x/2 - 1 and n_x - 1) have E = 0, which cuts the
    periodic cell into two bodies: pillar A (x < gaps[0]) and pillar B.
    Pillar A holds a centred square soft inclusion of ``inclusion`` voxels per
    side with E = soft_ratio * E_hard.  Returns (E, mask_A, mask_B).
    """
    nx = n[0]
    g0 = nx // 2 - 1 if gaps[0] is None else gaps[0]
    g1 = nx - 1 if gaps[1] is None else gaps[1]
    shape = array_shape(n)
    E = np.full(shape, float(E_hard))
    ix = np.arange(nx)
    E[..., ix == g0] = 0.0
    E[..., ix == g1] = 0.0
    maskA = np.broadcast_to(ix < g0, shape).copy()
    maskB = np.broadcast_to((ix > g0) & (ix < g1), shape).copy()
    # soft inclusion at the centre of pillar A (in every z plane for 3D: a fibre)
    cx = g0 // 2
    lo = cx - inclusion // 2
    sl_x = slice(lo, lo + inclusion)
    ny = n[1]
    sl_y = slice(ny // 2 - inclusion // 2, ny // 2 - inclusion // 2 + inclusion)
    if len(n) == 2:
        E[sl_y, sl_x] = soft_ratio * E_hard
    else:
        E[:, sl_y, sl_x] = soft_ratio * E_hard
    return E, maskA, maskB


def uneven_batch_2d(count=64, sides=(64, 128, 256, 512), sigma_px=8.0, seed=1004):
    """Batch of square 2D two-phase RVEs of uneven size.

    Returns a list of ``(n, E_field)`` with the side drawn uniformly from
    ``sides``, the stiff volume fraction from U(0.3, 0.7) and the contrast
    log-uniformly from [10, 1000] (matrix modulus 1).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s = int(rng.choice(sides))
        vf = float(rng.uniform(0.3, 0.7))
        contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(1000.0))))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        E = thresholded_gaussian((s, s), sigma_px=sigma_px, vf=vf, E_hi=contrast, E_lo=1.0,
                                 seed=sub_seed)
        out.append(((s, s), E))
    return out


def unit_load_cases(dim):
    """The Mandel unit strains e_1 ... e_ns, one load case per row."""
    ns = 3 if dim == 2 else 6
    return np.eye(ns)


def config_inputs(name):
    """Inputs of the named workloads.

    Returns a dict with ``n`` (grid sizes, x first), ``E`` (per-voxel Young's
    modulus), ``nu`` and ``E_macro`` (load cases, Mandel rows).
    """
    if name == "disc32":          # 2D 32x32, disc r=0.25L, E 10/1, one load case
        n = (32, 32)
        return dict(n=n, E=circular_inclusion(n, 0.25, 10.0, 1.0), nu=0.3,
                    E_macro=np.array([[0.01, 0.0, 0.0]]))
    if name == "gauss1024":       # 2D 1024^2 thresholded Gaussian, contrast 100, 3 load cases
        n = (1024, 1024)
        return dict(n=n, E=thresholded_gaussian(n, 8.0, 0.5, 100.0, 1.0, seed=1002), nu=0.3,
                    E_macro=unit_load_cases(2))
    if name == "spheres128":      # 3D 128^3 spheres r=6, vf 0.2, contrast 1000, 6 load cases
        n = (128, 128, 128)
        return dict(n=n, E=random_spheres(n, 6.0, 0.20, 1000.0, 1.0, seed=1003), nu=0.3,
                    E_macro=unit_load_cases(3))
    if name == "lognormal64":     # 3D 64^3 log-normal, objective C_1111
        n = (64, 64, 64)
        return dict(n=n, E=lognormal_field(n, 0.0, 1.0, seed=1005), nu=0.3,
                    E_macro=unit_load_cases(3))
    if name == "lognormal128":    # 3D 128^3 log-normal, one load case (profiling size)
        n = (128, 128, 128)
        return dict(n=n, E=lognormal_field(n, 0.0, 1.0, seed=1007), nu=0.3,
                    E_macro=unit_load_cases(3)[:1])
    if name == "lognormal256":    # 3D 256^3 log-normal, one load case (throughput)
        n = (256, 256, 256)
        return dict(n=n, E=lognormal_field(n, 0.0, 1.0, seed=1006), nu=0.3,
                    E_macro=unit_load_cases(3)[:1])
    if name == "lognormal256x256x32":   # profiling size with the 256-point x and y transforms
        n = (256, 256, 32)
        return dict(n=n, E=lognormal_field(n, 0.0, 1.0, seed=1011), nu=0.3,
                    E_macro=unit_load_cases(3)[:1])
    if name == "lognormal32x32x256":    # profiling size with the 256-point z transform (pass C)
        n = (32, 32, 256)
        return dict(n=n, E=lognormal_field(n, 0.0, 1.0, seed=1012), nu=0.3,
                    E_macro=unit_load_cases(3)[:1])
    raise KeyError(name)
