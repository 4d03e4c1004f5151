"""The seeded input generators (CPU): each recipe does what its description
says — phase rule, volume fraction, periodicity, distribution, seeds.

These inputs feed both the oracle and the GPU path, so a wrong recipe would
not show up as a parity failure; it is checked here on its own.
"""
import numpy as np
import pytest

import microstructures as ms


def test_array_shape_is_x_fastest():
    assert ms.array_shape((8, 4)) == (4, 8)
    assert ms.array_shape((8, 4, 2)) == (2, 4, 8)


def test_circular_inclusion_uses_voxel_centres_strictly_inside():
    n = (32, 24)
    E = ms.circular_inclusion(n, radius=0.25, E_incl=10.0, E_matrix=1.0)
    assert E.shape == (24, 32) and set(np.unique(E)) == {1.0, 10.0}
    for iy in range(n[1]):
        for ix in range(n[0]):
            x, y = (ix + 0.5) / n[0], (iy + 0.5) / n[1]
            inside = (x - 0.5) ** 2 + (y - 0.5) ** 2 < 0.25 ** 2
            assert E[iy, ix] == (10.0 if inside else 1.0)
    # mirror symmetric about the cell centre; area close to pi r^2
    assert np.array_equal(E, E[::-1, :]) and np.array_equal(E, E[:, ::-1])
    big = ms.circular_inclusion((256, 256), 0.25)
    assert abs((big > 1).mean() - np.pi * 0.25 ** 2) < 2e-3


def test_ball_in_3d():
    E = ms.circular_inclusion((16, 16, 16), radius=0.3, E_incl=5.0)
    assert E.shape == (16, 16, 16)
    assert np.array_equal(E, np.transpose(E, (1, 0, 2))) and np.array_equal(E, np.transpose(E, (2, 1, 0)))
    assert abs((E > 1).mean() - 4.0 / 3.0 * np.pi * 0.3 ** 3) < 0.02


def test_periodic_gaussian_filter():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((32, 48))
    g = ms._periodic_gaussian_filter(f, 3.0)
    # circular convolution commutes with periodic shifts and keeps the mean
    assert np.allclose(ms._periodic_gaussian_filter(np.roll(f, (5, -7), (0, 1)), 3.0),
                       np.roll(g, (5, -7), (0, 1)), atol=1e-12)
    assert abs(g.mean() - f.mean()) < 1e-12
    # it smooths: the variance drops, the field stays real and finite
    assert g.var() < 0.1 * f.var() and np.all(np.isfinite(g))
    # a delta spreads into a normalised, symmetric periodic bump
    d = np.zeros((64, 64)); d[0, 0] = 1.0
    k = ms._periodic_gaussian_filter(d, 2.0)
    assert abs(k.sum() - 1.0) < 1e-12 and np.allclose(k, np.roll(k[::-1, ::-1], (1, 1), (0, 1)), atol=1e-15)


@pytest.mark.parametrize("vf", [0.3, 0.5, 0.7])
def test_thresholded_gaussian_volume_fraction_and_seed(vf):
    n = (64, 64)
    E = ms.thresholded_gaussian(n, sigma_px=4.0, vf=vf, E_hi=100.0, E_lo=1.0, seed=7)
    assert set(np.unique(E)) == {1.0, 100.0}
    assert abs((E == 100.0).mean() - vf) <= 1.0 / E.size
    assert np.array_equal(E, ms.thresholded_gaussian(n, 4.0, vf, 100.0, 1.0, seed=7))
    assert not np.array_equal(E, ms.thresholded_gaussian(n, 4.0, vf, 100.0, 1.0, seed=8))


def test_gauss1024_workload():
    cfg = ms.config_inputs("gauss1024")
    E = cfg["E"]
    assert cfg["n"] == (1024, 1024) and E.shape == (1024, 1024) and cfg["nu"] == 0.3
    assert set(np.unique(E)) == {1.0, 100.0} and abs((E == 100.0).mean() - 0.5) <= 1e-6
    assert np.array_equal(cfg["E_macro"], np.eye(3))
    # a smooth two-phase field: most neighbours share the phase (white noise would give 50%)
    same = (E == np.roll(E, 1, axis=1)).mean()
    assert same > 0.9


def test_random_spheres_recipe():
    n, r = (40, 40, 40), 4.0
    E = ms.random_spheres(n, radius=r, vf=0.12, E_incl=1000.0, E_matrix=1.0, seed=11)
    assert E.shape == (40, 40, 40) and set(np.unique(E)) == {1.0, 1000.0}
    frac = (E > 1).mean()
    ball = 4.0 / 3.0 * np.pi * r ** 3 / E.size
    assert 0.12 <= frac < 0.12 + 1.5 * ball          # stops at the first sphere past the target
    assert np.array_equal(E, ms.random_spheres(n, r, 0.12, 1000.0, 1.0, seed=11))
    # one sphere: a periodic ball of about 4/3 pi r^3 voxels, symmetric about its centre voxel
    one = ms.random_spheres(n, radius=r, vf=1e-9, seed=12) > 1
    assert abs(one.sum() - 4.0 / 3.0 * np.pi * r ** 3) < 0.25 * 4.0 / 3.0 * np.pi * r ** 3
    # the number of spheres is the inside voxel count over a ball's (no two share a voxel,
    # so the count of separate 26-connected pieces can't exceed it)
    from scipy import ndimage
    lab, k = ndimage.label(E > 1, structure=np.ones((3, 3, 3)))
    assert k >= 1 and k <= int(round(frac * E.size / (0.75 * 4.0 / 3.0 * np.pi * r ** 3))) + 1


def test_lognormal_field_distribution():
    E = ms.lognormal_field((64, 64, 64), mu=0.2, sigma=0.7, seed=3)
    logE = np.log(E)
    assert np.all(E > 0)
    assert abs(logE.mean() - 0.2) < 5 * 0.7 / np.sqrt(E.size)
    assert abs(logE.std() - 0.7) < 0.01
    # independent voxels: neighbour correlation is at the sampling-noise level
    c = np.corrcoef(logE.ravel(), np.roll(logE, 1, axis=2).ravel())[0, 1]
    assert abs(c) < 5 / np.sqrt(E.size)


def test_laminate_depends_on_x_only():
    layers = np.arange(1.0, 9.0)
    E = ms.laminate((8, 4, 2), layers)
    assert E.shape == (2, 4, 8)
    assert np.array_equal(E, np.broadcast_to(layers, (2, 4, 8)))


def test_porous_lognormal():
    E = ms.porous_lognormal((64, 64), void_fraction=0.25, seed=9)
    void = E == 0.0
    assert abs(void.mean() - 0.25) < 5 * np.sqrt(0.25 * 0.75 / E.size)
    assert np.all(E[~void] > 0)
    assert np.array_equal(E, ms.porous_lognormal((64, 64), 0.25, seed=9))


@pytest.mark.parametrize("n", [(32, 16), (32, 16, 8)])
def test_two_pillars(n):
    E, A, B = ms.two_pillars(n, E_hard=2.0, soft_ratio=0.1, inclusion=3)
    ix = np.broadcast_to(np.arange(n[0]), E.shape)
    gaps = (ix == n[0] // 2 - 1) | (ix == n[0] - 1)
    assert np.all(E[gaps] == 0.0) and np.all(E[~gaps] > 0.0)
    assert not np.any(A & B) and np.array_equal(A | B, ~gaps)
    soft = E == 0.2
    assert soft.sum() == 9 * (n[2] if len(n) == 3 else 1)
    assert np.all(A[soft])                              # the inclusion sits in pillar A
    assert np.all(E[B] == 2.0)                          # pillar B is homogeneous


def test_uneven_batch():
    batch = ms.uneven_batch_2d(count=12, sides=(16, 32, 64), sigma_px=2.0, seed=21)
    assert len(batch) == 12
    for n, E in batch:
        assert n[0] == n[1] and n[0] in (16, 32, 64) and E.shape == (n[1], n[0])
        lo, hi = E.min(), E.max()
        assert lo == 1.0 and 10.0 <= hi <= 1000.0
        assert 0.3 - 1.0 / E.size <= (E == hi).mean() <= 0.7 + 1.0 / E.size
    sizes = {n[0] for n, _ in ms.uneven_batch_2d(count=64, seed=1004)}
    assert sizes == {64, 128, 256, 512}


def test_small_named_configs():
    d = ms.config_inputs("disc32")
    assert d["n"] == (32, 32) and d["E_macro"].shape == (1, 3) and d["E_macro"][0, 0] == 0.01
    assert np.array_equal(d["E"], ms.circular_inclusion((32, 32), 0.25, 10.0, 1.0))
    l64 = ms.config_inputs("lognormal64")
    assert l64["E"].shape == (64, 64, 64) and l64["E_macro"].shape == (6, 6)
    with pytest.raises(KeyError):
        ms.config_inputs("no_such_workload")
