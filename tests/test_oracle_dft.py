"""Pins of the oracle's DFT pair and of its slab-wise projection.

The DFT of Appendix A (Eqs. discrete-fourier-trafo and
inverse-discrete-fourier-trafo) is F(k) = sum_r f(r) exp(-i k.r) with
k_a = 2 pi m_a / (n_a h_a), r_a = j_a h_a, and the inverse carries +i and 1/N.
Both of the oracle's evaluations (the direct matrix product per axis and
scipy's FFT) are checked here against those sums written out as plain loops
on a small non-square grid, so a wrong sign, a missing 1/N or a transposed
axis fails.
"""
import itertools

import numpy as np
import pytest

from oracle.fe_projection import (Problem, array_shape, dft_direct, dft_fast, irdft_fast, projection_matrices,
                                  rdft_fast)


def dft_by_loops(f, inverse=False):
    """The sums of Appendix A, one term at a time (f has shape (n_z, n_y, n_x))."""
    shape = f.shape
    N = f.size
    out = np.zeros(shape, dtype=np.complex128)
    sign = 1.0 if inverse else -1.0
    for k in itertools.product(*[range(s) for s in shape]):
        acc = 0.0 + 0.0j
        for r in itertools.product(*[range(s) for s in shape]):
            phase = sum(ka * ra / s for ka, ra, s in zip(k, r, shape))
            acc += f[r] * np.exp(sign * 2j * np.pi * phase)
        out[k] = acc / N if inverse else acc
    return out


@pytest.mark.parametrize("shape", [(4, 6, 5), (3, 8)])
@pytest.mark.parametrize("dft", [dft_direct, dft_fast])
def test_dft_equals_the_defining_sums(shape, dft):
    rng = np.random.default_rng(7)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    F = dft_by_loops(f)
    assert np.abs(dft(f) - F).max() < 1e-12 * np.abs(F).max()
    Fi = dft_by_loops(f, inverse=True)
    assert np.abs(dft(f, inverse=True) - Fi).max() < 1e-12 * np.abs(Fi).max()


@pytest.mark.parametrize("shape", [(4, 6, 5), (3, 8), (5, 6)])
def test_real_half_spectrum_equals_the_defining_sums(shape):
    # the real-field form keeps k_x = 0..n_x/2 (x is the last array axis)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(shape)
    F = dft_by_loops(f)
    H = rdft_fast(f)
    assert H.shape[-1] == shape[-1] // 2 + 1
    assert np.abs(H - F[..., : shape[-1] // 2 + 1]).max() < 1e-12 * np.abs(F).max()
    assert np.abs(irdft_fast(H, shape) - f).max() < 1e-13


def test_dft_sign_on_a_shifted_delta():
    # a unit impulse at r0 transforms to exp(-i k.r0): the sign of the forward DFT
    shape = (4, 6, 5)
    r0 = (1, 2, 3)
    f = np.zeros(shape)
    f[r0] = 1.0
    k = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    want = np.exp(-2j * np.pi * sum(ka * ra / s for ka, ra, s in zip(k, r0, shape)))
    for dft in (dft_direct, dft_fast):
        assert np.abs(dft(f) - want).max() < 1e-13


def test_round_trip_and_parseval():
    rng = np.random.default_rng(8)
    f = rng.standard_normal((6, 4, 10))
    for dft in (dft_direct, dft_fast):
        F = dft(f)
        assert np.abs(dft(F, inverse=True) - f).max() < 1e-13
        assert abs(np.sum(np.abs(F) ** 2) / f.size - np.sum(f ** 2)) < 1e-11 * np.sum(f ** 2)


@pytest.mark.parametrize("n", [(8, 6), (4, 6, 4)])
def test_solve_is_the_same_with_either_dft(n):
    rng = np.random.default_rng(9)
    E = np.exp(rng.standard_normal(array_shape(n)))
    Pd = Problem(n, E, 0.3, dft="direct")
    Pf = Problem(n, E, 0.3, dft="fft")
    ns = Pd.ns
    Em = np.eye(ns)[0]
    ed, itd, _ = Pd.solve(Em, tol=1e-13)
    ef, itf, _ = Pf.solve(Em, tol=1e-13)
    assert np.abs(ed - ef).max() < 1e-11 * np.abs(ef).max()
    assert np.abs(Pd.mean_stress(ed) - Pf.mean_stress(ef)).max() < 1e-12 * np.abs(Pf.mean_stress(ef)).max()


@pytest.mark.parametrize("n", [(6, 8), (4, 6, 5)])
def test_slab_wise_projection_equals_explicit_G(n):
    # project_hat takes the wavevectors one slab of the slowest axis at a time;
    # with one row per slab it must still equal the explicit m x m matrices G(k)
    rng = np.random.default_rng(10)
    P = Problem(n, np.ones(array_shape(n)), 0.3)
    P.slab_entries = 1          # forces one row of the slowest axis per slab
    fh = rng.standard_normal((P.m,) + array_shape(n)) + 1j * rng.standard_normal((P.m,) + array_shape(n))
    G = projection_matrices(P.B)
    want = np.moveaxis((G @ np.moveaxis(fh, 0, -1)[..., None])[..., 0], -1, 0)
    got = P.project_hat(fh.copy())
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
