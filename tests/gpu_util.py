"""Helpers of the GPU parity tests (build once, seeded inputs, comparisons)."""
import functools

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2105_03297_gb300.build import build_library
    build_library()
    torch.cuda.set_device(0)


def lognormal(n, seed, sigma=1.0):
    shape = tuple(reversed(n))
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(shape))


def rel_max(a, b):
    """max |a - b| / max |b| (matrix-max norm used for effective stiffness)."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@functools.lru_cache(maxsize=None)
def oracle_tangent(n, seed, sigma=1.0, nu=0.3, tol=1e-13):
    """C_eff of the oracle for lognormal(n, seed, sigma), unit load cases; cached
    so that parametrisations over precision and operator form share one solve."""
    from oracle.fe_projection import Problem
    ns = 3 if len(n) == 2 else 6
    C, _, _ = Problem(n, lognormal(n, seed, sigma), nu).effective_tangent(np.eye(ns), tol=tol)
    return C
