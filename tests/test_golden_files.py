"""The stored expected values under tests/golden/ (CPU).

They were written by tests/golden/make_golden.py from the oracle alone.  The
small case is re-solved here and must agree; the large ones (hours of oracle
time) are checked against what holds for any exact effective stiffness of the
regenerated input field: symmetric, positive definite, between the Voigt and
Reuss bounds, and isotropic-looking where the field is statistically isotropic.
A file from another microstructure, an unconverged solve or a transposed
matrix fails one of these.
"""
import json
import os

import numpy as np
import pytest

import microstructures as ms
from oracle.closed_forms import voigt_reuss
from oracle.fe_projection import Problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def test_disc32_is_reproduced_by_the_oracle():
    ref = _load("disc32")
    cfg = ms.config_inputs("disc32")
    P = Problem(cfg["n"], cfg["E"], cfg["nu"])
    C, _, _ = P.effective_tangent(np.eye(3), tol=ref["tol"])
    assert np.abs(C - np.array(ref["C_eff"])).max() < 1e-11 * np.abs(C).max()
    eps, _, _ = P.solve(cfg["E_macro"][0], tol=ref["tol"])
    assert np.allclose(P.mean_stress(eps), ref["mean_stress"][0], rtol=1e-10, atol=0)
    assert np.abs(np.array(ref["C_eff_fem"]) - C).max() < 1e-10 * np.abs(C).max()


def _bounds_ok(C, E, nu, dim):
    V, R = voigt_reuss(E, nu, dim)
    lo = np.linalg.eigvalsh(C - R).min()
    hi = np.linalg.eigvalsh(V - C).min()
    return lo > -1e-10 * np.abs(C).max() and hi > -1e-10 * np.abs(C).max()


@pytest.mark.parametrize("name", ["gauss1024", "lognormal64", "spheres128"])
def test_stored_tangents_are_admissible(name):
    ref = _load(name)
    cfg = ms.config_inputs(name)
    assert list(cfg["n"]) == ref["n"] and cfg["nu"] == ref["nu"]
    C = np.array(ref["C_eff"])
    dim = len(cfg["n"])
    ns = 3 if dim == 2 else 6
    assert C.shape == (ns, ns)
    assert np.abs(C - C.T).max() < 1e-9 * np.abs(C).max()          # symmetric (major symmetry)
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0              # positive definite
    assert _bounds_ok(0.5 * (C + C.T), cfg["E"], cfg["nu"], dim)      # Voigt >= C >= Reuss
    # statistically isotropic fields: the normal diagonal entries agree to a few percent,
    # and normal-shear couplings are small against the diagonal
    d = np.diag(C)[:dim]
    assert d.max() / d.min() < 1.1
    assert np.abs(C[:dim, dim:]).max() < 0.05 * d.min()


def test_spheres128_parts_merge_into_the_tangent():
    C = np.array(_load("spheres128")["C_eff"])
    for l in range(6):
        part = _load(f"spheres128_lc{l}")
        assert part["rel_residual"] <= 1e-12
        assert np.allclose(C[:, l], part["mean_stress"], rtol=0, atol=1e-15 * np.abs(C).max())


def test_lognormal64_adjoint_sample_is_consistent():
    ref = _load("lognormal64")
    C = np.array(ref["C_eff"])
    W = np.array(ref["adjoint_W"])
    # Euler's identity for the degree-1 homogeneous J = W : C_eff
    assert abs(ref["adjoint_euler_sum"] - np.sum(W * C)) < 1e-9 * abs(np.sum(W * C))
    g = np.array(ref["adjoint_grad"])
    assert np.all(g > 0)                                            # J = C_1111 grows with every modulus
    assert len(set(ref["adjoint_voxels"])) == len(ref["adjoint_voxels"]) == 16


def test_stored_256_mean_stress_is_admissible():
    """The 256^3 log-normal field under a unit xx strain: the stored mean stress
    is column 1 of an effective stiffness, so its xx entry lies between the
    Reuss and Voigt values of that entry, the field is statistically isotropic
    (yy and zz agree, shears are small), and the energy e_xx : C : e_xx is the
    xx entry (positive)."""
    ref = _load("lognormal256")
    cfg = ms.config_inputs("lognormal256")
    assert list(cfg["n"]) == ref["n"] and cfg["nu"] == ref["nu"]
    S = np.array(ref["mean_stress"])
    assert S.shape == (1, 6) and ref["iterations"][0] > 0
    s = S[0]
    V, R = voigt_reuss(cfg["E"], cfg["nu"], 3)
    assert R[0, 0] <= s[0] <= V[0, 0]
    assert abs(s[1] - s[2]) < 1e-3 * s[1]
    assert np.abs(s[3:]).max() < 0.05 * s[0]
    assert s[0] > s[1] > 0
