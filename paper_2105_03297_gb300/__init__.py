"""GB300 linear-finite-element compatibility-projection homogenization.

The projected conjugate-gradient solver of Leute et al. (small-strain linear
elasticity on linear triangles / Kuhn tetrahedra, projection
G(k) = B (B^H B)^-1 B^H), implemented as hand-written sm_103a CUDA kernels
behind the C ABI of ``include/rve.h``.  This package is the thin Python
binding (``RVE``) and the ``torch.autograd.Function`` of the effective
stiffness.
"""
from ._rve import (RVE, RVEBatch, RVE_ERR_ARG, RVE_ERR_NONFINITE, RVE_ERR_NOT_CONVERGED, RVE_ERR_UNSUPPORTED_SIZE,
                   RVE_OK, RveError, load)

__all__ = ["RVE", "RVEBatch", "RveError", "load", "RVE_OK", "RVE_ERR_ARG", "RVE_ERR_NONFINITE",
           "RVE_ERR_NOT_CONVERGED", "RVE_ERR_UNSUPPORTED_SIZE"]
