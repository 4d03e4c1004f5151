"""Differentiable effective stiffness: C_eff(E) with the adjoint gradient.

``effective_stiffness(E, nu)`` solves the n_s unit load cases on the GPU
(``rve_solve``) and returns the Mandel effective tangent as a float64 tensor.
Its backward pass calls ``rve_adjoint`` with W = dL/dC_eff: the adjoint
projected-CG solves reuse the same operator, and the per-voxel gradient is
dJ/dE_v = 1/(N n_q) sum_{Theta in v} sum_{a,l} W_al (e_a + lambda_a) : Cbar : eps_l.
"""
from __future__ import annotations

import numpy as np
import torch

from ._rve import RVE


class EffectiveStiffness(torch.autograd.Function):
    """autograd.Function of E (per-voxel Young's moduli) -> C_eff (n_s x n_s)."""

    @staticmethod
    def forward(ctx, E, nu, precision, rel_tol, max_iter):
        if not E.is_cuda:
            raise ValueError("E must be a CUDA tensor")
        n = tuple(reversed(E.shape))  # E is (n_y, n_x) or (n_z, n_y, n_x)
        stream = torch.cuda.current_stream(E.device).cuda_stream
        r = RVE(n, precision=precision, stream=stream)
        Ec = E.detach().contiguous().to(torch.float64)
        r.set_material(Ec, float(nu))
        ns = r.ns
        code, info = r.solve(np.eye(ns), rel_tol=rel_tol, max_iter=max_iter)
        C = r.effective_tangent()
        ctx.rve = r
        ctx.shape = E.shape
        ctx.dtype = E.dtype
        ctx.rel_tol = rel_tol
        ctx.max_iter = max_iter
        ctx.info = info
        return torch.as_tensor(C, dtype=torch.float64, device=E.device)

    @staticmethod
    def backward(ctx, grad_C):
        r = ctx.rve
        W = grad_C.detach().to(torch.float64).cpu().numpy()
        g = torch.empty(int(np.prod(ctx.shape)), dtype=torch.float64, device=grad_C.device)
        r.adjoint(W, rel_tol=ctx.rel_tol, max_iter=ctx.max_iter, out=g)
        r.close()
        ctx.rve = None
        return g.reshape(ctx.shape).to(ctx.dtype), None, None, None, None


def effective_stiffness(E: torch.Tensor, nu: float, precision: str = "mixed", rel_tol: float = 1e-11,
                        max_iter: int = 20000) -> torch.Tensor:
    """Mandel effective stiffness of the periodic cell with moduli E (differentiable in E)."""
    return EffectiveStiffness.apply(E, nu, precision, rel_tol, max_iter)
