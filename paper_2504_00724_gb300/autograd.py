"""Differentiable solve: u = L^{-1}(f - N g) as a torch.autograd.Function.

Forward is ccm_solve; backward is one adjoint solve: with lambda = L^{-T} dJ/du,
dJ/df = lambda and dJ/dg = -N^T lambda (eq. PoissonResidualForm differentiated).  Only
marshalling happens here; both solves and N^T run in the library."""
from __future__ import annotations

import torch


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, g, solver):
        u, _ = solver.solve(f.contiguous(), None if g is None else g.contiguous())
        ctx.solver = solver
        ctx.has_g = g is not None
        return u

    @staticmethod
    def backward(ctx, grad_u):
        solver = ctx.solver
        lam, _ = solver.solve_T(grad_u.contiguous())
        grad_g = None
        if ctx.has_g:
            _, ng = solver.apply_T(lam, want_u=False, want_g=True)
            grad_g = -ng
        return lam, grad_g, None


def solve(solver, f, g=None):
    """u = L^{-1}(f - N g) with gradients to f and g (float64 CUDA tensors, [ny, nx] / [nseg])."""
    return _Solve.apply(f, g, solver)
