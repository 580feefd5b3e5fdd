"""Differentiable solve: x = A^{-1} b with gradients for b and A's stored values.

The backward pass is an adjoint solve A^T lambda = dL/dx with the transposed
MGR cycle (FGMRES on A^T, every step in the CUDA library), giving
dL/db = lambda and dL/dA_ij = -lambda_i x_j on the stored block pattern.
"""
from __future__ import annotations

import torch

from .mgr import MGRSolver


class MGRSolveFn(torch.autograd.Function):
    """forward(values, b, solver, rtol, maxit) -> x.

    `values` is the (nnzb, b, b) tensor of A's stored blocks.  When they are
    not the values the solver last took (at setup, refresh or update), they
    are handed to the solver's outer operator first (mgr_update_values), so x
    and the gradients always belong to `values`; the hierarchy built before
    stays the preconditioner (call solver.refresh to rebuild it).
    """

    @staticmethod
    def forward(ctx, values, rhs, solver: MGRSolver, rtol: float, maxit: int):
        if tuple(values.shape) != (solver.nnzb, solver.b, solver.b):
            raise ValueError(f"values has shape {tuple(values.shape)}, the solver's pattern "
                             f"holds ({solver.nnzb}, {solver.b}, {solver.b}) blocks")
        if not solver.holds_values(values):
            solver.update_values(values.detach())
        x, info = solver.solve(rhs.contiguous(), rtol=rtol, maxit=maxit)
        if info["status"] != 0:
            raise RuntimeError(f"forward solve did not converge: {info}")
        ctx.solver, ctx.rtol, ctx.maxit = solver, rtol, maxit
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, info = ctx.solver.solve(gx.contiguous(), rtol=ctx.rtol, maxit=ctx.maxit,
                                     transpose=True)
        if info["status"] != 0:
            raise RuntimeError(f"adjoint solve did not converge: {info}")
        dvals = ctx.solver.grad_values(lam, x)
        return dvals, lam, None, None, None


def mgr_solve_fn(values, rhs, solver: MGRSolver, rtol: float = 1e-10, maxit: int = 1000):
    """x = A^{-1} rhs, differentiable in `values` (A's blocks) and `rhs`."""
    return MGRSolveFn.apply(values, rhs, solver, rtol, maxit)
