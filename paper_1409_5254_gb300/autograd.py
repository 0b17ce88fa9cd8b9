"""torch.autograd.Function over the batched solve and its hand-written adjoint.

u = DGTimeSolve.apply(f, u0, lam, batch): forward runs tmg_solve_batched on the
packed load vectors f and initial values u0 (the batch plan holds p_t, tau
and the lambda values it was built for -- ``lam`` is passed only so that
autograd can return dJ/dlambda).  backward runs tmg_adjoint_batched: the
transposed, backward-in-time cycle gives dJ/df = mu, dJ/du0 = a^T mu_0 and
dJ/dlambda = -tau sum_n mu_n^T Mhat u_n per instance.  With
save_solution=False the forward solution is not kept for backward but
recomputed there (halves the memory held between the passes).
"""
from __future__ import annotations

import numpy as np
import torch

from .tmg import Batch


class DGTimeSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, u0, lam, batch: Batch, save_solution: bool = True):
        if lam.numel() != batch.n or not np.allclose(lam.detach().cpu().numpy(), batch.lam, rtol=0, atol=0):
            raise ValueError("lam differs from the values the batch plan was built for")
        u = batch.solve(f.contiguous(), u0.contiguous())
        ctx.batch = batch
        ctx.save_solution = save_solution
        if save_solution:
            ctx.save_for_backward(u)
        else:
            ctx.save_for_backward(f, u0)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        if ctx.save_solution:
            (u,) = ctx.saved_tensors
        else:
            f, u0 = ctx.saved_tensors
            u = ctx.batch.solve(f.contiguous(), u0.contiguous())
        dJdf, du0, dlam = ctx.batch.adjoint(grad_u.contiguous(), u)
        return dJdf, du0, dlam, None, None


def solve(f, u0, lam, batch: Batch, save_solution: bool = True):
    """Differentiable batched solve (see DGTimeSolve)."""
    return DGTimeSolve.apply(f, u0, lam, batch, save_solution)
