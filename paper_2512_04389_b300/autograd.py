"""Differentiable sparse solve x = A^{-1} b on the GPU factors.

``LUSolve.apply(values, b, plan)`` factors A (values in the CSC order of the
plan's pattern) and solves.  Its hand-written backward reuses the stored
factors: lam = A^{-T} dl/dx by the transposed solve (U^T then L^T), then
dl/db = lam and dl/dvalues[p] = -sum_c lam(row_p, c) x(col_p, c), gathered
over A's pattern by a library kernel.  No dense matrix is ever formed.
"""
import torch

from . import slu as S


class LUSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, plan):
        F = S.Factor(plan, values.detach().contiguous())
        x = F.solve(b.detach())
        ctx.factor = F
        ctx.b_was_vector = b.dim() == 1
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        F = ctx.factor
        lam = F.solve_transpose(gx.contiguous())
        lm = lam.reshape(lam.shape[0], -1)
        xm = x.reshape(x.shape[0], -1)
        gv = F.grad_values(lm, xm)
        return gv, lam, None


def lu_solve(values, b, plan):
    """x = A(values)^{-1} b, differentiable in values and b."""
    return LUSolve.apply(values, b, plan)
