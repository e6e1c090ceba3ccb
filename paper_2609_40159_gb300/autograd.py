"""Differentiable solves.

The backward of x = L^{-1} b is the transpose solve g_b = L^{-T} g_x, run by
the library over the reversed row / level order, followed by the value
gradient on L's pattern, g_L[i, j] = -sum_r g_b[i, r] x[j, r] (diagonal
included).  x is kept from the forward pass, not recomputed.  For a rewritten
system x = L'^{-1} (b + T b) the gradient with respect to b is
g_b' + T^T g_b' with g_b' = L'^{-T} g_x, and the value gradient is on L'.
"""
from __future__ import annotations

import torch

from .api import BatchPlan, Plan


class SpTRSVFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, plan):
        if vals.data_ptr() != plan.A.vals.data_ptr():
            raise ValueError("vals must be the value tensor the plan was built on")
        x = plan.solve(b)
        ctx.plan = plan
        ctx.squeeze = b.dim() == 1
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        plan = ctx.plan
        n = plan.A.n
        g = gx.contiguous().view(n, -1)
        x2 = x.view(n, -1)
        gbp = plan.solve_transpose(g)
        gvals = plan.grad_vals(gbp, x2) if ctx.needs_input_grad[0] else None
        gb = None
        if ctx.needs_input_grad[1]:
            gb = plan.tt_apply(gbp) if plan.T is not None else gbp
            if ctx.squeeze:
                gb = gb.view(-1)
        return gvals, gb, None


def solve(plan: Plan, b: torch.Tensor, vals: torch.Tensor | None = None) -> torch.Tensor:
    """Autograd-aware x = L^{-1} b (L'^{-1}(b + T b) for a rewritten plan)."""
    return SpTRSVFunction.apply(plan.A.vals if vals is None else vals, b, plan)


class BatchSpTRSVFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals_packed, b_packed, plan):
        if vals_packed.data_ptr() != plan.vals.data_ptr() or vals_packed.numel() != plan.vals.numel():
            raise ValueError("vals_packed must be the plan's packed value tensor (plan.vals)")
        x = plan.solve(b_packed)
        ctx.plan = plan
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        plan = ctx.plan
        gbp = plan.solve_transpose(gx.contiguous())
        gvals = plan.grad_vals(gbp, x) if ctx.needs_input_grad[0] else None
        gb = None
        if ctx.needs_input_grad[1]:
            gb = plan.tt_apply(gbp) if any(T is not None for T in plan.Ts) else gbp
        return gvals, gb, None


def batch_solve(plan: BatchPlan, b_packed: torch.Tensor, vals_packed: torch.Tensor | None = None) -> torch.Tensor:
    """Autograd-aware batched solve (x_m = L_m^{-1} b_m, or L'_m^{-1}(b_m + T_m b_m)
    for a rewritten system, every system in one launch).  ``vals_packed``
    must be the plan's packed value tensor ``plan.vals`` (default), whose
    slice [vals_offset[m], vals_offset[m+1]) is what system m's solve reads;
    its gradient is the value gradient of every system on its own (for a
    rewritten system: L''s) pattern.  The plan needs transpose=True for the
    backward pass."""
    return BatchSpTRSVFunction.apply(plan.vals if vals_packed is None else vals_packed, b_packed, plan)
