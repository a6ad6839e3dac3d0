"""torch.autograd.Function over the fused evaluation kernel.

Forward and backward both come from one launch of ``cr_eval``: the kernel
writes the cost and the hand-written Jacobian-transpose gradient (link
transforms recomputed on chip, never stored in HBM); backward only scales the
stored gradient by the incoming cost gradient.
"""
from __future__ import annotations

import torch

from . import crgb


class EvalFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, robot, problem, params):
        out = crgb.evaluate(robot, problem, theta.detach(), params, want_grad=True,
                            want_terms=False)
        ctx.save_for_backward(out["grad"])
        ctx.mark_non_differentiable(out["cfree"])
        return out["cost"], out["cfree"]

    @staticmethod
    def backward(ctx, grad_cost, grad_cfree):
        (g,) = ctx.saved_tensors
        return grad_cost.view(-1, 1, 1) * g, None, None, None


def trajectory_cost(theta, robot, problem, params=None):
    """Differentiable total cost [B] of trajectories theta [B, H, dof]."""
    cost, _ = EvalFn.apply(theta, robot, problem, params)
    return cost
