"""torch.autograd.Function for the shadow-minutes of a ground region as a function of the
building heights.  Forward and backward both run in the CUDA library: the forward pass sets
the heights (the scene's mesh and BVH are rebuilt on the device), accumulates the step
masks, and computes S and dS/dh from the sun times at which each receiver's shadow status
flips (FP64 for the grazing geometry); backward scales the stored gradient."""
from __future__ import annotations

import torch

from . import binding as B


class ShadowMinutes(torch.autograd.Function):
    """S(h) = weighted shadow-minutes of `grid` under `sun` for building heights h."""

    @staticmethod
    def forward(ctx, heights, scene, grid, sun, step_minutes, weights=None):
        scene.set_heights(heights)
        g, S = B.sa_height_grad(scene, grid, sun, step_minutes, weights)
        ctx.save_for_backward(g.to(heights.dtype))
        return S.to(heights.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None


def shadow_minutes(heights, scene, grid, sun, step_minutes, weights=None):
    return ShadowMinutes.apply(heights, scene, grid, sun, step_minutes, weights)
