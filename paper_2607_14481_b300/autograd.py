"""torch.autograd adjoint of the rasterizer: forward = gs_project + gs_bin_sort
+ gs_render_fwd, backward = gs_render_bwd in its replay form: per tile the
forward's list is walked again front to back to recover each pixel's final
transmittance and last blended splat, then back to front recovering
T_i = T_{i+1} / (1 - alpha_i).  Between the two passes only the per-Gaussian
splat records and the tile lists are kept; no per-pixel state (not the image,
not the transmittance) is stored.

The differentiable inputs are the flat parameter buffer of an Arena (its
layout is the library's: means4 | scale_opa | quat | planar SH) and a
per-view pose twist xi = (v, omega) [V,6] at which the camera poses are
perturbed on the left, T <- Exp(xi) T.  The twist must be zero: its gradient
is the pose gradient at the current poses, the quantity a pose optimiser
consumes.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from .raster import Arena, Rasterizer


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, buf: torch.Tensor, pose_twist: torch.Tensor, arena: Arena, rast: Rasterizer,
                poses: torch.Tensor, want_alpha: bool):
        if pose_twist is not None and bool(torch.any(pose_twist != 0)):
            raise ValueError("pose_twist must be zero (the gradient is taken at the current poses)")
        image = rast.new_image()
        alpha = rast.new_alpha() if want_alpha else None
        rast.forward(arena, poses, image, alpha, check=True)
        ctx.arena, ctx.rast, ctx.poses = arena, rast, poses
        ctx.want_alpha = want_alpha
        # nothing per pixel is kept: the backward replays the tile lists
        if want_alpha:
            return image, alpha
        return image, torch.empty(0, device=image.device)

    @staticmethod
    def backward(ctx, dimage: torch.Tensor, dalpha: Optional[torch.Tensor]):
        arena, rast, poses = ctx.arena, ctx.rast, ctx.poses
        grads = arena.like()
        dpose = torch.zeros((rast.views, 6), dtype=torch.float32, device=dimage.device)
        da = dalpha.contiguous() if (ctx.want_alpha and dalpha is not None) else None
        # image=None selects the replay backward (recomputed transmittance)
        rast.backward(arena, poses, dimage.contiguous(), da, grads, dpose, None)
        return grads.buf, dpose, None, None, None, None


def render(arena: Arena, rast: Rasterizer, poses: torch.Tensor, pose_twist: Optional[torch.Tensor] = None,
           want_alpha: bool = False) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
    """Differentiable render of the rasterizer's views.  Returns the flat image
    (views concatenated, each [3,H,W]) and, if asked, the flat alpha.  Gradients
    flow to arena.buf (set requires_grad on it) and to pose_twist.  One
    Rasterizer holds the state of one outstanding forward."""
    if pose_twist is None:
        pose_twist = torch.zeros((rast.views, 6), dtype=torch.float32, device=arena.buf.device)
    img, al = _RenderFn.apply(arena.buf, pose_twist, arena, rast, poses, want_alpha)
    return img, (al if want_alpha else None)
