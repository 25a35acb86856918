"""One optimisation iteration of the joint Gaussian optimisation (render ->
loss -> backward -> Adam, §5.2), over a fixed set of views, runnable eagerly or
captured once in a CUDA graph and replayed.

Every buffer is allocated before the first run and the Adam step counters
live on the device, so a captured step replays with no host work beyond the
graph launch.  All arithmetic runs in libgs kernels.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import raster
from .raster import Arena, ImageLoss, Rasterizer


class TrainStep:
    """Forward, image loss (L1 or MSE), backward (parameters and pose twist),
    fused Adam (parameters + poses) for the views of `rast`; with `adam` (a
    raster.adam_params config whose step_dev is this step's) the parameters'
    Adam step runs inside the per-Gaussian backward.  With fused=True
    (the default) the composite, the loss and the per-pixel backward run as
    one persistent launch over all views' tiles (gs_render_fused); otherwise
    as three launches (gs_render_fwd, gs_image_loss, gs_render_bwd_pixels).

    poses, dpose, pose_m, pose_v, pose_steps: device tensors with one row per
    view of this step (slices of larger per-trajectory tensors are fine);
    targets: flat device tensor laid out like the rendered image;
    step_dev: device int32 scalar shared by every step of a run."""

    def __init__(self, arena: Arena, grads: Arena, m: Arena, v: Arena, groups, rast: Rasterizer,
                 poses: torch.Tensor, targets: torch.Tensor, step_dev: torch.Tensor,
                 pose_m: Optional[torch.Tensor] = None, pose_v: Optional[torch.Tensor] = None,
                 pose_steps: Optional[torch.Tensor] = None, pose_lr: float = 1e-4, loss_kind: int = 0,
                 status: Optional[torch.Tensor] = None, image: Optional[torch.Tensor] = None,
                 dimage: Optional[torch.Tensor] = None, loss: Optional[ImageLoss] = None,
                 cams: Optional[Sequence] = None, fused: bool = True, adam=None):
        self.arena, self.grads, self.m, self.v, self.groups = arena, grads, m, v, groups
        self.rast = rast
        self.cams = list(cams) if cams is not None else list(rast.cams)
        self.poses = poses
        self.targets = targets
        self.step_dev = step_dev
        dev = arena.buf.device
        V = len(self.cams)
        self.dpose = torch.zeros((V, 6), dtype=torch.float32, device=dev)
        self.pose_m, self.pose_v, self.pose_steps = pose_m, pose_v, pose_steps
        self.pose_lr = pose_lr
        self.kind = loss_kind
        self.status = status
        self.img = image if image is not None else rast.new_image()
        self.dimg = dimage if dimage is not None else rast.new_image()
        self.loss = loss if loss is not None else ImageLoss(dev)
        self.fused = fused
        # gs_adam_params_cfg (raster.adam_params): the parameters' Adam step
        # fused into the per-Gaussian backward; None: a separate gs_adam_step
        self.adam = adam
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    def body(self) -> None:
        r = self.rast
        r.set_cameras(self.cams)
        r.project(self.arena, self.poses)
        r.bin_sort()
        if self.fused:
            # composite + loss + per-pixel backward: one persistent launch
            r.fused(self.targets, self.kind, self.img, None, self.loss.loss)
        else:
            r.render_fwd(self.img, None)
            self.loss(self.img, self.targets, self.dimg, self.kind)
            r.backward_pixels(self.dimg, None, self.img)
        with_pose = self.pose_m is not None
        groups = self.groups
        if self.adam is not None:
            r.backward_gaussians_adam(self.arena, self.poses, self.grads, self.m, self.v, self.adam, self.dpose)
            # the parameters are updated; the poses and the step counter remain
            # (an empty group when there is no pose step)
            groups = [] if with_pose else [raster.empty_adam_group()]
        else:
            r.backward_gaussians(self.arena, self.poses, self.grads, self.dpose)
        raster.adam_step(self.arena, self.grads, self.m, self.v, 0, groups, status=self.status,
                         pose=self.poses if with_pose else None, dpose=self.dpose if with_pose else None,
                         pose_m=self.pose_m, pose_v=self.pose_v, pose_lr=self.pose_lr,
                         step_dev=self.step_dev, pose_steps_dev=self.pose_steps)

    def capture(self, pool=None) -> None:
        """Record body() into a CUDA graph (the recorded kernels read every
        count from device memory, so the graph stays valid while the pair
        capacity is not exceeded)."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, pool=pool):
            self.body()
        self.graph = g

    def run(self) -> None:
        if self.graph is not None:
            self.graph.replay()
        else:
            self.body()
