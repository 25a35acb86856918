"""Local bundle adjustment (Sec. 5.1) through gs_ba_solve: argument
marshalling only; every step runs in the library's kernels."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import torch

from . import _lib


def _p(t: Optional[torch.Tensor]):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class BundleAdjuster:
    """Device workspace and problem description of one local BA window:
    num_cams keyframes (fixed[k] = True: kept), num_points landmarks with
    obs_per_point observation slots each (obs_cam int32 [K, M], -1 = empty;
    obs_uv float32 [K, M, 2]; both on the device).  solve() runs gs_ba_solve on
    the current stream without host synchronisation, so it can be captured in
    a CUDA graph."""

    def __init__(self, obs_cam: torch.Tensor, obs_uv: torch.Tensor, num_cams: int, fixed: Sequence[bool],
                 cx: float, cy: float, opt_focal: bool = True, max_iters: int = 64):
        self.L = _lib.load()
        if obs_cam.dtype != torch.int32 or obs_uv.dtype != torch.float32 or not obs_cam.is_cuda:
            raise TypeError("obs_cam must be device int32 [K, M] and obs_uv device float32 [K, M, 2]")
        K, M = obs_cam.shape
        if tuple(obs_uv.shape) != (K, M, 2):
            raise ValueError("obs_uv must be [K, M, 2]")
        if len(fixed) != num_cams:
            raise ValueError("fixed must have one flag per keyframe")
        self.obs_cam, self.obs_uv = obs_cam.contiguous(), obs_uv.contiguous()
        self.K, self.M, self.N = int(K), int(M), int(num_cams)
        self.prob = _lib.GsBaProblem()
        self.prob.num_cams, self.prob.num_points, self.prob.obs_per_point = self.N, self.K, self.M
        self.prob.opt_focal = 1 if opt_focal else 0
        self.prob.cx, self.prob.cy = float(cx), float(cy)
        self.prob.obs_cam, self.prob.obs_uv = self.obs_cam.data_ptr(), self.obs_uv.data_ptr()
        for k, f in enumerate(fixed):
            self.prob.fixed[k] = 1 if f else 0
        dev = obs_cam.device
        nbytes = int(self.L.gs_ba_workspace_bytes(self.N, self.K, self.M))
        if nbytes == 0:
            raise ValueError("problem size out of range")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off:off + nbytes]
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.trace = torch.zeros(max(1, max_iters), 4, dtype=torch.float64, device=dev)
        self.max_iters = int(max_iters)

    def solve(self, poses: torch.Tensor, points: torch.Tensor, focal: torch.Tensor, iters: int = 10,
              lambda0: float = 1e-3) -> None:
        """poses float32 [N, 12] (world->camera [R | t] row-major), points
        float32 [K, 3], focal float32 [1]: device tensors updated in place;
        self.trace[:iters] receives (cost, candidate cost, lambda, accepted)."""
        for t, shape in ((poses, (self.N, 12)), (points, (self.K, 3)), (focal, (1,))):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"expected a contiguous device float32 tensor of shape {shape}")
        if iters > self.max_iters:
            raise ValueError(f"iters > max_iters ({self.max_iters})")
        _lib.check(self.L.gs_ba_solve(C.byref(self.prob), _p(poses), _p(points), _p(focal), int(iters),
                                      float(lambda0), _p(self.trace), _p(self.status), _p(self.ws_view),
                                      self.ws_view.numel(), _stream()), "gs_ba_solve")


def bundle_adjust(poses, points, focal: float, obs_cam, obs_uv, cx: float, cy: float, fixed, opt_focal=True,
                  iters=10, lambda0=1e-3, device="cuda"):
    """One-shot helper: copies the problem to the device, runs `iters`
    iterations and returns (poses [N, 12], points [K, 3], focal, trace
    [iters, 4], status) on the host."""
    dev = torch.device(device)
    P = torch.as_tensor(poses, dtype=torch.float32).reshape(-1, 12).to(dev).contiguous()
    X = torch.as_tensor(points, dtype=torch.float32).reshape(-1, 3).to(dev).contiguous()
    f = torch.tensor([float(focal)], dtype=torch.float32, device=dev)
    cam = torch.as_tensor(obs_cam, dtype=torch.int32).to(dev).contiguous()
    uv = torch.as_tensor(obs_uv, dtype=torch.float32).to(dev).contiguous()
    ba = BundleAdjuster(cam, uv, P.shape[0], [bool(v) for v in fixed], cx, cy, opt_focal, max_iters=max(1, iters))
    ba.solve(P, X, f, iters=iters, lambda0=lambda0)
    torch.cuda.current_stream().synchronize()
    return (P.cpu().numpy(), X.cpu().numpy(), float(f.item()), ba.trace[:iters].cpu().numpy(),
            int(ba.status.item()))
