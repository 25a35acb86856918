"""Tensor-level API: device buffers held in torch tensors, every step run by
libgs (include/gs.h).  torch supplies device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from .synth import Camera, Scene


def _p(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Arena:
    """Per-Gaussian float arrays in the library's layout inside one flat
    float32 buffer: [means4 (4n) | scale_opa (4n) | quat (4n) | sh (3 nc n)],
    padded to a multiple of 4 floats.  Parameters, gradients and both Adam
    moments use the same layout, so one fused Adam launch covers them all."""

    def __init__(self, n: int, sh_degree: int, device="cuda", buf: Optional[torch.Tensor] = None):
        self.n = int(n)
        self.sh_degree = int(sh_degree)
        self.nc = (self.sh_degree + 1) ** 2
        self.size = 12 * self.n + 3 * self.nc * self.n
        self.padded = (self.size + 3) // 4 * 4
        if buf is None:
            buf = torch.zeros(max(self.padded, 4), dtype=torch.float32, device=device)
        self.buf = buf
        n4 = 4 * self.n
        self.means4 = buf[0:n4].view(self.n, 4)
        self.scale_opa = buf[n4:2 * n4].view(self.n, 4)
        self.quat = buf[2 * n4:3 * n4].view(self.n, 4)
        self.sh = buf[3 * n4:3 * n4 + 3 * self.nc * self.n].view(3 * self.nc, self.n)

    @classmethod
    def from_scene(cls, sc: Scene, device="cuda", capacity: Optional[int] = None) -> "Arena":
        """The scene's Gaussians in the first sc.n rows; with a larger
        capacity the remaining rows are zero (room for hierarchy nodes)."""
        a = cls(sc.n if capacity is None else capacity, sc.sh_degree, device)
        h = np.zeros(a.padded, np.float32)
        n, nc, k = a.n, a.nc, sc.n
        assert k <= n
        h[0:4 * n].reshape(n, 4)[:k, :3] = sc.means
        so = h[4 * n:8 * n].reshape(n, 4)
        so[:k, :3] = sc.log_scales
        so[:k, 3] = sc.opa_logits
        h[8 * n:12 * n].reshape(n, 4)[:k] = sc.quats
        h[12 * n:12 * n + 3 * nc * n].reshape(3 * nc, n)[:, :k] = sc.sh.reshape(k, 3 * nc).T
        a.buf.copy_(torch.from_numpy(h).to(a.buf.device))
        return a

    def like(self) -> "Arena":
        return Arena(self.n, self.sh_degree, self.buf.device)

    def to_natural(self) -> dict:
        """Host float64 copies in natural layout (means [n,3], log_scales [n,3],
        quats [n,4], opa_logits [n], sh [n,3,nc])."""
        h = self.buf.detach().cpu().numpy().astype(np.float64)
        n, nc = self.n, self.nc
        m4 = h[0:4 * n].reshape(n, 4)
        so = h[4 * n:8 * n].reshape(n, 4)
        return {"means": m4[:, :3].copy(), "means_pad": m4[:, 3].copy(), "log_scales": so[:, :3].copy(),
                "opa_logits": so[:, 3].copy(), "quats": h[8 * n:12 * n].reshape(n, 4).copy(),
                "sh": h[12 * n:12 * n + 3 * nc * n].reshape(3 * nc, n).T.reshape(n, 3, nc).copy()}

    def struct(self, n: Optional[int] = None):
        """gs_params over the first n rows (default all), SH planes strided by
        the arena's row count."""
        return _lib.GsParams(self.means4.data_ptr(), self.scale_opa.data_ptr(), self.quat.data_ptr(),
                             self.sh.data_ptr(), self.n if n is None else int(n), self.sh_degree, self.n)

    def rw_struct(self):
        """The same arrays as writable pointers (gs_grads layout)."""
        return _lib.GsGrads(self.means4.data_ptr(), self.scale_opa.data_ptr(), self.quat.data_ptr(),
                            self.sh.data_ptr(), self.n, self.sh_degree, self.n)

    def adam_groups(self, lr_means=1.6e-4, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3,
                    lr_sh_dc=2.5e-3, lr_sh_rest=1.25e-4) -> List[_lib.GsAdamGroup]:
        """Non-overlapping groups, one per parameter kind; the scale_opa float4
        gives its first three lanes the scale rate and its fourth the opacity
        rate; per channel the SH DC plane (k = 0) and the higher bands
        (k = 1 .. nc-1) are separate groups."""
        n, nc = self.n, self.nc
        G = _lib.GsAdamGroup
        f4 = C.c_float * 4
        groups = [G(0, 4 * n, f4(lr_means, lr_means, lr_means, 0.0)),
                  G(4 * n, 8 * n, f4(lr_scale, lr_scale, lr_scale, lr_opacity)),
                  G(8 * n, 12 * n, f4(lr_quat, lr_quat, lr_quat, lr_quat))]
        for ch in range(3):
            b = 12 * n + ch * nc * n
            groups.append(G(b, b + n, f4(lr_sh_dc, lr_sh_dc, lr_sh_dc, lr_sh_dc)))
            if nc > 1:
                groups.append(G(b + n, b + nc * n, f4(lr_sh_rest, lr_sh_rest, lr_sh_rest, lr_sh_rest)))
        return groups


def empty_adam_group() -> _lib.GsAdamGroup:
    """An Adam group of no element (for a gs_adam_step that only advances the
    device step counter)."""
    return _lib.GsAdamGroup(0, 0, (C.c_float * 4)(0.0, 0.0, 0.0, 0.0))


def adam_params(sh_degree: int, lr_means=1.6e-4, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3, lr_sh_dc=2.5e-3,
                lr_sh_rest=1.25e-4, beta1=0.9, beta2=0.999, eps=1e-15, step: int = 0,
                step_dev: Optional[torch.Tensor] = None, skip_dev: Optional[torch.Tensor] = None,
                status: Optional[torch.Tensor] = None) -> _lib.GsAdamParamsCfg:
    """gs_adam_params_cfg with the rates of Arena.adam_groups (the same update
    as gs_adam_step over those groups)."""
    nc = (sh_degree + 1) ** 2
    f4 = C.c_float * 4
    sh = (C.c_float * 48)(*[(lr_sh_dc if p % nc == 0 else lr_sh_rest) if p < 3 * nc else 0.0 for p in range(48)])
    return _lib.GsAdamParamsCfg(f4(lr_means, lr_means, lr_means, 0.0), f4(lr_scale, lr_scale, lr_scale, lr_opacity),
                                f4(lr_quat, lr_quat, lr_quat, lr_quat), sh, beta1, beta2, eps, int(step), 15,
                                _p(step_dev), _p(skip_dev), _p(status))


def sim3_update(arena: Arena, kf: torch.Tensor, sim3: torch.Tensor, status: Optional[torch.Tensor] = None):
    """gs_sim3_update: every Gaussian of the arena moves with the Sim(3)
    correction of its keyframe kf[i] (int32 [n], device; < 0: unchanged);
    sim3 [K, 8] float32 (qw, qx, qy, qz, tx, ty, tz, s).  Returns the status
    word (bit 0: a keyframe id without a correction)."""
    L = _lib.load()
    assert kf.dtype == torch.int32 and kf.numel() >= arena.n and sim3.dtype == torch.float32
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=arena.buf.device)
    rw = arena.rw_struct()
    sim3 = sim3.contiguous()
    _lib.check(L.gs_sim3_update(C.byref(rw), _p(kf), _p(sim3), sim3.shape[0], _p(status), _stream()),
               "gs_sim3_update")
    return status


class LodHierarchy:
    """Three-level hierarchy (gs_lod_build) over the first n_leaf Gaussians of
    a node arena; coarse nodes are written after the leaves."""

    def __init__(self, arena: Arena, n_leaf: int):
        self.L = _lib.load()
        self.arena, self.n_leaf = arena, int(n_leaf)
        self.n_nodes = int(self.L.gs_lod_nodes(self.n_leaf))
        if self.n_nodes > arena.n:
            raise ValueError(f"arena holds {arena.n} rows, the hierarchy needs {self.n_nodes}")
        dev = arena.buf.device
        self.parent = torch.empty(max(1, self.n_nodes), dtype=torch.int32, device=dev)
        self.ws = torch.empty(max(1, self.L.gs_lod_build_workspace(self.n_leaf)), dtype=torch.uint8, device=dev)

    def build(self) -> None:
        rw = self.arena.rw_struct()
        _lib.check(self.L.gs_lod_build(C.byref(rw), self.n_leaf, _p(self.parent), _p(self.ws), self.ws.numel(),
                                       _stream()), "gs_lod_build")

    def nodes(self):
        return self.arena.struct(self.n_nodes)


class Hierarchy:
    """Progressive hierarchy (gs_hier_*) over the rows of a node arena: the
    first n_leaf rows are the leaves, all active; analyses append merged
    nodes after the rows in use (up to the arena's rows)."""

    def __init__(self, arena: Arena, n_leaf: int):
        self.L = _lib.load()
        self.arena = arena
        cap = arena.n
        dev = arena.buf.device
        self.capacity = cap
        self.parent = torch.full((cap,), -1, dtype=torch.int32, device=dev)
        self.child = torch.full((4 * cap,), -1, dtype=torch.int32, device=dev)
        self.active = torch.zeros(cap, dtype=torch.uint8, device=dev)
        self.active[:n_leaf] = 1
        self.n_nodes = torch.tensor([n_leaf], dtype=torch.int32, device=dev)
        self.info = torch.zeros(8, dtype=torch.int32, device=dev)
        self.ws = torch.empty(max(1, self.L.gs_hier_workspace(cap)), dtype=torch.uint8, device=dev)
        self.pose = torch.zeros(12, dtype=torch.float32, device=dev)

    def struct(self):
        return _lib.GsHier(self.parent.data_ptr(), self.child.data_ptr(), self.active.data_ptr(),
                           self.n_nodes.data_ptr(), self.info.data_ptr(), self.capacity)

    def _pose(self, cam: Camera):
        self.pose.copy_(torch.from_numpy(np.asarray(cam.pose12(), np.float32).reshape(-1)))
        return _p(self.pose)

    def analyze(self, cam: Camera, znear=0.2, tau_l=0.5, m: Optional[Arena] = None, v: Optional[Arena] = None):
        rw, h = self.arena.rw_struct(), self.struct()
        ms = m.rw_struct() if m is not None else None
        vs = v.rw_struct() if v is not None else None
        c = cameras_struct([cam])
        _lib.check(self.L.gs_hier_analyze(C.byref(rw), C.byref(h), C.byref(ms) if ms else None,
                                          C.byref(vs) if vs else None, self._pose(cam), c, float(znear),
                                          float(tau_l), _p(self.ws), self.ws.numel(), _stream()), "gs_hier_analyze")

    def refine(self, cam: Camera, znear=0.2, tau_h=1.0, passes=16, m: Optional[Arena] = None,
               v: Optional[Arena] = None):
        rw, h = self.arena.rw_struct(), self.struct()
        ms = m.rw_struct() if m is not None else None
        vs = v.rw_struct() if v is not None else None
        c = cameras_struct([cam])
        _lib.check(self.L.gs_hier_refine(C.byref(rw), C.byref(h), C.byref(ms) if ms else None,
                                         C.byref(vs) if vs else None, self._pose(cam), c, float(znear),
                                         float(tau_h), int(passes), _p(self.ws), self.ws.numel(), _stream()),
                   "gs_hier_refine")

    def state(self) -> dict:
        """Host copies (synchronises): n_nodes, info, parent, child [cap,4], active."""
        n = int(self.n_nodes.item())
        return {"n_nodes": n, "info": self.info.cpu().numpy().astype(np.int64), "parent": self.parent.cpu().numpy(),
                "child": self.child.cpu().numpy().reshape(-1, 4), "active": self.active.cpu().numpy()}


def cameras_struct(cams: Sequence[Camera]):
    arr = (_lib.GsCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = _lib.GsCamera(c.fx, c.fy, c.cx, c.cy, c.width, c.height)
    return arr


def poses_tensor(cams: Sequence[Camera], device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.stack([c.pose12() for c in cams]).astype(np.float32)).to(device).contiguous()


def parse_fused_schedule(name: str):
    """(tile, schedule bits) of a fused-pass schedule name as autotune_fused
    reports them: "<tw>x<th>_b<128|64|32>_<viewmajor|longest>"."""
    parts = name.split("_")
    if len(parts) != 3 or not parts[1].startswith("b"):
        raise ValueError(f"fused schedule {name!r}: expected <tw>x<th>_b<n>_<viewmajor|longest>")
    tile = tuple(int(x) for x in parts[0].split("x"))
    if tile not in _lib.TILE_SHAPES:
        raise ValueError(f"fused schedule {name!r}: tile shape not one of {_lib.TILE_SHAPES}")
    batches = {128: 0, 64: 1, 32: 2}
    bt = int(parts[1][1:])
    if bt not in batches or parts[2] not in ("viewmajor", "longest"):
        raise ValueError(f"fused schedule {name!r}: splats per batch 128, 64 or 32; order viewmajor or longest")
    bits = _lib.GS_SCHED_FUSED_BATCH(batches[bt]) | (_lib.GS_SCHED_FUSED_LONGEST_FIRST if parts[2] == "longest" else 0)
    return tile, bits


class Rasterizer:
    """Splat records, tile lists and workspaces for a fixed set of views.

    forward(): gs_project -> gs_bin_sort -> gs_render_fwd
    backward(): gs_render_bwd
    The pair capacity grows on overflow when forward(check=True) reads the
    device counts (one 16-byte copy); with check=False nothing synchronises."""

    def __init__(self, n: int, sh_degree: int, cams: Sequence[Camera], bg=(0.0, 0.0, 0.0), znear=0.2,
                 clamp_jacobian=True, capacity: Optional[int] = None, device="cuda", keep_keys=False,
                 largest_first: bool = True, tile=(16, 16)):
        self.L = _lib.load()
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.device = torch.device(device)
        self.tile = (int(tile[0]), int(tile[1]))
        self.set_cameras(cams)
        self.cfg = _lib.GsRasterCfg(self.tile[0], self.tile[1], (C.c_float * 3)(*bg), float(znear),
                                    int(bool(clamp_jacobian)))
        V = self.views
        self.splat_buf = torch.empty(self.L.gs_splats_bytes(self.n, V), dtype=torch.uint8, device=self.device)
        self.splats = _lib.GsSplats()
        _lib.check(self.L.gs_splats_carve(_p(self.splat_buf), self.n, V, C.byref(self.splats)), "gs_splats_carve")
        self.pair_off = torch.empty(max(1, self.n * V), dtype=torch.int32, device=self.device)
        self.counts = torch.zeros(4, dtype=torch.int32, device=self.device)
        self.keep_keys = keep_keys
        self.largest_first = largest_first
        self.capacity = 0
        self.set_capacity(capacity if capacity is not None else max(4096, 4 * self.n * V))

    def set_cameras(self, cams: Sequence[Camera]) -> None:
        cams = list(cams)
        if hasattr(self, "views") and len(cams) != self.views:
            raise ValueError("number of views is fixed per Rasterizer")
        self.cams = cams
        self.views = len(cams)
        self.cam_struct = cameras_struct(cams)
        self.num_tiles = self.tiles_for(self.tile)
        # ranges and tile order hold the largest tile count of any supported shape
        self.max_tiles = max(self.tiles_for(t) for t in _lib.TILE_SHAPES)
        self.pixels = sum(c.width * c.height for c in cams)
        if hasattr(self, "ranges") and self.ranges.numel() >= 2 * self.max_tiles:
            if hasattr(self, "ws_bwd") and self.max_tiles > self._ws_tiles:
                self._alloc_pairs()  # the fused pass's per-tile terms for more tiles
            return
        self.ranges = torch.zeros(max(2, 2 * self.max_tiles), dtype=torch.int32, device=self.device)
        self.tile_order = torch.zeros(max(1, self.max_tiles), dtype=torch.int32, device=self.device)
        if hasattr(self, "ws_bwd"):
            self._alloc_pairs()

    def tiles_for(self, tile) -> int:
        tw, th = tile
        return sum(((c.width + tw - 1) // tw) * ((c.height + th - 1) // th) for c in self.cams)

    def set_tile(self, tile) -> None:
        """Tile shape (16x16, 32x8 or 8x32) of the following calls."""
        self.tile = (int(tile[0]), int(tile[1]))
        self.cfg.tile_w, self.cfg.tile_h = self.tile
        self.num_tiles = self.tiles_for(self.tile)

    def set_fused_schedule(self, name: str) -> None:
        """Pins the fused pass's schedule instead of autotuning it: `name` is
        one of autotune_fused's candidates, "<tw>x<th>_b<splats per
        batch>_<viewmajor|longest>" (e.g. "8x32_b64_viewmajor")."""
        tile, bits = parse_fused_schedule(name)
        self.set_tile(tile)
        keep = self.cfg.schedule & ~(_lib.GS_SCHED_FUSED_BATCH(3) | _lib.GS_SCHED_FUSED_LONGEST_FIRST)
        self.cfg.schedule = keep | bits

    def set_capacity(self, cap: int) -> None:
        cap = int(cap)
        if cap == self.capacity:
            return
        self.capacity = cap
        self.vals = torch.empty(max(1, cap), dtype=torch.int32, device=self.device)
        self.keys = torch.empty(max(1, cap), dtype=torch.int64, device=self.device) if self.keep_keys else None
        self._alloc_pairs()

    def _alloc_pairs(self) -> None:
        cap = self.capacity
        self.ws_bin = torch.empty(self.L.gs_bin_sort_workspace(self.n, self.views, cap), dtype=torch.uint8,
                                  device=self.device)
        # the fused pass's workspace: the backward's layout plus its counter and
        # per-tile loss terms, for the most tiles any camera set so far had
        self._ws_tiles = max(self.max_tiles, getattr(self, "_ws_tiles", 0))
        self.ws_bwd = torch.empty(self.L.gs_render_fused_workspace(self.n, self.views, cap, self._ws_tiles),
                                  dtype=torch.uint8, device=self.device)

    def bins_struct(self, with_order: Optional[bool] = None):
        """The tile lists; the longest-first tile order is computed only when
        the schedule reads it (or when asked, for the autotuner)."""
        if with_order is None:
            with_order = bool(self.cfg.schedule & (_lib.GS_SCHED_FWD_LONGEST_FIRST | _lib.GS_SCHED_BWD_LONGEST_FIRST
                                                   | _lib.GS_SCHED_FUSED_LONGEST_FIRST))
        order = self.tile_order.data_ptr() if (self.largest_first and with_order) else None
        return _lib.GsBins(self.vals.data_ptr(), self.ranges.data_ptr(), self.pair_off.data_ptr(),
                           self.keys.data_ptr() if self.keys is not None else None, self.counts.data_ptr(),
                           self.capacity, self.num_tiles, order)

    def new_image(self) -> torch.Tensor:
        return torch.empty(3 * self.pixels, dtype=torch.float32, device=self.device)

    def new_alpha(self) -> torch.Tensor:
        return torch.empty(self.pixels, dtype=torch.float32, device=self.device)

    def split(self, flat: torch.Tensor, channels: int) -> List[torch.Tensor]:
        out, off = [], 0
        for c in self.cams:
            k = channels * c.width * c.height
            t = flat[off:off + k]
            out.append(t.view(channels, c.height, c.width) if channels > 1 else t.view(c.height, c.width))
            off += k
        return out

    # -- stages -----------------------------------------------------------
    def project(self, params: Arena, poses: torch.Tensor) -> None:
        assert poses.is_contiguous() and poses.dtype == torch.float32 and poses.numel() == 12 * self.views
        ps = params.struct()
        _lib.check(self.L.gs_project(C.byref(ps), _p(poses), self.cam_struct, self.views, C.byref(self.cfg),
                                     C.byref(self.splats), _stream()), "gs_project")

    def project_lod(self, lod: "LodHierarchy", poses: torch.Tensor, tau: float = 1.0) -> None:
        """gs_project_lod over the hierarchy's nodes (the Rasterizer holds
        lod.n_nodes Gaussians)."""
        assert self.n == lod.n_nodes
        ps = lod.nodes()
        _lib.check(self.L.gs_project_lod(C.byref(ps), lod.n_leaf, _p(lod.parent), float(tau), _p(poses),
                                         self.cam_struct, self.views, C.byref(self.cfg), C.byref(self.splats),
                                         _stream()), "gs_project_lod")

    def project_hier(self, hier: "Hierarchy", poses: torch.Tensor, tau_h: float = 1.0, from_roots=False) -> None:
        """gs_project_hier: each view's cut of the progressive hierarchy over
        this Rasterizer's n node rows (the active set refined for the view),
        or, from_roots, gs_project_hier_render (the render cut descending from
        the roots)."""
        ps = hier.arena.struct(self.n)
        h = hier.struct()
        fn = self.L.gs_project_hier_render if from_roots else self.L.gs_project_hier
        _lib.check(fn(C.byref(ps), C.byref(h), float(tau_h), _p(poses), self.cam_struct, self.views,
                      C.byref(self.cfg), C.byref(self.splats), _stream()), "gs_project_hier")

    def bin_sort(self) -> None:
        b = self.bins_struct()
        _lib.check(self.L.gs_bin_sort(C.byref(self.splats), self.cam_struct, self.views, C.byref(self.cfg),
                                      C.byref(b), _p(self.ws_bin), self.ws_bin.numel(), _stream()), "gs_bin_sort")

    def bin_sort_noalloc(self) -> None:
        """gs_bin_sort_noalloc: the same binning with libgs's static scratch
        (small scenes; no workspace)."""
        b = self.bins_struct()
        _lib.check(self.L.gs_bin_sort_noalloc(C.byref(self.splats), self.cam_struct, self.views, C.byref(self.cfg),
                                              C.byref(b), _stream()), "gs_bin_sort_noalloc")

    def render_fwd(self, image: torch.Tensor, alpha: Optional[torch.Tensor]) -> None:
        b = self.bins_struct()
        _lib.check(self.L.gs_render_fwd(C.byref(self.splats), C.byref(b), self.cam_struct, self.views,
                                        C.byref(self.cfg), _p(image), _p(alpha), _stream()), "gs_render_fwd")

    def autotune(self, image: torch.Tensor, dimage: torch.Tensor, reps: int = 5) -> dict:
        """gs_autotune_blend on the current tile lists: picks the composite
        and backward schedules (tile order, splats per batch) and keeps them
        in this Rasterizer's config.  Synchronises.  Returns the candidates'
        times and the chosen schedule."""
        # the current lists once more, with their longest-first order
        b = self.bins_struct(with_order=True)
        _lib.check(self.L.gs_bin_sort(C.byref(self.splats), self.cam_struct, self.views, C.byref(self.cfg),
                                      C.byref(b), _p(self.ws_bin), self.ws_bin.numel(), _stream()), "gs_bin_sort")
        t = (C.c_float * 10)()
        _lib.check(self.L.gs_autotune_blend(C.byref(self.splats), C.byref(b), self.cam_struct, self.views,
                                            C.byref(self.cfg), _p(image), _p(dimage), self.n, _p(self.ws_bwd),
                                            self.ws_bwd.numel(), int(reps), t, _stream()), "gs_autotune_blend")
        names = [f"fwd_{o}_{b}" for o in ("natural", "longest") for b in (128, 64, 256)] + \
                [f"bwd_{o}_{b}" for o in ("natural", "longest") for b in (128, 64)]
        return {"schedule": int(self.cfg.schedule), "ms": {k: float(v) for k, v in zip(names, t)}}

    def fused(self, target: torch.Tensor, loss_kind: int, image: torch.Tensor, alpha: Optional[torch.Tensor],
              loss: torch.Tensor) -> None:
        """gs_render_fused: composite, image loss against target and the
        per-pixel backward in one persistent launch; the per-pair gradients
        stay in the workspace for backward_gaussians()."""
        b = self.bins_struct()
        _lib.check(self.L.gs_render_fused(C.byref(self.splats), C.byref(b), self.cam_struct, self.views,
                                          C.byref(self.cfg), _p(target), int(loss_kind), _p(image), _p(alpha),
                                          _p(loss), self.n, _p(self.ws_bwd), self.ws_bwd.numel(), _stream()),
                   "gs_render_fused")

    def autotune_fused(self, params: "Arena", poses: torch.Tensor, target: torch.Tensor, loss_kind: int,
                       image: torch.Tensor, loss: torch.Tensor, reps: int = 5) -> dict:
        """gs_autotune_fused: picks the tile shape, splats per batch and work
        order of the fused pass on this workload (re-projecting and re-binning
        per shape) and keeps them in this Rasterizer.  Synchronises.  Returns
        the candidates' times and the choice."""
        ps = params.struct()
        b = self.bins_struct(with_order=True)
        t = (C.c_float * 18)()
        _lib.check(self.L.gs_autotune_fused(C.byref(ps), _p(poses), self.cam_struct, self.views, C.byref(self.cfg),
                                            C.byref(self.splats), C.byref(b), self.max_tiles, _p(self.ws_bin),
                                            self.ws_bin.numel(), _p(target), int(loss_kind), _p(image), _p(loss),
                                            _p(self.ws_bwd), self.ws_bwd.numel(), int(reps), t, _stream()),
                   "gs_autotune_fused")
        self.tile = (int(self.cfg.tile_w), int(self.cfg.tile_h))
        self.num_tiles = self.tiles_for(self.tile)
        names = [f"{tw}x{th}_b{bt}_{o}" for tw, th in _lib.TILE_SHAPES for bt in (128, 64, 32)
                 for o in ("viewmajor", "longest")]
        return {"tile": list(self.tile), "schedule": int(self.cfg.schedule),
                "ms": {k: float(v) for k, v in zip(names, t)}}

    def render_stats(self) -> dict:
        """Work counts of the current tile lists (synchronises): pairs tested
        (after the kernels' warp culling) and blended by the forward, the
        backward's walk length, list length, and the pairs the plain per-pixel
        loop evaluates (up to each pixel's stop)."""
        st = torch.zeros(5, dtype=torch.int64, device=self.device)
        b = self.bins_struct()
        _lib.check(self.L.gs_render_stats(C.byref(self.splats), C.byref(b), self.cam_struct, self.views,
                                          C.byref(self.cfg), _p(st), _stream()), "gs_render_stats")
        v = st.cpu().numpy()
        return {"tested": int(v[0]), "blended": int(v[1]), "walk": int(v[2]), "listed": int(v[3]),
                "evaluated": int(v[4])}

    def read_counts(self) -> np.ndarray:
        return self.counts.cpu().numpy().view(np.uint32).copy()

    def forward(self, params: Arena, poses: torch.Tensor, image=None, alpha=None, check=True,
                lod: Optional["LodHierarchy"] = None, tau: float = 1.0):
        """Project (with the level-of-detail cut when lod is given), bin and
        composite."""
        image = self.new_image() if image is None else image
        if lod is not None:
            self.project_lod(lod, poses, tau)
        else:
            self.project(params, poses)
        self.bin_sort()
        if check:
            cnt = self.read_counts()
            if cnt[2] & 2:
                raise RuntimeError("gs_bin_sort reported an out-of-range index (internal error)")
            if cnt[2] & 1:
                self.set_capacity(int(cnt[1] * 1.25) + 1024)
                self.bin_sort()
                if self.read_counts()[2] != 0:
                    raise RuntimeError("pair capacity still exceeded after growing it")
        self.render_fwd(image, alpha)
        return image, alpha

    def backward(self, params: Arena, poses: torch.Tensor, dimage: torch.Tensor, dalpha: Optional[torch.Tensor],
                 grads: Arena, dpose: Optional[torch.Tensor], image: Optional[torch.Tensor] = None) -> None:
        """image: the forward's output for the current tile lists; with it and
        no dalpha the per-tile pass is the single front-to-back one."""
        ps = params.struct()
        gs = grads.struct()
        b = self.bins_struct()
        _lib.check(self.L.gs_render_bwd(C.byref(ps), _p(poses), self.cam_struct, self.views, C.byref(self.splats),
                                        C.byref(b), C.byref(self.cfg), _p(dimage), _p(dalpha), _p(image),
                                        C.byref(gs), _p(dpose), _p(self.ws_bwd), self.ws_bwd.numel(), _stream()),
                   "gs_render_bwd")

    def backward_pixels(self, dimage: torch.Tensor, dalpha: Optional[torch.Tensor] = None,
                        image: Optional[torch.Tensor] = None) -> None:
        b = self.bins_struct()
        _lib.check(self.L.gs_render_bwd_pixels(C.byref(self.splats), C.byref(b), self.cam_struct, self.views,
                                               C.byref(self.cfg), _p(dimage), _p(dalpha), _p(image), self.n,
                                               _p(self.ws_bwd), self.ws_bwd.numel(), _stream()),
                   "gs_render_bwd_pixels")

    def backward_gaussians(self, params: Arena, poses: torch.Tensor, grads: Arena,
                           dpose: Optional[torch.Tensor]) -> None:
        ps = params.struct()
        gs = grads.struct()
        b = self.bins_struct()
        _lib.check(self.L.gs_render_bwd_gaussians(C.byref(ps), _p(poses), self.cam_struct, self.views,
                                                  C.byref(self.splats), C.byref(b), C.byref(self.cfg), C.byref(gs),
                                                  _p(dpose), _p(self.ws_bwd), self.ws_bwd.numel(), _stream()),
                   "gs_render_bwd_gaussians")

    def backward_gaussians_adam(self, params: Arena, poses: torch.Tensor, grads: Arena, m: Arena, v: Arena,
                                adam: _lib.GsAdamParamsCfg, dpose: Optional[torch.Tensor]) -> None:
        """gs_render_bwd_gaussians_adam: the per-Gaussian backward with the
        Adam update of the parameters fused in (grads receives the means,
        scale/opacity and rotation gradients only)."""
        ps, gs_, ms, vs = params.rw_struct(), grads.rw_struct(), m.rw_struct(), v.rw_struct()
        b = self.bins_struct()
        _lib.check(self.L.gs_render_bwd_gaussians_adam(C.byref(ps), _p(poses), self.cam_struct, self.views,
                                                       C.byref(self.splats), C.byref(b), C.byref(self.cfg),
                                                       C.byref(gs_), C.byref(ms), C.byref(vs), C.byref(adam),
                                                       _p(dpose), _p(self.ws_bwd), self.ws_bwd.numel(), _stream()),
                   "gs_render_bwd_gaussians_adam")

    # -- splat records as tensors (tests, tools) -------------------------------
    def splat_views(self) -> dict:
        """Device tensor views of the splat arrays, shaped [V, n, ...]."""
        m = self.n * self.views
        sp = self.splats
        base = self.splat_buf.data_ptr()

        def view(ptr, count, dtype, shape):
            off = ptr - base
            nbytes = count * torch.tensor([], dtype=dtype).element_size()
            return self.splat_buf[off:off + nbytes].view(dtype).view(shape)

        V, n = self.views, self.n
        return {"xy": view(sp.xy, 4 * m, torch.float32, (V, n, 4)),
                "conic": view(sp.conic, 4 * m, torch.float32, (V, n, 4)),
                "rgb": view(sp.rgb, 4 * m, torch.float32, (V, n, 4)),
                "depth": view(sp.depth, m, torch.float32, (V, n)),
                "rect": view(sp.rect, 2 * m, torch.int32, (V, n, 2)),
                "touched": view(sp.touched, m, torch.int32, (V, n)),
                "aux": view(sp.aux, m, torch.int32, (V, n))}

    def splat_arrays(self) -> dict:
        """Host copies of the splat arrays (unsigned fields as uint32)."""
        out = {}
        for k, t in self.splat_views().items():
            a = t.cpu().numpy()
            out[k] = a.view(np.uint32) if a.dtype == np.int32 else a
        return out


def adam_step(params: Arena, grads: Arena, m: Arena, v: Arena, step: int, groups, beta1=0.9, beta2=0.999,
              eps=1e-15, status: Optional[torch.Tensor] = None, pose: Optional[torch.Tensor] = None,
              dpose: Optional[torch.Tensor] = None, pose_m: Optional[torch.Tensor] = None,
              pose_v: Optional[torch.Tensor] = None, pose_lr: float = 1e-4, pose_step: int = 0,
              step_dev: Optional[torch.Tensor] = None, pose_steps_dev: Optional[torch.Tensor] = None,
              skip_dev: Optional[torch.Tensor] = None) -> None:
    """Fused Adam over the whole arena (+ optional pose step).  With step_dev
    (a device int32 scalar) the step is read and incremented on the device, so
    the call can be captured in a CUDA graph."""
    L = _lib.load()
    garr = (_lib.GsAdamGroup * max(1, len(groups)))(*groups)  # no group: the pose step alone
    cfg = _lib.GsAdamCfg(garr, len(groups), beta1, beta2, eps, _p(status), _p(pose), _p(dpose), _p(pose_m),
                         _p(pose_v), pose.shape[0] if pose is not None else 0, pose_lr, int(pose_step),
                         _p(step_dev), _p(pose_steps_dev), _p(skip_dev))
    _lib.check(L.gs_adam_step(_p(params.buf), _p(grads.buf), _p(m.buf), _p(v.buf), params.padded, C.byref(cfg),
                              int(step), _stream()), "gs_adam_step")


class ImageLoss:
    """L1 (kind 0) or MSE (kind 1) of images against targets, with dL/dimage."""

    def __init__(self, device="cuda"):
        self.L = _lib.load()
        self.ws = torch.empty(self.L.gs_image_loss_workspace(), dtype=torch.uint8, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def __call__(self, image: torch.Tensor, target: torch.Tensor, grad: Optional[torch.Tensor], kind: int = 0):
        assert image.numel() == target.numel()
        _lib.check(self.L.gs_image_loss(_p(image), _p(target), image.numel(), int(kind), _p(grad), _p(self.loss),
                                        _p(self.ws), self.ws.numel(), _stream()), "gs_image_loss")
        return self.loss
