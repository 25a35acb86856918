"""Python handle of the streaming session (gs_session_* in include/gs.h):
argument marshalling only; batching, admission, the device work and the
latency accounting run in libgs."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib
from .synth import Camera, Scene


def default_config(max_gaussians: int, sh_degree: int = 3, max_batch_views: int = 8, max_width: int = 1920,
                   max_height: int = 1080, max_inflight: int = 2, hbm_budget_gb: float = 80.0,
                   pair_factor: float = 4.0, loss_kind: int = 0, bg=(0.0, 0.0, 0.0), znear: float = 0.2,
                   lr_means=1.6e-4, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3, lr_sh_dc=2.5e-3,
                   lr_sh_rest=1.25e-4, lod: bool = False, lod_tau: float = 1.0,
                   tile=(16, 16)) -> _lib.GsSessionConfig:
    """lod: a progressive hierarchy (merge below lod_tau / 2 px, reload above
    lod_tau px, analysed by Session.analyze); renders draw its render cut
    (descent from the roots), trains each view's cut of the active set.
    tile: 16x16, 32x8 or 8x32."""
    raster = _lib.GsRasterCfg(int(tile[0]), int(tile[1]), (C.c_float * 3)(*bg), float(znear), 1)
    return _lib.GsSessionConfig(int(max_gaussians), int(sh_degree), int(max_batch_views), int(max_width),
                                int(max_height), int(max_inflight), int(hbm_budget_gb * (1 << 30)),
                                float(pair_factor), raster, lr_means, lr_scale, lr_opacity, lr_quat, lr_sh_dc,
                                lr_sh_rest, 0.9, 0.999, 1e-15, int(loss_kind), int(bool(lod)), float(lod_tau))


def plan(cfg: _lib.GsSessionConfig) -> dict:
    L = _lib.load()
    out = _lib.GsSessionPlan()
    st = L.gs_session_plan(C.byref(cfg), C.byref(out))
    return {"status": st, "fixed_bytes": out.fixed_bytes, "context_bytes": out.context_bytes,
            "initial_pair_capacity": out.initial_pair_capacity, "contexts": out.contexts}


def now() -> float:
    return _lib.load().gs_session_now()


class Session:
    def __init__(self, cfg: _lib.GsSessionConfig):
        self.L = _lib.load()
        self.cfg = cfg
        self.nc = (cfg.sh_degree + 1) ** 2
        h = C.c_void_p()
        _lib.check(self.L.gs_session_create(C.byref(cfg), C.byref(h)), "gs_session_create")
        self.h = h
        self._keep = {}  # host buffers referenced by queued requests
        self._borrowed = {}  # pinned targets the session reads until their requests complete

    def close(self):
        if self.h:
            _lib.check(self.L.gs_session_destroy(self.h), "gs_session_destroy")
            self.h = None
            self._keep.clear()
            self._borrowed.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, sc: Scene) -> None:
        if sc.sh_degree != self.cfg.sh_degree:
            raise ValueError(f"scene has SH degree {sc.sh_degree}, the session {self.cfg.sh_degree}")
        if sc.sh.shape != (sc.n, 3, self.nc):
            raise ValueError(f"sh must be [{sc.n}][3][{self.nc}], got {sc.sh.shape}")
        arrs = [np.ascontiguousarray(a, np.float32) for a in
                (sc.means, sc.log_scales, sc.quats, sc.opa_logits, sc.sh)]
        ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs]
        _lib.check(self.L.gs_session_add_gaussians(self.h, sc.n, *ptrs), "gs_session_add_gaussians")

    def submit(self, kind: int, cam: Camera, target=None, want_image: bool = False,
               arrival: float = 0.0, borrow_target: bool = False) -> int:
        """target: [3][H][W] float32, copied during the call; with
        borrow_target a pinned CPU torch tensor that the session reads until
        the request completes (GS_REQUEST_BORROW_TARGET; this object keeps a
        reference until wait() or times() has seen it complete)."""
        req = _lib.GsRequest()
        req.kind = kind
        req.cam = _lib.GsCamera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        req.pose = (C.c_float * 12)(*np.asarray(cam.pose12(), np.float32).tolist())
        tgt = None
        if target is not None and borrow_target:
            import torch
            if not (isinstance(target, torch.Tensor) and target.device.type == "cpu" and target.is_pinned()
                    and target.dtype == torch.float32 and target.is_contiguous()
                    and tuple(target.shape) == (3, cam.height, cam.width)):
                raise ValueError("a borrowed target is a contiguous pinned float32 CPU tensor [3][H][W]")
            tgt = target
            req.target = target.data_ptr()
            req.flags = _lib.GS_REQUEST_BORROW_TARGET
        elif target is not None:
            tgt = np.ascontiguousarray(target, np.float32)
            req.target = tgt.ctypes.data
        img = None
        if want_image:
            img = np.zeros((3, cam.height, cam.width), np.float32)
            req.image_out = img.ctypes.data
        req.arrival_s = float(arrival)
        rid = C.c_int64()
        _lib.check(self.L.gs_session_submit(self.h, C.byref(req), C.byref(rid)), "gs_session_submit")
        self._keep[rid.value] = img
        if borrow_target and tgt is not None:
            self._borrowed[rid.value] = tgt
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 60000) -> Optional[np.ndarray]:
        _lib.check(self.L.gs_session_wait(self.h, rid, timeout_ms), "gs_session_wait")
        self._borrowed.pop(rid, None)
        return self._keep.pop(rid, None)

    def times(self, rid: int) -> Optional[tuple]:
        """(arrival, completion) in gs_session_now seconds, None while pending."""
        a, d = C.c_double(), C.c_double()
        st = self.L.gs_session_times(self.h, rid, C.byref(a), C.byref(d))
        if st == _lib.GS_ERR_BUSY:
            return None
        self._borrowed.pop(rid, None)
        _lib.check(st, "gs_session_times")
        return a.value, d.value

    def image(self, rid: int) -> Optional[np.ndarray]:
        return self._keep.get(rid)

    def set_keyframe(self, kf: int) -> None:
        """Tag the Gaussians added next with keyframe kf (< 0: none)."""
        _lib.check(self.L.gs_session_set_keyframe(self.h, int(kf)), "gs_session_set_keyframe")

    def loop_closure(self, sim3) -> None:
        """Move every tagged Gaussian with its keyframe's correction
        sim3[k] = (qw, qx, qy, qz, tx, ty, tz, s)."""
        s = np.ascontiguousarray(sim3, np.float32).reshape(-1, 8)
        _lib.check(self.L.gs_session_loop_closure(self.h, s.shape[0], s.ctypes.data_as(C.POINTER(C.c_float))),
                   "gs_session_loop_closure")

    def keyframe_weights(self, num_kf: int, min_keep: int = 50, frac: float = 0.05) -> dict:
        """Sampling probabilities of keyframes [0, num_kf) (Sec. 6.2), with the
        leaf counts and the kept mask."""
        p = np.zeros(num_kf, np.float64)
        c = np.zeros(num_kf, np.uint32)
        k = np.zeros(num_kf, np.uint8)
        _lib.check(self.L.gs_session_keyframe_weights(self.h, int(num_kf), int(min_keep), float(frac),
                                                      p.ctypes.data_as(C.POINTER(C.c_double)),
                                                      c.ctypes.data_as(C.POINTER(C.c_uint32)),
                                                      k.ctypes.data_as(C.POINTER(C.c_uint8))),
                   "gs_session_keyframe_weights")
        return {"p": p, "counts": c, "kept": k.astype(bool)}

    def sample_keyframes(self, num_kf: int, m: int, rng: np.random.Generator) -> np.ndarray:
        """m keyframes drawn with the weights of keyframe_weights."""
        p = self.keyframe_weights(num_kf)["p"]
        return rng.choice(num_kf, size=m, p=p)

    def hold(self, on: bool = True) -> None:
        """Pause (or resume) admission: requests submitted while held are
        batched together on resume."""
        _lib.check(self.L.gs_session_hold(self.h, int(bool(on))), "gs_session_hold")

    def drain(self, timeout_ms: int = 120000) -> None:
        _lib.check(self.L.gs_session_drain(self.h, timeout_ms), "gs_session_drain")

    def analyze(self, cam: Camera) -> bool:
        """gs_session_analyze from a new keyframe's camera: the hierarchy's
        merge and reload run into the back buffer of the active set.  Returns
        False when the previous analysis is still running (nothing issued)."""
        c = _lib.GsCamera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        pose = (C.c_float * 12)(*np.asarray(cam.pose12(), np.float32).tolist())
        st = self.L.gs_session_analyze(self.h, C.byref(c), pose)
        if st == _lib.GS_ERR_BUSY:
            return False
        _lib.check(st, "gs_session_analyze")
        return True

    def hierarchy(self) -> dict:
        """gs_session_read_hierarchy: the node rows in use (leaf slots, then
        merged nodes) with their parameters, links and front active flags."""
        rows = C.c_int64(0)
        _lib.check(self.L.gs_session_read_hierarchy(self.h, 0, C.byref(rows), None, None, None, None, None, None,
                                                    None), "gs_session_read_hierarchy")
        n = rows.value
        out = {"means4": np.zeros((n, 4), np.float32), "scale_opa": np.zeros((n, 4), np.float32),
               "quat": np.zeros((n, 4), np.float32), "sh": np.zeros((3 * self.nc, n), np.float32),
               "parent": np.zeros(n, np.int32), "child": np.zeros((n, 4), np.int32),
               "active": np.zeros(n, np.uint8)}
        _lib.check(self.L.gs_session_read_hierarchy(self.h, n, C.byref(rows), *(out[k].ctypes.data for k in (
            "means4", "scale_opa", "quat", "sh", "parent", "child", "active"))), "gs_session_read_hierarchy")
        assert rows.value == n
        return out

    def inject_alloc_failures(self, count: int) -> None:
        """The session's next `count` device allocations fail as if the
        device were out of memory (host-side fault injection, for tests)."""
        _lib.check(self.L.gs_session_inject_alloc_failures(self.h, int(count)), "gs_session_inject_alloc_failures")

    def stats(self) -> dict:
        s = _lib.GsStats()
        _lib.check(self.L.gs_session_stats(self.h, C.byref(s)), "gs_session_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def params(self) -> dict:
        st = self.stats()
        n = st["gaussians"]
        m4 = np.zeros((n, 4), np.float32)
        so = np.zeros((n, 4), np.float32)
        q = np.zeros((n, 4), np.float32)
        sh = np.zeros((3 * self.nc, n), np.float32)
        _lib.check(self.L.gs_session_read_params(self.h, m4.ctypes.data, so.ctypes.data, q.ctypes.data,
                                                 sh.ctypes.data), "gs_session_read_params")
        return {"means4": m4, "scale_opa": so, "quat": q, "sh": sh}

    def save(self, path: str) -> None:
        _lib.check(self.L.gs_session_save(self.h, path.encode()), "gs_session_save")

    def load(self, path: str) -> None:
        _lib.check(self.L.gs_session_load(self.h, path.encode()), "gs_session_load")
