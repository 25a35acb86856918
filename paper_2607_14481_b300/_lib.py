"""ctypes binding of include/gs.h (argument marshalling only).

Loads paper_2607_14481_b300/_build/libgs.so.  A missing or unloadable library
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgs.so")

GS_OK, GS_ERR_INVALID, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_NONFINITE, GS_ERR_BUSY = range(7)
GS_MAX_VIEWS = 64
GS_TILE = 16
GS_SCHED_FWD_LONGEST_FIRST, GS_SCHED_BWD_LONGEST_FIRST, GS_SCHED_FUSED_LONGEST_FIRST = 0x1, 0x2, 0x4
TILE_SHAPES = ((16, 16), (32, 8), (8, 32))


def GS_SCHED_FUSED_BATCH(b: int) -> int:
    return int(b) << 12
GS_MAX_ADAM_GROUPS = 64
GS_BA_MAX_CAMS, GS_BA_MAX_FREE, GS_BA_MAX_OBS = 64, 20, 16
GS_BA_BAD_OBS, GS_BA_SOLVE_FAILED, GS_BA_DEGENERATE = 0x1, 0x2, 0x4

EXPORTED = (
    "gs_last_error", "gs_version", "gs_built_arch", "gs_splats_bytes", "gs_splats_carve",
    "gs_project", "gs_bin_sort_workspace", "gs_bin_sort", "gs_bin_sort_noalloc", "gs_render_fwd",
    "gs_render_bwd_workspace", "gs_render_bwd", "gs_render_bwd_pixels", "gs_render_bwd_gaussians",
    "gs_render_bwd_gaussians_adam",
    "gs_adam_step", "gs_image_loss_workspace", "gs_image_loss", "gs_render_stats",
    "gs_lod_nodes", "gs_lod_build_workspace", "gs_lod_build", "gs_project_lod", "gs_sim3_update", "gs_keyframe_counts", "gs_autotune_blend",
    "gs_render_fused_workspace", "gs_render_fused", "gs_autotune_fused",
    "gs_hier_workspace", "gs_hier_analyze", "gs_hier_refine", "gs_project_hier", "gs_project_hier_render",
    "gs_ba_workspace_bytes", "gs_ba_solve",
    "gs_session_now", "gs_session_plan", "gs_session_create", "gs_session_add_gaussians", "gs_session_submit",
    "gs_session_poll", "gs_session_wait", "gs_session_drain", "gs_session_hold", "gs_session_times", "gs_session_set_keyframe", "gs_session_loop_closure", "gs_session_keyframe_weights", "gs_session_stats", "gs_session_read_params",
    "gs_session_save", "gs_session_load", "gs_session_inject_alloc_failures", "gs_session_analyze",
    "gs_session_read_hierarchy", "gs_session_destroy",
)

GS_REQUEST_RENDER, GS_REQUEST_TRAIN = 0, 1


class GsError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what} failed with status {status}: {msg}")
        self.status = status


class GsParams(C.Structure):
    _fields_ = [("means4", C.c_void_p), ("scale_opa", C.c_void_p), ("quat", C.c_void_p),
                ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32), ("sh_stride", C.c_int64)]


GsGrads = GsParams  # same layout (non-const pointers)


class GsCamera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class GsRasterCfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("bg", C.c_float * 3),
                ("znear", C.c_float), ("clamp_jacobian", C.c_int32), ("schedule", C.c_uint32)]


class GsSplats(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("conic", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
                ("rect", C.c_void_p), ("touched", C.c_void_p), ("aux", C.c_void_p),
                ("n", C.c_int64), ("views", C.c_int32)]


class GsBins(C.Structure):
    _fields_ = [("vals", C.c_void_p), ("ranges", C.c_void_p), ("pair_off", C.c_void_p),
                ("keys", C.c_void_p), ("counts", C.c_void_p), ("capacity", C.c_int64),
                ("num_tiles", C.c_int64), ("tile_order", C.c_void_p)]


class GsHier(C.Structure):
    _fields_ = [("parent", C.c_void_p), ("child", C.c_void_p), ("active", C.c_void_p), ("n_nodes", C.c_void_p),
                ("info", C.c_void_p), ("capacity", C.c_int64)]


class GsAdamGroup(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64), ("lr", C.c_float * 4)]


class GsAdamCfg(C.Structure):
    _fields_ = [("groups", C.POINTER(GsAdamGroup)), ("num_groups", C.c_int32), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("status", C.c_void_p), ("pose", C.c_void_p),
                ("dpose", C.c_void_p), ("pose_m", C.c_void_p), ("pose_v", C.c_void_p),
                ("views", C.c_int32), ("pose_lr", C.c_float), ("pose_step", C.c_int32),
                ("step_dev", C.c_void_p), ("pose_steps_dev", C.c_void_p), ("skip_dev", C.c_void_p)]


class GsAdamParamsCfg(C.Structure):
    _fields_ = [("lr_means4", C.c_float * 4), ("lr_scale_opa", C.c_float * 4), ("lr_quat", C.c_float * 4),
                ("lr_sh", C.c_float * 48), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("update_mask", C.c_uint32), ("step_dev", C.c_void_p),
                ("skip_dev", C.c_void_p), ("status", C.c_void_p)]


class GsBaProblem(C.Structure):
    _fields_ = [("num_cams", C.c_int32), ("num_points", C.c_int32), ("obs_per_point", C.c_int32),
                ("opt_focal", C.c_int32), ("cx", C.c_float), ("cy", C.c_float), ("obs_cam", C.c_void_p),
                ("obs_uv", C.c_void_p), ("fixed", C.c_uint8 * GS_BA_MAX_CAMS)]


class GsSessionConfig(C.Structure):
    _fields_ = [("max_gaussians", C.c_int64), ("sh_degree", C.c_int32), ("max_batch_views", C.c_int32),
                ("max_width", C.c_int32), ("max_height", C.c_int32), ("max_inflight", C.c_int32),
                ("hbm_budget_bytes", C.c_uint64), ("pair_factor", C.c_double), ("raster", GsRasterCfg),
                ("lr_means", C.c_float), ("lr_scale", C.c_float), ("lr_opacity", C.c_float),
                ("lr_quat", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("loss_kind", C.c_int32),
                ("lod", C.c_int32), ("lod_tau", C.c_float)]


GS_REQUEST_BORROW_TARGET = 1


class GsRequest(C.Structure):
    _fields_ = [("kind", C.c_int32), ("cam", GsCamera), ("pose", C.c_float * 12), ("target", C.c_void_p),
                ("image_out", C.c_void_p), ("arrival_s", C.c_double), ("flags", C.c_int32)]


class GsStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64),
                ("inflight", C.c_int64), ("iterations", C.c_int64), ("batches", C.c_int64), ("retries", C.c_int64),
                ("lod_builds", C.c_int64),
                ("gaussians", C.c_int64), ("pixels", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mean_ms", C.c_double), ("max_ms", C.c_double), ("wall_s", C.c_double),
                ("hbm_in_use", C.c_uint64), ("hbm_budget", C.c_uint64), ("contexts", C.c_int32),
                ("train_beside_render", C.c_int64)]


class GsSessionPlan(C.Structure):
    _fields_ = [("fixed_bytes", C.c_size_t), ("context_bytes", C.c_size_t), ("initial_pair_capacity", C.c_int64),
                ("contexts", C.c_int32)]


_lib = None


def noalloc_scratch_bytes() -> int:
    """Bytes of gs_bin_sort_noalloc's static scratch, read from the library's
    data symbol gs_noalloc_scratch_bytes."""
    return int(C.c_uint64.in_dll(load(), "gs_noalloc_scratch_bytes").value)


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libgs.so; raises if it is absent or lacks a declared symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgs.so not found at {path}: build it with paper_2607_14481_b300/build.py")
    L = C.CDLL(path)
    for name in EXPORTED:
        if not hasattr(L, name):
            raise RuntimeError(f"libgs.so lacks symbol {name}")
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    P = C.POINTER
    L.gs_last_error.argtypes = [C.c_char_p, sz]
    L.gs_last_error.restype = sz
    L.gs_version.restype = i32
    L.gs_built_arch.restype = i32
    L.gs_splats_bytes.argtypes = [i64, i32]
    L.gs_splats_bytes.restype = sz
    L.gs_splats_carve.argtypes = [vp, i64, i32, P(GsSplats)]
    L.gs_project.argtypes = [P(GsParams), vp, P(GsCamera), i32, P(GsRasterCfg), P(GsSplats), vp]
    L.gs_bin_sort_workspace.argtypes = [i64, i32, i64]
    L.gs_bin_sort_workspace.restype = sz
    L.gs_bin_sort.argtypes = [P(GsSplats), P(GsCamera), i32, P(GsRasterCfg), P(GsBins), vp, sz, vp]
    L.gs_bin_sort_noalloc.argtypes = [P(GsSplats), P(GsCamera), i32, P(GsRasterCfg), P(GsBins), vp]
    L.gs_render_fwd.argtypes = [P(GsSplats), P(GsBins), P(GsCamera), i32, P(GsRasterCfg), vp, vp, vp]
    L.gs_render_bwd_workspace.argtypes = [i64, i32, i64]
    L.gs_render_bwd_workspace.restype = sz
    L.gs_render_bwd.argtypes = [P(GsParams), vp, P(GsCamera), i32, P(GsSplats), P(GsBins),
                                P(GsRasterCfg), vp, vp, vp, P(GsGrads), vp, vp, sz, vp]
    L.gs_render_bwd_pixels.argtypes = [P(GsSplats), P(GsBins), P(GsCamera), i32, P(GsRasterCfg), vp, vp, vp,
                                       i64, vp, sz, vp]
    L.gs_render_bwd_gaussians_adam.argtypes = [P(GsGrads), vp, P(GsCamera), i32, P(GsSplats), P(GsBins),
                                               P(GsRasterCfg), P(GsGrads), P(GsGrads), P(GsGrads),
                                               P(GsAdamParamsCfg), vp, vp, sz, vp]
    L.gs_render_bwd_gaussians.argtypes = [P(GsParams), vp, P(GsCamera), i32, P(GsSplats), P(GsBins),
                                          P(GsRasterCfg), P(GsGrads), vp, vp, sz, vp]
    L.gs_adam_step.argtypes = [vp, vp, vp, vp, i64, P(GsAdamCfg), i32, vp]
    L.gs_autotune_blend.argtypes = [P(GsSplats), P(GsBins), P(GsCamera), i32, P(GsRasterCfg), vp, vp, i64, vp, sz,
                                    i32, C.POINTER(C.c_float), vp]
    L.gs_render_fused_workspace.argtypes = [i64, i32, i64, i64]
    L.gs_render_fused_workspace.restype = sz
    L.gs_render_fused.argtypes = [P(GsSplats), P(GsBins), P(GsCamera), i32, P(GsRasterCfg), vp, i32, vp, vp, vp,
                                  i64, vp, sz, vp]
    L.gs_autotune_fused.argtypes = [P(GsParams), vp, P(GsCamera), i32, P(GsRasterCfg), P(GsSplats), P(GsBins), i64,
                                    vp, sz, vp, i32, vp, vp, vp, sz, i32, C.POINTER(C.c_float), vp]
    L.gs_hier_workspace.argtypes = [i64]
    L.gs_hier_workspace.restype = sz
    L.gs_hier_analyze.argtypes = [P(GsGrads), P(GsHier), P(GsGrads), P(GsGrads), vp, P(GsCamera), C.c_float,
                                  C.c_float, vp, sz, vp]
    L.gs_hier_refine.argtypes = [P(GsGrads), P(GsHier), P(GsGrads), P(GsGrads), vp, P(GsCamera), C.c_float,
                                 C.c_float, i32, vp, sz, vp]
    L.gs_project_hier.argtypes = [P(GsParams), P(GsHier), C.c_float, vp, P(GsCamera), i32, P(GsRasterCfg),
                                  P(GsSplats), vp]
    L.gs_project_hier_render.argtypes = [P(GsParams), P(GsHier), C.c_float, vp, P(GsCamera), i32,
                                         P(GsRasterCfg), P(GsSplats), vp]
    L.gs_sim3_update.argtypes = [P(GsGrads), vp, vp, i32, vp, vp]
    L.gs_keyframe_counts.argtypes = [vp, i64, i32, vp, vp]
    L.gs_lod_nodes.argtypes = [i64]
    L.gs_lod_nodes.restype = i64
    L.gs_lod_build_workspace.argtypes = [i64]
    L.gs_lod_build_workspace.restype = sz
    L.gs_lod_build.argtypes = [P(GsGrads), i64, vp, vp, sz, vp]
    L.gs_project_lod.argtypes = [P(GsParams), i64, vp, C.c_float, vp, P(GsCamera), i32, P(GsRasterCfg), P(GsSplats),
                                 vp]
    L.gs_ba_workspace_bytes.argtypes = [i32, i32, i32]
    L.gs_ba_workspace_bytes.restype = sz
    L.gs_ba_solve.argtypes = [P(GsBaProblem), vp, vp, vp, i32, C.c_double, vp, vp, vp, sz, vp]
    L.gs_render_stats.argtypes = [P(GsSplats), P(GsBins), P(GsCamera), i32, P(GsRasterCfg), vp, vp]
    L.gs_image_loss_workspace.argtypes = []
    L.gs_image_loss_workspace.restype = sz
    L.gs_image_loss.argtypes = [vp, vp, i64, i32, vp, vp, vp, sz, vp]
    L.gs_session_now.restype = C.c_double
    L.gs_session_plan.argtypes = [P(GsSessionConfig), P(GsSessionPlan)]
    L.gs_session_create.argtypes = [P(GsSessionConfig), P(vp)]
    L.gs_session_add_gaussians.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.gs_session_submit.argtypes = [vp, P(GsRequest), P(i64)]
    L.gs_session_poll.argtypes = [vp, i64, P(i32)]
    L.gs_session_wait.argtypes = [vp, i64, i32]
    L.gs_session_drain.argtypes = [vp, i32]
    L.gs_session_hold.argtypes = [vp, i32]
    L.gs_session_set_keyframe.argtypes = [vp, i32]
    L.gs_session_loop_closure.argtypes = [vp, i32, C.POINTER(C.c_float)]
    L.gs_session_keyframe_weights.argtypes = [vp, i32, i32, C.c_float, C.POINTER(C.c_double),
                                              C.POINTER(C.c_uint32), C.POINTER(C.c_uint8)]
    L.gs_session_times.argtypes = [vp, i64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.gs_session_stats.argtypes = [vp, P(GsStats)]
    L.gs_session_read_params.argtypes = [vp, vp, vp, vp, vp]
    L.gs_session_save.argtypes = [vp, C.c_char_p]
    L.gs_session_load.argtypes = [vp, C.c_char_p]
    L.gs_session_inject_alloc_failures.argtypes = [vp, i32]
    L.gs_session_analyze.argtypes = [vp, P(GsCamera), C.POINTER(C.c_float)]
    L.gs_session_read_hierarchy.argtypes = [vp, C.c_int64, C.POINTER(C.c_int64), vp, vp, vp, vp, vp, vp, vp]
    L.gs_session_destroy.argtypes = [vp]
    for name in ("gs_session_plan", "gs_session_create", "gs_session_add_gaussians", "gs_session_submit",
                 "gs_session_poll", "gs_session_wait", "gs_session_drain", "gs_session_hold", "gs_session_times", "gs_session_set_keyframe", "gs_session_loop_closure", "gs_session_keyframe_weights", "gs_session_stats",
                 "gs_session_read_params", "gs_session_save", "gs_session_load", "gs_session_inject_alloc_failures",
                 "gs_session_analyze", "gs_session_read_hierarchy", "gs_session_destroy"):
        getattr(L, name).restype = C.c_int
    for name in ("gs_splats_carve", "gs_project", "gs_bin_sort", "gs_bin_sort_noalloc", "gs_render_fwd",
                 "gs_render_bwd",
                 "gs_render_bwd_pixels", "gs_render_bwd_gaussians", "gs_render_bwd_gaussians_adam", "gs_adam_step",
                 "gs_image_loss",
                 "gs_render_stats", "gs_lod_build", "gs_project_lod", "gs_sim3_update", "gs_keyframe_counts", "gs_autotune_blend",
                 "gs_ba_solve", "gs_render_fused", "gs_autotune_fused", "gs_hier_analyze", "gs_hier_refine",
                 "gs_project_hier", "gs_project_hier_render"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def last_error() -> str:
    L = load()
    buf = C.create_string_buffer(1024)
    L.gs_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int, what: str) -> None:
    if status != GS_OK:
        raise GsError(status, what, last_error())
