"""The C-ABI library builds, loads and exports every entry point include/gs.h
declares; host-side argument checks reject bad calls before any device work
(no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_2607_14481_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "gs.h")).read()
    return sorted(set(re.findall(r"GS_API\s+[\w\s\*]+?\b(gs_\w+)\s*\(", text)))


def test_header_declarations_match_binding_list():
    assert set(_declared()) == set(_lib.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_noalloc_scratch_size_is_exported(lib):
    # the binding reads the scratch size from the library's data symbol
    text = open(os.path.join(ROOT, "include", "gs.h")).read()
    m = re.search(r"#define GS_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    assert m and _lib.noalloc_scratch_bytes() == int(m.group(1)) << int(m.group(2))


def test_version_and_arch(lib):
    assert lib.gs_version() == 1
    assert lib.gs_built_arch() == 1030


def test_size_queries(lib):
    a = lib.gs_splats_bytes(1000, 2)
    b = lib.gs_splats_bytes(2000, 2)
    assert 0 < a < b
    # 3 float4 + depth + rect + touched + aux = 64 B per (view, Gaussian) + alignment
    assert b >= 64 * 2000 * 2
    assert lib.gs_bin_sort_workspace(1000, 1, 10_000) > lib.gs_bin_sort_workspace(1000, 1, 1000)
    assert lib.gs_render_bwd_workspace(1000, 1, 10_000) >= 36 * 10_000


def test_lod_sizes_and_validation(lib):
    assert lib.gs_lod_nodes(0) == 0 and lib.gs_lod_nodes(1) == 3 and lib.gs_lod_nodes(8) == 10
    assert lib.gs_lod_nodes(9) == 9 + 2 + 1 and lib.gs_lod_nodes(65) == 65 + 9 + 2
    assert lib.gs_lod_build_workspace(1000) > lib.gs_lod_build_workspace(10)
    nodes = _lib.GsGrads(256, 256, 256, 256, 10, 0, 0)  # 10 rows cannot hold 9 leaves + 3 coarse nodes
    st = lib.gs_lod_build(C.byref(nodes), 9, C.c_void_p(256), C.c_void_p(256), 1 << 20, None)
    assert st == _lib.GS_ERR_INVALID and "needs 12" in _lib.last_error()


def test_unknown_schedule_rejected_on_host(lib):
    cam = (_lib.GsCamera * 1)(_lib.GsCamera(100.0, 100.0, 32.0, 32.0, 64, 64))
    sp = _lib.GsSplats(256, 256, 256, 256, 256, 256, 256, 10, 1)
    bins = _lib.GsBins(16, 16, 16, None, 16, 100, 16)
    for sched in (3 << 4, 2 << 8, 3 << 12, 1 << 16):
        cfg = _lib.GsRasterCfg(16, 16, (C.c_float * 3)(0, 0, 0), 0.2, 1, sched)
        st = lib.gs_render_fwd(C.byref(sp), C.byref(bins), cam, 1, C.byref(cfg), C.c_void_p(256), None, None)
        assert st == _lib.GS_ERR_INVALID and "schedule" in _lib.last_error()


def test_invalid_arguments_rejected_on_host(lib):
    cam = (_lib.GsCamera * 1)(_lib.GsCamera(100.0, 100.0, 32.0, 32.0, 64, 64))
    cfg = _lib.GsRasterCfg(16, 16, (C.c_float * 3)(0, 0, 0), 0.2, 1)
    sp = _lib.GsSplats()
    st = lib.gs_project(None, None, cam, 1, C.byref(cfg), C.byref(sp), None)
    assert st == _lib.GS_ERR_INVALID
    assert "params" in _lib.last_error()
    params = _lib.GsParams(None, None, None, None, 0, 5, 0)
    st = lib.gs_project(C.byref(params), None, cam, 1, C.byref(cfg), C.byref(sp), None)
    assert st == _lib.GS_ERR_INVALID and "sh_degree" in _lib.last_error()
    bad = _lib.GsRasterCfg(8, 8, (C.c_float * 3)(0, 0, 0), 0.2, 1)  # 64-pixel tiles are not supported
    params = _lib.GsParams(None, None, None, None, 0, 0, 0)
    st = lib.gs_project(C.byref(params), None, cam, 1, C.byref(bad), C.byref(sp), None)
    assert st == _lib.GS_ERR_INVALID and "tile" in _lib.last_error()
    st = lib.gs_project(C.byref(params), None, cam, 0, C.byref(cfg), C.byref(sp), None)
    assert st == _lib.GS_ERR_INVALID
    grp = (_lib.GsAdamGroup * 1)(_lib.GsAdamGroup(0, 4, (C.c_float * 4)(1, 1, 1, 1)))
    acfg = _lib.GsAdamCfg(grp, 1, 0.9, 0.999, 1e-15, None, None, None, None, None, 0, 0.0, 0, None, None, None)
    st = lib.gs_adam_step(None, None, None, None, 0, C.byref(acfg), 0, None)
    assert st == _lib.GS_ERR_INVALID and "step" in _lib.last_error()
    st = lib.gs_adam_step(None, None, None, None, 4, C.byref(acfg), 1, None)
    assert st == _lib.GS_ERR_INVALID
    # a workspace that is too small is reported as GS_ERR_OOM before any launch
    bins = _lib.GsBins(16, 16, 16, None, 16, 100, 16)
    sp = _lib.GsSplats(256, 256, 256, 256, 256, 256, 256, 10, 1)
    st = lib.gs_bin_sort(C.byref(sp), cam, 1, C.byref(cfg), C.byref(bins), C.c_void_p(256), 16, None)
    assert st == _lib.GS_ERR_OOM and "workspace" in _lib.last_error()


def test_session_plan_admits_by_budget(lib):
    from paper_2607_14481_b300 import session
    small = session.default_config(1_000_000, max_batch_views=8, hbm_budget_gb=0.5)
    p = session.plan(small)
    assert p["status"] == _lib.GS_ERR_OOM and p["contexts"] == 0
    assert "budget" in _lib.last_error()
    mid = session.default_config(1_000_000, max_batch_views=8, max_inflight=4, hbm_budget_gb=80.0)
    q = session.plan(mid)
    assert q["status"] == _lib.GS_OK and 1 <= q["contexts"] <= 4
    # the arenas: parameters, gradients and two moments of (12 + 48) floats per Gaussian
    assert q["fixed_bytes"] >= 4 * 60 * 4 * 1_000_000
    need = q["fixed_bytes"] + 2 * q["context_bytes"]
    two = session.default_config(1_000_000, max_batch_views=8, max_inflight=4, hbm_budget_gb=need / (1 << 30))
    assert session.plan(two)["contexts"] == 2


def test_bundle_adjustment_validation(lib):
    """gs_ba_solve rejects bad problems on the host, before any device work."""
    assert lib.gs_ba_workspace_bytes(20, 10000, 8) > 0
    assert lib.gs_ba_workspace_bytes(0, 10, 8) == 0
    assert lib.gs_ba_workspace_bytes(65, 10, 8) == 0
    assert lib.gs_ba_workspace_bytes(20, 10, 17) == 0
    fake = C.c_void_p(256)  # never dereferenced: every call below fails its checks first
    trace = C.c_void_p(0)

    def call(prob, iters=10, lam=1e-3, ws_bytes=1 << 30, poses=fake):
        return lib.gs_ba_solve(C.byref(prob), poses, fake, fake, iters, lam, trace, fake, fake, ws_bytes,
                               C.c_void_p(0))

    prob = _lib.GsBaProblem()
    prob.num_cams, prob.num_points, prob.obs_per_point, prob.opt_focal = 24, 100, 8, 1
    prob.obs_cam, prob.obs_uv = 256, 256
    for k in range(3):
        prob.fixed[k] = 1
    assert call(prob) == _lib.GS_ERR_INVALID          # 21 free keyframes
    assert "free keyframes" in _lib.last_error()
    prob.fixed[3] = 1
    assert call(prob, lam=0.0) == _lib.GS_ERR_INVALID
    assert call(prob, lam=float("nan")) == _lib.GS_ERR_INVALID
    assert call(prob, iters=-1) == _lib.GS_ERR_INVALID
    assert call(prob, poses=C.c_void_p(0)) == _lib.GS_ERR_INVALID
    assert call(prob, ws_bytes=16) == _lib.GS_ERR_OOM
    prob.obs_per_point = 0
    assert call(prob) == _lib.GS_ERR_INVALID
