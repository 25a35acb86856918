// C entry points of include/gs.h: argument validation, workspace carving,
// error reporting.  No entry point allocates device memory or synchronises.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "gs_internal.h"

namespace gs {

static thread_local std::string t_last_error;

gs_status fail(gs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

gs_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return GS_OK;
}

bool make_view_table(const gs_camera* cams, int views, ViewTable* vt, int tw, int th) {
  if (!cams || views <= 0 || views > GS_MAX_VIEWS) {
    fail(GS_ERR_INVALID, "views must be in [1, %d] with a camera array", GS_MAX_VIEWS);
    return false;
  }
  if (!tile_shape_ok(tw, th)) {
    fail(GS_ERR_INVALID, "unsupported tile shape %dx%d (16x16, 32x8 or 8x32)", tw, th);
    return false;
  }
  std::memset(vt, 0, sizeof(*vt));
  vt->views = views;
  vt->tw = tw;
  vt->th = th;
  int64_t tiles = 0, pix = 0;
  for (int v = 0; v < views; ++v) {
    const gs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 16 * 4096 || c.height > 16 * 4096 ||
        !(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy)) {
      fail(GS_ERR_INVALID, "camera %d: bad intrinsics or size", v);
      return false;
    }
    ViewInfo& vi = vt->v[v];
    vi.fx = c.fx; vi.fy = c.fy; vi.cx = c.cx; vi.cy = c.cy;
    vi.W = c.width; vi.H = c.height;
    vi.TX = (c.width + tw - 1) / tw;
    vi.TY = (c.height + th - 1) / th;
    vi.tile_base = (int32_t)tiles;
    vi.pix_base = pix;
    tiles += (int64_t)vi.TX * vi.TY;
    pix += (int64_t)c.width * c.height;
  }
  if (tiles >= (1ll << 30)) {
    fail(GS_ERR_INVALID, "too many tiles (%lld)", (long long)tiles);
    return false;
  }
  vt->total_tiles = (int32_t)tiles;
  return true;
}

size_t bin_sort_workspace_bytes(int64_t m, int64_t cap);
gs_status launch_bin_sort(const gs_splats& sp, const ViewTable& vt, const gs_bins& bins, void* ws,
                          cudaStream_t s);

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static gs_status check_cfg(const gs_raster_cfg* cfg) {
  if (!cfg) return fail(GS_ERR_INVALID, "cfg is NULL");
  if (!tile_shape_ok(cfg->tile_w, cfg->tile_h))
    return fail(GS_ERR_INVALID, "tile must be 16x16, 32x8 or 8x32 (got %dx%d)", cfg->tile_w, cfg->tile_h);
  if (!(cfg->znear > 0.f)) return fail(GS_ERR_INVALID, "znear must be > 0");
  if ((cfg->schedule & ~kSchedKnown) || ((cfg->schedule >> kSchedFwdBatchShift) & 3u) == 3u ||
      ((cfg->schedule >> kSchedFusedBatchShift) & 3u) == 3u ||
      ((cfg->schedule >> kSchedBwdBatchShift) & 3u) > 1u)
    return fail(GS_ERR_INVALID, "unknown schedule 0x%x", cfg->schedule);

  return GS_OK;
}

static gs_status check_params(const gs_params* p) {
  if (!p) return fail(GS_ERR_INVALID, "params is NULL");
  if (p->n < 0 || p->n >= (1ll << 31)) return fail(GS_ERR_INVALID, "n out of range");
  if (p->sh_stride != 0 && p->sh_stride < p->n) return fail(GS_ERR_INVALID, "sh_stride must be 0 or >= n");
  if (p->sh_degree < 0 || p->sh_degree > 3) return fail(GS_ERR_INVALID, "sh_degree must be 0..3");
  if (p->n > 0 && (!p->means4 || !p->scale_opa || !p->quat || !p->sh))
    return fail(GS_ERR_INVALID, "NULL parameter array");
  if (!aligned(p->means4, 16) || !aligned(p->scale_opa, 16) || !aligned(p->quat, 16))
    return fail(GS_ERR_INVALID, "parameter arrays must be 16-byte aligned");
  return GS_OK;
}

static gs_status check_splats(const gs_splats* sp, int64_t n, int views) {
  if (!sp) return fail(GS_ERR_INVALID, "splats is NULL");
  if (sp->n != n || sp->views != views) return fail(GS_ERR_INVALID, "splats sized for another n/views");
  if (n > 0 && (!sp->xy || !sp->conic || !sp->rgb || !sp->depth || !sp->rect || !sp->touched || !sp->aux))
    return fail(GS_ERR_INVALID, "NULL splat array");
  if (!aligned(sp->xy, 16) || !aligned(sp->conic, 16) || !aligned(sp->rgb, 16) || !aligned(sp->rect, 8))
    return fail(GS_ERR_INVALID, "splat arrays misaligned");
  if ((uint64_t)n * (uint64_t)views >= (1ull << 32))
    return fail(GS_ERR_INVALID, "n * views must be < 2^32");
  return GS_OK;
}

static gs_status check_bins(const gs_bins* b, const ViewTable& vt, int64_t n) {
  if (!b) return fail(GS_ERR_INVALID, "bins is NULL");
  if (!b->vals || !b->ranges || !b->pair_off || !b->counts) return fail(GS_ERR_INVALID, "NULL bins array");
  if (b->capacity < 0 || b->capacity >= (1ll << 32) - 1) return fail(GS_ERR_INVALID, "capacity out of range");
  if (vt.total_tiles > bin_sort_max_tiles())
    return fail(GS_ERR_INVALID, "%d tiles exceed the binning limit of %lld", vt.total_tiles,
                (long long)bin_sort_max_tiles());
  if (b->num_tiles != vt.total_tiles)
    return fail(GS_ERR_INVALID, "bins.num_tiles (%lld) != tiles of the views (%d)", (long long)b->num_tiles,
                vt.total_tiles);
  (void)n;
  return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_last_error(char* buf, size_t len) {
  const std::string& e = t_last_error;
  if (buf && len > 0) {
    size_t k = std::min(len - 1, e.size());
    std::memcpy(buf, e.data(), k);
    buf[k] = '\0';
  }
  return e.size();
}

int32_t gs_version(void) { return 1; }

int32_t gs_built_arch(void) {
#ifdef GS_BUILT_ARCH
  return GS_BUILT_ARCH;
#else
  return 0;
#endif
}

static size_t splat_layout(int64_t n, int32_t views, char* base, gs_splats* out) {
  const size_t m = (size_t)std::max<int64_t>(0, n) * (size_t)std::max(0, views);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1), 256);
    return p;
  };
  float* xy = (float*)take(16 * m);
  float* conic = (float*)take(16 * m);
  float* rgb = (float*)take(16 * m);
  float* depth = (float*)take(4 * m);
  uint32_t* rect = (uint32_t*)take(8 * m);
  uint32_t* touched = (uint32_t*)take(4 * m);
  uint32_t* aux = (uint32_t*)take(4 * m);
  if (out) {
    out->xy = xy; out->conic = conic; out->rgb = rgb; out->depth = depth;
    out->rect = rect; out->touched = touched; out->aux = aux;
    out->n = n; out->views = views;
  }
  return off;
}

size_t gs_splats_bytes(int64_t n, int32_t views) { return splat_layout(n, views, nullptr, nullptr); }

gs_status gs_splats_carve(void* base, int64_t n, int32_t views, gs_splats* out) {
  GS_NVTX("gs_splats_carve");
  if (!base || !out) return fail(GS_ERR_INVALID, "NULL base or out");
  if (n < 0 || views <= 0 || views > GS_MAX_VIEWS) return fail(GS_ERR_INVALID, "bad n or views");
  if (reinterpret_cast<uintptr_t>(base) % 256) return fail(GS_ERR_INVALID, "base must be 256-byte aligned");
  splat_layout(n, views, static_cast<char*>(base), out);
  return GS_OK;
}

gs_status gs_project(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                     int32_t views, const gs_raster_cfg* cfg, gs_splats* out, gs_stream stream) {
  GS_NVTX("gs_project");
  gs_status st;
  if ((st = check_params(params)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if ((st = check_splats(out, params->n, views)) != GS_OK) return st;
  return launch_project(*params, poses_dev, vt, *cfg, *out, (cudaStream_t)stream);
}

gs_status gs_sim3_update(gs_grads* params, const int32_t* kf_dev, const float* sim3_dev, int32_t num_kf,
                         uint32_t* status_dev, gs_stream stream) {
  GS_NVTX("gs_sim3_update");
  if (!params) return fail(GS_ERR_INVALID, "params is NULL");
  gs_params view{params->means4, params->scale_opa, params->quat, params->sh, params->n, params->sh_degree,
                 params->sh_stride};
  gs_status st;
  if ((st = check_params(&view)) != GS_OK) return st;
  if (num_kf < 0) return fail(GS_ERR_INVALID, "num_kf < 0");
  if (params->n > 0 && (!kf_dev || !status_dev || (num_kf > 0 && !sim3_dev)))
    return fail(GS_ERR_INVALID, "NULL keyframe ids, corrections or status");
  return launch_sim3_update(*params, kf_dev, sim3_dev, num_kf, status_dev, (cudaStream_t)stream);
}

gs_status gs_keyframe_counts(const int32_t* kf_dev, int64_t n, int32_t num_kf, uint32_t* counts_dev,
                             gs_stream stream) {
  GS_NVTX("gs_keyframe_counts");
  if (n < 0 || num_kf < 0) return fail(GS_ERR_INVALID, "n or num_kf < 0");
  if ((n > 0 && !kf_dev) || (num_kf > 0 && !counts_dev)) return fail(GS_ERR_INVALID, "NULL array");
  return launch_keyframe_counts(kf_dev, n, num_kf, counts_dev, (cudaStream_t)stream);
}

static bool ba_sizes_ok(int32_t num_cams, int32_t num_points, int32_t obs_per_point) {
  return num_cams >= 1 && num_cams <= GS_BA_MAX_CAMS && num_points >= 0 && num_points < (1 << 23) &&
         obs_per_point >= 1 && obs_per_point <= GS_BA_MAX_OBS;
}

size_t gs_ba_workspace_bytes(int32_t num_cams, int32_t num_points, int32_t obs_per_point) {
  if (!ba_sizes_ok(num_cams, num_points, obs_per_point)) return 0;
  return ba_workspace_bytes(num_cams, num_points, obs_per_point);
}

gs_status gs_ba_solve(const gs_ba_problem* prob, float* poses, float* points, float* focal, int32_t iters,
                      double lambda0, double* trace, uint32_t* status, void* ws, size_t ws_bytes,
                      gs_stream stream) {
  GS_NVTX("gs_ba_solve");
  if (!prob) return fail(GS_ERR_INVALID, "problem is NULL");
  if (!ba_sizes_ok(prob->num_cams, prob->num_points, prob->obs_per_point))
    return fail(GS_ERR_INVALID, "num_cams must be 1..%d, num_points 0..2^23-1, obs_per_point 1..%d",
                GS_BA_MAX_CAMS, GS_BA_MAX_OBS);
  int n_free = 0;
  for (int k = 0; k < prob->num_cams; ++k) n_free += prob->fixed[k] ? 0 : 1;
  if (n_free > GS_BA_MAX_FREE) return fail(GS_ERR_INVALID, "%d free keyframes (at most %d)", n_free, GS_BA_MAX_FREE);
  if (iters < 0) return fail(GS_ERR_INVALID, "iters < 0");
  if (!(lambda0 > 0.0) || !std::isfinite(lambda0)) return fail(GS_ERR_INVALID, "lambda0 must be finite and > 0");
  if (!poses || !focal || !status || !ws) return fail(GS_ERR_INVALID, "NULL poses, focal, status or workspace");
  if (prob->num_points > 0 && (!points || !prob->obs_cam || !prob->obs_uv))
    return fail(GS_ERR_INVALID, "NULL points or observations");
  if ((reinterpret_cast<uintptr_t>(prob->obs_uv) & 7) || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(GS_ERR_INVALID, "obs_uv must be 8-byte and ws 256-byte aligned");
  const size_t need = ba_workspace_bytes(prob->num_cams, prob->num_points, prob->obs_per_point);
  if (ws_bytes < need) return fail(GS_ERR_OOM, "workspace %zu bytes, need %zu", ws_bytes, need);
  if (iters == 0) return GS_OK;
  return launch_ba(*prob, poses, points, focal, iters, lambda0, trace, status, ws, (cudaStream_t)stream);
}

int64_t gs_lod_nodes(int64_t n_leaf) {
  return n_leaf <= 0 ? 0 : n_leaf + lod_level1(n_leaf) + lod_level2(n_leaf);
}

size_t gs_lod_build_workspace(int64_t n_leaf) { return lod_build_workspace_bytes(std::max<int64_t>(0, n_leaf)); }

gs_status gs_lod_build(gs_grads* nodes, int64_t n_leaf, int32_t* parent_dev, void* ws, size_t ws_bytes,
                       gs_stream stream) {
  GS_NVTX("gs_lod_build");
  if (!nodes) return fail(GS_ERR_INVALID, "nodes is NULL");
  gs_params view{nodes->means4, nodes->scale_opa, nodes->quat, nodes->sh, nodes->n, nodes->sh_degree,
                 nodes->sh_stride};
  gs_status st;
  if ((st = check_params(&view)) != GS_OK) return st;
  if (n_leaf < 0 || n_leaf > (1ll << 30)) return fail(GS_ERR_INVALID, "n_leaf out of range");
  if (gs_lod_nodes(n_leaf) > nodes->n)
    return fail(GS_ERR_INVALID, "nodes hold %lld Gaussians, the hierarchy over %lld leaves needs %lld",
                (long long)nodes->n, (long long)n_leaf, (long long)gs_lod_nodes(n_leaf));
  if (n_leaf > 0 && !parent_dev) return fail(GS_ERR_INVALID, "parent is NULL");
  const size_t need = gs_lod_build_workspace(n_leaf);
  if (!ws || ws_bytes < need) return fail(GS_ERR_OOM, "lod_build workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  return launch_lod_build(*nodes, n_leaf, parent_dev, ws, (cudaStream_t)stream);
}

gs_status gs_project_lod(const gs_params* nodes, int64_t n_leaf, const int32_t* parent_dev, float tau,
                         const float* poses_dev, const gs_camera* cams, int32_t views, const gs_raster_cfg* cfg,
                         gs_splats* out, gs_stream stream) {
  GS_NVTX("gs_project_lod");
  gs_status st;
  if ((st = check_params(nodes)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if (n_leaf < 0 || n_leaf > nodes->n) return fail(GS_ERR_INVALID, "n_leaf out of range");
  if (nodes->n > 0 && !parent_dev) return fail(GS_ERR_INVALID, "parent is NULL");
  if (!(tau >= 0.f)) return fail(GS_ERR_INVALID, "tau must be >= 0");
  if ((st = check_splats(out, nodes->n, views)) != GS_OK) return st;
  return launch_project(*nodes, poses_dev, vt, *cfg, *out, (cudaStream_t)stream, parent_dev, n_leaf, tau);
}

static gs_status check_hier(const gs_grads* nodes, const gs_hier* h) {
  if (!nodes || !h) return fail(GS_ERR_INVALID, "NULL nodes or hierarchy");
  gs_params view{nodes->means4, nodes->scale_opa, nodes->quat, nodes->sh, nodes->n, nodes->sh_degree,
                 nodes->sh_stride};
  gs_status st;
  if ((st = check_params(&view)) != GS_OK) return st;
  if (h->capacity < 1 || h->capacity > nodes->n || h->capacity >= (1ll << 31))
    return fail(GS_ERR_INVALID, "hierarchy capacity must be 1..nodes->n");
  if (!h->parent || !h->child || !h->active || !h->n_nodes)
    return fail(GS_ERR_INVALID, "NULL hierarchy array");
  return GS_OK;
}

size_t gs_hier_workspace(int64_t capacity) { return hier_workspace_bytes(std::max<int64_t>(1, capacity)); }

gs_status gs_hier_analyze(gs_grads* nodes, gs_hier* h, const gs_grads* adam_m, const gs_grads* adam_v,
                          const float* pose_dev, const gs_camera* cam, float znear, float tau_l, void* ws,
                          size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_hier_analyze");
  gs_status st;
  if ((st = check_hier(nodes, h)) != GS_OK) return st;
  if (!pose_dev || !cam) return fail(GS_ERR_INVALID, "NULL pose or camera");
  if (!(znear > 0.f) || !(tau_l > 0.f)) return fail(GS_ERR_INVALID, "znear and tau_l must be > 0");
  const size_t need = gs_hier_workspace(h->capacity);
  if (!ws || ws_bytes < need) return fail(GS_ERR_OOM, "hier workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  return launch_hier_analyze(*nodes, *h, adam_m, adam_v, pose_dev, *cam, znear, tau_l, ws, (cudaStream_t)stream);
}

gs_status gs_hier_refine(gs_grads* nodes, gs_hier* h, const gs_grads* adam_m, const gs_grads* adam_v,
                         const float* pose_dev, const gs_camera* cam, float znear, float tau_h, int32_t passes,
                         void* ws, size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_hier_refine");
  gs_status st;
  if ((st = check_hier(nodes, h)) != GS_OK) return st;
  if (!pose_dev || !cam) return fail(GS_ERR_INVALID, "NULL pose or camera");
  if (!(znear > 0.f) || !(tau_h > 0.f) || passes < 1 || passes > 64)
    return fail(GS_ERR_INVALID, "znear, tau_h must be > 0 and passes 1..64");
  const size_t need = gs_hier_workspace(h->capacity);
  if (!ws || ws_bytes < need) return fail(GS_ERR_OOM, "hier workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  return launch_hier_refine(*nodes, *h, adam_m, adam_v, pose_dev, *cam, znear, tau_h, passes, ws,
                            (cudaStream_t)stream);
}

gs_status gs_project_hier(const gs_params* nodes, const gs_hier* h, float tau_h, const float* poses_dev,
                          const gs_camera* cams, int32_t views, const gs_raster_cfg* cfg, gs_splats* out,
                          gs_stream stream) {
  GS_NVTX("gs_project_hier");
  gs_status st;
  if ((st = check_params(nodes)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if (!h || !h->parent || !h->child || !h->active || !h->n_nodes || h->capacity < nodes->n)
    return fail(GS_ERR_INVALID, "hierarchy arrays must cover nodes->n rows");
  if (!(tau_h > 0.f)) return fail(GS_ERR_INVALID, "tau_h must be > 0");
  if ((st = check_splats(out, nodes->n, views)) != GS_OK) return st;
  return launch_project(*nodes, poses_dev, vt, *cfg, *out, (cudaStream_t)stream, nullptr, 0, tau_h, h);
}

gs_status gs_project_hier_render(const gs_params* nodes, const gs_hier* h, float tau, const float* poses_dev,
                                 const gs_camera* cams, int32_t views, const gs_raster_cfg* cfg, gs_splats* out,
                                 gs_stream stream) {
  GS_NVTX("gs_project_hier_render");
  gs_status st;
  if ((st = check_params(nodes)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if (!h || !h->parent || !h->child || !h->n_nodes || h->capacity < nodes->n)
    return fail(GS_ERR_INVALID, "hierarchy arrays must cover nodes->n rows");
  if (!(tau > 0.f)) return fail(GS_ERR_INVALID, "tau must be > 0");
  if ((st = check_splats(out, nodes->n, views)) != GS_OK) return st;
  return launch_project(*nodes, poses_dev, vt, *cfg, *out, (cudaStream_t)stream, nullptr, 0, tau, h, true);
}

size_t gs_bin_sort_workspace(int64_t n, int32_t views, int64_t capacity) {
  return bin_sort_workspace_bytes(std::max<int64_t>(0, n) * std::max(0, views), std::max<int64_t>(0, capacity));
}

gs_status gs_bin_sort(const gs_splats* splats, const gs_camera* cams, int32_t views,
                      const gs_raster_cfg* cfg, gs_bins* out, void* ws, size_t ws_bytes,
                      gs_stream stream) {
  GS_NVTX("gs_bin_sort");
  gs_status st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!splats) return fail(GS_ERR_INVALID, "splats is NULL");
  if ((st = check_splats(splats, splats->n, views)) != GS_OK) return st;
  if ((st = check_bins(out, vt, splats->n)) != GS_OK) return st;
  const size_t need = gs_bin_sort_workspace(splats->n, views, out->capacity);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "bin_sort workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  return launch_bin_sort(*splats, vt, *out, ws, (cudaStream_t)stream);
}

gs_status gs_render_fwd(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                        int32_t views, const gs_raster_cfg* cfg, float* image, float* alpha,
                        gs_stream stream) {
  GS_NVTX("gs_render_fwd");
  gs_status st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!splats) return fail(GS_ERR_INVALID, "splats is NULL");
  if ((st = check_splats(splats, splats->n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, splats->n)) != GS_OK) return st;
  if (!image) return fail(GS_ERR_INVALID, "image is NULL");
  return launch_render_fwd(*splats, *bins, vt, *cfg, image, alpha, (cudaStream_t)stream);
}

static size_t bwd_layout(int64_t n, int32_t views, int64_t capacity, char* base, float** partials,
                         float** pose_partials, float** drgb) {
  const int64_t warps = pose_partial_warps(n);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1), 256);
    return p;
  };
  float* pa = (float*)take(sizeof(float) * kPartialStride * (size_t)std::max<int64_t>(0, capacity));
  float* pp = (float*)take(sizeof(float) * 9 * (size_t)warps * (size_t)std::max(1, views));
  // three float4 planes per (view, Gaussian): summed geometry / opacity and colour gradients
  float* dc = (float*)take(sizeof(float) * 12 * (size_t)std::max<int64_t>(0, n) * (size_t)std::max(1, views));
  if (drgb) *drgb = dc;
  if (partials) *partials = pa;
  if (pose_partials) *pose_partials = pp;
  return off;
}

}  // extern "C"

namespace gs {
size_t render_bwd_ws_bytes(int64_t n, int32_t views, int64_t capacity) {
  return bwd_layout(n, views, capacity, nullptr, nullptr, nullptr, nullptr);
}

void render_bwd_ws_layout(int64_t n, int32_t views, int64_t capacity, void* ws, float** partials,
                          float** pose_partials, float** drgb) {
  bwd_layout(n, views, capacity, static_cast<char*>(ws), partials, pose_partials, drgb);
}
}  // namespace gs

extern "C" {

size_t gs_render_bwd_workspace(int64_t n, int32_t views, int64_t capacity) {
  return bwd_layout(n, views, capacity, nullptr, nullptr, nullptr, nullptr);
}

gs_status gs_render_bwd_pixels(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                               int32_t views, const gs_raster_cfg* cfg, const float* dL_dimage,
                               const float* dL_dalpha, const float* image, int64_t n, void* ws,
                               size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_render_bwd_pixels");
  gs_status st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if ((st = check_splats(splats, n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, n)) != GS_OK) return st;
  if (!dL_dimage) return fail(GS_ERR_INVALID, "dL_dimage is NULL");
  const size_t need = gs_render_bwd_workspace(n, views, bins->capacity);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "render_bwd workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  float *partials, *pose_partials, *drgb;
  bwd_layout(n, views, bins->capacity, static_cast<char*>(ws), &partials, &pose_partials, &drgb);
  return launch_render_bwd(*splats, *bins, vt, *cfg, dL_dimage, dL_dalpha, image, partials,
                           (cudaStream_t)stream);
}

gs_status gs_render_bwd_gaussians(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                                  int32_t views, const gs_splats* splats, const gs_bins* bins,
                                  const gs_raster_cfg* cfg, gs_grads* grads, float* dL_dpose, void* ws,
                                  size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_render_bwd_gaussians");
  gs_status st;
  if ((st = check_params(params)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if ((st = check_splats(splats, params->n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, params->n)) != GS_OK) return st;
  if (!grads || grads->n != params->n || grads->sh_degree != params->sh_degree ||
      (grads->sh_stride != 0 && grads->sh_stride < grads->n))
    return fail(GS_ERR_INVALID, "grads must match params");
  if (params->n > 0 && (!grads->means4 || !grads->scale_opa || !grads->quat || !grads->sh))
    return fail(GS_ERR_INVALID, "NULL gradient array");
  if (!aligned(grads->means4, 16) || !aligned(grads->scale_opa, 16) || !aligned(grads->quat, 16))
    return fail(GS_ERR_INVALID, "gradient arrays must be 16-byte aligned");
  const size_t need = gs_render_bwd_workspace(params->n, views, bins->capacity);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "render_bwd workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  float *partials, *pose_partials, *drgb;
  bwd_layout(params->n, views, bins->capacity, static_cast<char*>(ws), &partials, &pose_partials, &drgb);
  return launch_project_bwd(*params, poses_dev, vt, *cfg, *splats, *bins, partials, *grads, pose_partials,
                            dL_dpose, drgb, (cudaStream_t)stream);
}

static gs_status check_like(const gs_grads* x, const gs_grads* params, const char* what) {
  if (!x || x->n != params->n || x->sh_degree != params->sh_degree || (x->sh_stride != 0 && x->sh_stride < x->n))
    return fail(GS_ERR_INVALID, "%s must match params", what);
  if (params->n > 0 && (!x->means4 || !x->scale_opa || !x->quat || !x->sh))
    return fail(GS_ERR_INVALID, "NULL %s array", what);
  if (!aligned(x->means4, 16) || !aligned(x->scale_opa, 16) || !aligned(x->quat, 16))
    return fail(GS_ERR_INVALID, "%s arrays must be 16-byte aligned", what);
  return GS_OK;
}

gs_status gs_render_bwd_gaussians_adam(gs_grads* params, const float* poses_dev, const gs_camera* cams,
                                       int32_t views, const gs_splats* splats, const gs_bins* bins,
                                       const gs_raster_cfg* cfg, gs_grads* grads, gs_grads* adam_m,
                                       gs_grads* adam_v, const gs_adam_params_cfg* adam, float* dL_dpose, void* ws,
                                       size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_render_bwd_gaussians_adam");
  if (!params || !adam) return fail(GS_ERR_INVALID, "NULL params or Adam settings");
  const gs_params pv{params->means4, params->scale_opa, params->quat, params->sh, params->n, params->sh_degree,
                     params->sh_stride};
  gs_status st;
  if ((st = check_params(&pv)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if ((st = check_splats(splats, params->n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, params->n)) != GS_OK) return st;
  if ((st = check_like(grads, params, "grads")) != GS_OK || (st = check_like(adam_m, params, "adam_m")) != GS_OK ||
      (st = check_like(adam_v, params, "adam_v")) != GS_OK)
    return st;
  if ((adam_m->sh_stride > 0 ? adam_m->sh_stride : adam_m->n) != (adam_v->sh_stride > 0 ? adam_v->sh_stride : adam_v->n))
    return fail(GS_ERR_INVALID, "adam_m and adam_v need the same sh_stride");
  if (adam->step < 1 && !adam->step_dev) return fail(GS_ERR_INVALID, "step must be >= 1");
  if (!(adam->beta1 >= 0.f && adam->beta1 < 1.f && adam->beta2 >= 0.f && adam->beta2 < 1.f && adam->eps >= 0.f))
    return fail(GS_ERR_INVALID, "bad Adam hyper-parameters");
  if (adam->update_mask & ~15u) return fail(GS_ERR_INVALID, "update_mask has bits beyond 0-3");
  const size_t need = gs_render_bwd_workspace(params->n, views, bins->capacity);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "render_bwd workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  float *partials, *pose_partials, *drgb;
  bwd_layout(params->n, views, bins->capacity, static_cast<char*>(ws), &partials, &pose_partials, &drgb);
  return launch_project_bwd_adam(pv, poses_dev, vt, *cfg, *splats, *bins, partials, *grads, pose_partials,
                                 dL_dpose, drgb, *params, *adam_m, *adam_v, *adam, (cudaStream_t)stream);
}

static size_t fused_layout(int64_t n, int32_t views, int64_t capacity, int64_t num_tiles, char* base,
                           uint32_t** queue, float** tile_loss) {
  size_t off = bwd_layout(n, views, capacity, nullptr, nullptr, nullptr, nullptr);
  if (queue) *queue = base ? reinterpret_cast<uint32_t*>(base + off) : nullptr;
  off += 256;
  if (tile_loss) *tile_loss = base ? reinterpret_cast<float*>(base + off) : nullptr;
  off += align_up(sizeof(float) * (size_t)std::max<int64_t>(1, num_tiles), 256);
  return off;
}

size_t gs_render_fused_workspace(int64_t n, int32_t views, int64_t capacity, int64_t num_tiles) {
  return fused_layout(n, views, capacity, num_tiles, nullptr, nullptr, nullptr);
}

gs_status gs_render_fused(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams, int32_t views,
                          const gs_raster_cfg* cfg, const float* target, int32_t loss_kind, float* image,
                          float* alpha, float* loss_dev, int64_t n, void* ws, size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_render_fused");
  gs_status st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if ((st = check_splats(splats, n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, n)) != GS_OK) return st;
  if (!target || !image || !loss_dev) return fail(GS_ERR_INVALID, "NULL target, image or loss");
  if (loss_kind != 0 && loss_kind != 1) return fail(GS_ERR_INVALID, "loss_kind must be 0 (L1) or 1 (MSE)");
  if ((cfg->schedule & GS_SCHED_FUSED_LONGEST_FIRST) && !bins->tile_order)
    return fail(GS_ERR_INVALID, "GS_SCHED_FUSED_LONGEST_FIRST needs bins.tile_order");
  const size_t need = gs_render_fused_workspace(n, views, bins->capacity, bins->num_tiles);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "render_fused workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  float *partials, *pose_partials, *drgb, *tile_loss;
  uint32_t* queue;
  bwd_layout(n, views, bins->capacity, static_cast<char*>(ws), &partials, &pose_partials, &drgb);
  fused_layout(n, views, bins->capacity, bins->num_tiles, static_cast<char*>(ws), &queue, &tile_loss);
  return launch_render_fused(*splats, *bins, vt, *cfg, target, loss_kind, image, alpha, loss_dev, partials,
                             tile_loss, queue, (cudaStream_t)stream);
}

gs_status gs_render_bwd(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                        int32_t views, const gs_splats* splats, const gs_bins* bins,
                        const gs_raster_cfg* cfg, const float* dL_dimage, const float* dL_dalpha,
                        const float* image, gs_grads* grads, float* dL_dpose, void* ws,
                        size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_render_bwd");
  gs_status st;
  if ((st = check_params(params)) != GS_OK) return st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!poses_dev) return fail(GS_ERR_INVALID, "poses is NULL");
  if ((st = check_splats(splats, params->n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, params->n)) != GS_OK) return st;
  if (!dL_dimage) return fail(GS_ERR_INVALID, "dL_dimage is NULL");
  if (!grads || grads->n != params->n || grads->sh_degree != params->sh_degree ||
      (grads->sh_stride != 0 && grads->sh_stride < grads->n))
    return fail(GS_ERR_INVALID, "grads must match params");
  if (params->n > 0 && (!grads->means4 || !grads->scale_opa || !grads->quat || !grads->sh))
    return fail(GS_ERR_INVALID, "NULL gradient array");
  if (!aligned(grads->means4, 16) || !aligned(grads->scale_opa, 16) || !aligned(grads->quat, 16))
    return fail(GS_ERR_INVALID, "gradient arrays must be 16-byte aligned");
  const size_t need = gs_render_bwd_workspace(params->n, views, bins->capacity);
  if (!ws || ws_bytes < need)
    return fail(GS_ERR_OOM, "render_bwd workspace: need %zu bytes, got %zu", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  float *partials, *pose_partials, *drgb;
  bwd_layout(params->n, views, bins->capacity, static_cast<char*>(ws), &partials, &pose_partials, &drgb);
  cudaStream_t s = (cudaStream_t)stream;
  st = launch_render_bwd(*splats, *bins, vt, *cfg, dL_dimage, dL_dalpha, image, partials, s);
  if (st != GS_OK) return st;
  return launch_project_bwd(*params, poses_dev, vt, *cfg, *splats, *bins, partials, *grads, pose_partials,
                            dL_dpose, drgb, s);
}

gs_status gs_adam_step(float* p, const float* g, float* m, float* v, int64_t n,
                       const gs_adam_cfg* cfg, int32_t step, gs_stream stream) {
  GS_NVTX("gs_adam_step");
  if (!cfg) return fail(GS_ERR_INVALID, "cfg is NULL");
  if (n < 0) return fail(GS_ERR_INVALID, "n < 0");
  if (step < 1 && !cfg->step_dev) return fail(GS_ERR_INVALID, "step must be >= 1");
  if (n > 0 && (!p || !g || !m || !v)) return fail(GS_ERR_INVALID, "NULL arena");
  if (!aligned(p, 16) || !aligned(g, 16) || !aligned(m, 16) || !aligned(v, 16))
    return fail(GS_ERR_INVALID, "arenas must be 16-byte aligned");
  if (cfg->num_groups < 0 || cfg->num_groups > GS_MAX_ADAM_GROUPS || (cfg->num_groups > 0 && !cfg->groups))
    return fail(GS_ERR_INVALID, "num_groups must be 0..%d", GS_MAX_ADAM_GROUPS);
  if (cfg->num_groups == 0 && !cfg->pose) return fail(GS_ERR_INVALID, "no group and no pose step");
  for (int k = 0; k < cfg->num_groups; ++k) {
    const gs_adam_group& G = cfg->groups[k];
    if (G.begin < 0 || G.end < G.begin || G.end > n) return fail(GS_ERR_INVALID, "group %d out of range", k);
    for (int j = 0; j < k; ++j) {
      const gs_adam_group& H = cfg->groups[j];
      if (G.begin < H.end && H.begin < G.end) return fail(GS_ERR_INVALID, "groups %d and %d overlap", j, k);
    }
    if ((G.end - G.begin + (int64_t)(16 * 256) - 1) / (16 * 256) >= (1ll << 30))
      return fail(GS_ERR_INVALID, "group %d too large", k);
  }
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f))
    return fail(GS_ERR_INVALID, "bad Adam hyper-parameters");
  if (cfg->pose && (cfg->views < 1 || !cfg->dpose || !cfg->pose_m || !cfg->pose_v))
    return fail(GS_ERR_INVALID, "pose step needs views, dpose, pose_m, pose_v");
  return launch_adam(p, g, m, v, n, *cfg, step, (cudaStream_t)stream);
}

gs_status gs_render_stats(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams, int32_t views,
                          const gs_raster_cfg* cfg, uint64_t* stats_dev, gs_stream stream) {
  GS_NVTX("gs_render_stats");
  gs_status st;
  if ((st = check_cfg(cfg)) != GS_OK) return st;
  ViewTable vt;
  if (!make_view_table(cams, views, &vt, cfg->tile_w, cfg->tile_h)) return GS_ERR_INVALID;
  if (!splats) return fail(GS_ERR_INVALID, "splats is NULL");
  if ((st = check_splats(splats, splats->n, views)) != GS_OK) return st;
  if ((st = check_bins(bins, vt, splats->n)) != GS_OK) return st;
  if (!stats_dev || !aligned(stats_dev, 8)) return fail(GS_ERR_INVALID, "stats must be 8-byte aligned device memory");
  return launch_render_stats(*splats, *bins, vt, reinterpret_cast<unsigned long long*>(stats_dev),
                             (cudaStream_t)stream);
}

size_t gs_image_loss_workspace(void) { return loss_workspace_bytes(); }

gs_status gs_image_loss(const float* image, const float* target, int64_t count, int32_t kind,
                        float* dL_dimage, float* loss_dev, void* ws, size_t ws_bytes, gs_stream stream) {
  GS_NVTX("gs_image_loss");
  if (count <= 0) return fail(GS_ERR_INVALID, "count must be > 0");
  if (!image || !target || !loss_dev) return fail(GS_ERR_INVALID, "NULL image, target or loss");
  if (kind != 0 && kind != 1) return fail(GS_ERR_INVALID, "kind must be 0 (L1) or 1 (MSE)");
  if (!ws || ws_bytes < loss_workspace_bytes())
    return fail(GS_ERR_OOM, "image_loss workspace: need %zu bytes, got %zu", loss_workspace_bytes(), ws_bytes);
  return launch_loss(image, target, count, kind, dL_dimage, loss_dev, ws, (cudaStream_t)stream);
}

}  // extern "C"
