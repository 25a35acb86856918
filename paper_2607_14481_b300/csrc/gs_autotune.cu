// Autotuners of the batched iteration's knobs.
//
// gs_autotune_blend: for the caller's current projection and tile lists it
// times every composite schedule (tile order: natural or longest lists first;
// splats per shared memory batch: 128, 64, 256) and every single-pass
// backward schedule (order; batch 128, 64) with CUDA events and keeps the
// fastest of each.  A schedule never changes a result, only the time.
//
// gs_autotune_fused: the knobs of the fused persistent pass, tile shape
// included.  The tile shape changes the tile lists, so every shape is
// projected and binned again; each candidate (shape x splats per batch x
// work order) is timed over projection + binning + the fused pass.
#include <chrono>
#include <cmath>
#include <thread>

#include "gs_internal.h"

namespace {

// Waits for an event with a bound (the GPU may be shared); false on timeout.
bool wait_event(cudaEvent_t ev, double timeout_s) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e;
  while ((e = cudaEventQuery(ev)) == cudaErrorNotReady) {
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s) return false;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return e == cudaSuccess;
}

}  // namespace

extern "C" gs_status gs_autotune_blend(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                                       int32_t views, gs_raster_cfg* cfg, float* image, const float* dL_dimage,
                                       int64_t n, void* ws, size_t ws_bytes, int32_t reps, float* times_ms,
                                       gs_stream stream) {
  GS_NVTX("gs_autotune_blend");
  if (!cfg || !bins) return gs::fail(GS_ERR_INVALID, "NULL cfg or bins");
  if (reps < 1 || reps > 1000) return gs::fail(GS_ERR_INVALID, "reps must be 1..1000");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return gs::check_launch("autotune event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return gs::check_launch("autotune event");
  }
  const uint32_t base = cfg->schedule;
  const uint32_t fwd_mask = GS_SCHED_FWD_LONGEST_FIRST | GS_SCHED_FWD_BATCH(3);
  const uint32_t bwd_mask = GS_SCHED_BWD_LONGEST_FIRST | GS_SCHED_BWD_BATCH(3);
  gs_status st = GS_OK;
  // time `reps` launches of one candidate (after one launch to warm it)
  auto timed = [&](uint32_t sched, bool fwd, float* ms) -> gs_status {
    gs_raster_cfg c = *cfg;
    c.schedule = sched;
    auto run = [&]() {
      return fwd ? gs_render_fwd(splats, bins, cams, views, &c, image, nullptr, stream)
                 : gs_render_bwd_pixels(splats, bins, cams, views, &c, dL_dimage, nullptr, image, n, ws, ws_bytes,
                                        stream);
    };
    gs_status r = run();
    if (r != GS_OK) return r;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && r == GS_OK; ++i) r = run();
    cudaEventRecord(e1, s);
    if (r != GS_OK) return r;
    if (!wait_event(e1, 60.0)) return gs::fail(GS_ERR_TIMEOUT, "autotune: a candidate did not finish");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)reps;
    return gs::check_launch("autotune");
  };
  const bool have_order = bins->tile_order != nullptr;
  uint32_t best_fwd = base & fwd_mask, best_bwd = base & bwd_mask;
  float t_fwd = INFINITY, t_bwd = INFINITY;
  int slot = 0;
  for (int order = 0; order < 2 && st == GS_OK; ++order)
    for (uint32_t b = 0; b < 3 && st == GS_OK; ++b, ++slot) {
      float ms = NAN;
      if (order == 0 || have_order) {
        const uint32_t sched = (order ? GS_SCHED_FWD_LONGEST_FIRST : 0u) | GS_SCHED_FWD_BATCH(b);
        st = timed((base & ~fwd_mask) | sched, true, &ms);
        if (st == GS_OK && ms < t_fwd) { t_fwd = ms; best_fwd = sched; }
      }
      if (times_ms) times_ms[slot] = ms;
    }
  // the image the backward reads: the composite with the chosen schedule
  if (st == GS_OK) {
    gs_raster_cfg c = *cfg;
    c.schedule = (base & ~fwd_mask) | best_fwd;
    st = gs_render_fwd(splats, bins, cams, views, &c, image, nullptr, stream);
  }
  for (int order = 0; order < 2 && st == GS_OK; ++order)
    for (uint32_t b = 0; b < 2 && st == GS_OK; ++b, ++slot) {
      float ms = NAN;
      if (order == 0 || have_order) {
        const uint32_t sched = (order ? GS_SCHED_BWD_LONGEST_FIRST : 0u) | GS_SCHED_BWD_BATCH(b);
        st = timed((base & ~bwd_mask) | best_fwd | sched, false, &ms);
        if (st == GS_OK && ms < t_bwd) { t_bwd = ms; best_bwd = sched; }
      }
      if (times_ms) times_ms[slot] = ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GS_OK) return st;
  cfg->schedule = best_fwd | best_bwd;
  return GS_OK;
}

namespace {

const int kShapes[3][2] = {{16, 16}, {32, 8}, {8, 32}};

int64_t tiles_of(const gs_camera* cams, int views, int tw, int th) {
  int64_t t = 0;
  for (int v = 0; v < views; ++v)
    t += (int64_t)((cams[v].width + tw - 1) / tw) * ((cams[v].height + th - 1) / th);
  return t;
}

}  // namespace

extern "C" gs_status gs_autotune_fused(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                                       int32_t views, gs_raster_cfg* cfg, gs_splats* splats, gs_bins* bins,
                                       int64_t ranges_tiles, void* bin_ws, size_t bin_ws_bytes, const float* target,
                                       int32_t loss_kind, float* image, float* loss_dev, void* ws, size_t ws_bytes,
                                       int32_t reps, float* times_ms, gs_stream stream) {
  GS_NVTX("gs_autotune_fused");
  if (!cfg || !bins || !params || !splats || !cams) return gs::fail(GS_ERR_INVALID, "NULL argument");
  if (reps < 1 || reps > 1000) return gs::fail(GS_ERR_INVALID, "reps must be 1..1000");
  if (views < 1 || views > GS_MAX_VIEWS) return gs::fail(GS_ERR_INVALID, "views must be 1..%d", GS_MAX_VIEWS);
  if (!bins->counts) return gs::fail(GS_ERR_INVALID, "bins.counts is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return gs::check_launch("autotune event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return gs::check_launch("autotune event");
  }
  const uint32_t fused_mask = GS_SCHED_FUSED_LONGEST_FIRST | GS_SCHED_FUSED_BATCH(3);
  const uint32_t base = cfg->schedule & ~fused_mask;
  gs_raster_cfg best = *cfg;
  float t_best = INFINITY;
  gs_status st = GS_OK;
  // one candidate: projection + binning + fused pass with configuration c
  auto step = [&](const gs_raster_cfg& c, gs_bins& b) -> gs_status {
    gs_status r = gs_project(params, poses_dev, cams, views, &c, splats, stream);
    if (r == GS_OK) r = gs_bin_sort(splats, cams, views, &c, &b, bin_ws, bin_ws_bytes, stream);
    if (r == GS_OK)
      r = gs_render_fused(splats, &b, cams, views, &c, target, loss_kind, image, nullptr, loss_dev, params->n, ws,
                          ws_bytes, stream);
    return r;
  };
  int slot = 0;
  for (int sh = 0; sh < 3 && st == GS_OK; ++sh) {
    gs_raster_cfg c = *cfg;
    c.tile_w = kShapes[sh][0];
    c.tile_h = kShapes[sh][1];
    gs_bins b = *bins;
    b.num_tiles = tiles_of(cams, views, c.tile_w, c.tile_h);
    const bool fits = b.num_tiles <= ranges_tiles &&
                      gs_render_fused_workspace(params->n, views, b.capacity, b.num_tiles) <= ws_bytes;
    bool ok = fits;
    if (ok) {
      // warm-up, then check the pair capacity
      c.schedule = base;
      st = step(c, b);
      uint32_t cnt[4] = {0, 0, 0, 0};
      if (st == GS_OK && cudaMemcpyAsync(cnt, b.counts, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = gs::check_launch("autotune counts");
      if (st == GS_OK) {
        cudaEventRecord(e1, s);
        if (!wait_event(e1, 60.0)) st = gs::fail(GS_ERR_TIMEOUT, "autotune: a candidate did not finish");
      }
      ok = st == GS_OK && cnt[2] == 0;
    }
    for (int bt = 0; bt < 3; ++bt)
      for (int order = 0; order < 2; ++order, ++slot) {
        float ms = NAN;
        if (ok && st == GS_OK && (order == 0 || b.tile_order)) {
          c.schedule = base | GS_SCHED_FUSED_BATCH(bt) | (order ? GS_SCHED_FUSED_LONGEST_FIRST : 0u);
          st = step(c, b);
          if (st == GS_OK) {
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps && st == GS_OK; ++i) st = step(c, b);
            cudaEventRecord(e1, s);
          }
          if (st == GS_OK && !wait_event(e1, 60.0))
            st = gs::fail(GS_ERR_TIMEOUT, "autotune: a candidate did not finish");
          if (st == GS_OK) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t / (float)reps;
            if (ms < t_best) {
              t_best = ms;
              best = c;
            }
            st = gs::check_launch("autotune");
          }
        }
        if (times_ms) times_ms[slot] = ms;
      }
  }
  if (st == GS_OK && !(t_best < INFINITY)) st = gs::fail(GS_ERR_OOM, "autotune: no candidate fits the buffers");
  if (st == GS_OK) {
    // leave the caller's buffers with the chosen configuration's results
    gs_bins b = *bins;
    b.num_tiles = tiles_of(cams, views, best.tile_w, best.tile_h);
    st = step(best, b);
    if (st == GS_OK) {
      *cfg = best;
      bins->num_tiles = b.num_tiles;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
