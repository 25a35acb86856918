// Autotuner of the blend schedule (the batched iteration's knobs): for the
// caller's current projection and tile lists it times every composite
// schedule (tile order: natural or longest lists first; splats per shared
// memory batch: 128, 64, 256) and every single-pass backward schedule (order;
// batch 128, 64) with CUDA events and keeps the fastest of each.  A schedule
// never changes a result, only the time.  The tile shape is fixed at 16x16
// by the binning (gs_raster_cfg.tile_w/h), so it is not a knob here.
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
