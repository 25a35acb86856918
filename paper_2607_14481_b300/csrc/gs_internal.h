// Host-side internals shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/gs.h"
#include "gs_device.cuh"

namespace gs {

// Record a failure message for gs_last_error (thread-local) and return `st`.
gs_status fail(gs_status st, const char* fmt, ...);
// Map the last CUDA error (if any) to GS_ERR_CUDA with a message.
gs_status check_launch(const char* what);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NVTX range over a scope (an ABI call or a session stage): visible in a
// profiler's timeline, a no-op when no tool is attached (NVTX 3 is header-only).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GS_NVTX(name) ::gs::NvtxRange gs_nvtx_scope_(name)

// Launches `kernel` so that it may start while the kernel before it on the
// stream finishes (programmatic dependent launch, kept in a captured graph):
// the kernel's first statement is chain_enter(), so only the launch and the
// start of its blocks overlap the predecessor's tail, not any of its reads.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Schedule bits of gs_raster_cfg (see gs.h).
constexpr uint32_t kSchedFwdLongestFirst = GS_SCHED_FWD_LONGEST_FIRST;
constexpr uint32_t kSchedBwdLongestFirst = GS_SCHED_BWD_LONGEST_FIRST;
constexpr int kSchedFwdBatchShift = 4;
constexpr int kSchedBwdBatchShift = 8;
constexpr int kSchedFusedBatchShift = 12;
constexpr uint32_t kSchedKnown = 0x7u | (3u << 4) | (3u << 8) | (3u << 12);

// Fills a ViewTable from host cameras for tiles of tw x th pixels; returns
// false (with a message) on invalid cameras or an unsupported tile shape.
bool make_view_table(const gs_camera* cams, int views, ViewTable* vt, int tw = kTile, int th = kTile);

// ---- kernels' host launchers (each enqueues on `s`, returns GS_OK or GS_ERR_CUDA)
// parent != nullptr: level-of-detail cut (nodes [0, n_leaf) are leaves);
// hier != nullptr: the view cut of the progressive hierarchy at tau (the
// active set refined for the view), or with hier_roots its render cut from
// the roots.
gs_status launch_project(const gs_params& p, const float* poses, const ViewTable& vt,
                         const gs_raster_cfg& cfg, const gs_splats& out, cudaStream_t s,
                         const int32_t* parent = nullptr, int64_t n_leaf = 0, float tau = 0.f,
                         const gs_hier* hier = nullptr, bool hier_roots = false);

// Per-Gaussian backward with the Adam update fused in (gs_grad.cu).
gs_status launch_project_bwd_adam(const gs_params& p, const float* poses, const ViewTable& vt,
                                  const gs_raster_cfg& cfg, const gs_splats& sp, const gs_bins& bins,
                                  const float* partials, const gs_grads& g, float* pose_partials, float* dpose,
                                  float* drgb, const gs_grads& prw, const gs_grads& m, const gs_grads& v,
                                  const gs_adam_params_cfg& acfg, cudaStream_t s);

// Progressive hierarchy (gs_hier.cu).
size_t hier_workspace_bytes(int64_t cap);
gs_status launch_hier_analyze(const gs_grads& nodes, const gs_hier& h, const gs_grads* m, const gs_grads* v,
                              const float* pose, const gs_camera& cam, float znear, float tau_l, void* ws,
                              cudaStream_t s);
gs_status launch_hier_refine(const gs_grads& nodes, const gs_hier& h, const gs_grads* m, const gs_grads* v,
                             const float* pose, const gs_camera& cam, float znear, float tau_h, int passes, void* ws,
                             cudaStream_t s);

// Loop-closure update: Gaussian i moves with the Sim(3) of keyframe kf[i].
gs_status launch_sim3_update(const gs_grads& p, const int32_t* kf, const float* sim3, int32_t num_kf,
                             uint32_t* status, cudaStream_t s);
gs_status launch_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);
// active (optional): only rows with a nonzero flag are counted.
gs_status launch_keyframe_counts(const int32_t* kf, int64_t n, int32_t num_kf, uint32_t* counts, cudaStream_t s,
                                 const uint8_t* active = nullptr);

// Local bundle adjustment (arguments validated by the caller).
size_t ba_workspace_bytes(int num_cams, int num_points, int obs_per_point);
gs_status launch_ba(const gs_ba_problem& prob, float* poses, float* points, float* focal, int iters,
                    double lambda0, double* trace, uint32_t* status, void* ws, cudaStream_t s);

// Level-of-detail hierarchy (coarse nodes after the leaves in `nodes`).
int64_t lod_level1(int64_t n);
int64_t lod_level2(int64_t n);
size_t lod_build_workspace_bytes(int64_t n);
gs_status launch_lod_build(const gs_grads& nodes, int64_t n_leaf, int32_t* parent, void* ws, cudaStream_t s);

// Exclusive scan of n_cap u32 values read every in_stride and written every
// out_stride elements (in place allowed); the number of valid entries is
// *n_dev (device); the total goes to *total_dev.
size_t scan_workspace(int64_t n_cap);
gs_status launch_scan(const uint32_t* in, int in_stride, uint32_t* out, int out_stride, const uint32_t* n_dev,
                      int64_t n_cap, uint32_t* total_dev, void* ws, cudaStream_t s);
// Largest number of tiles (all views) the binning workspace is sized for.
int64_t bin_sort_max_tiles();

// Stable LSD radix sort of (key, value) u32 pairs on key bits [0, bits);
// count *n_dev (device) <= n_cap.  keys/vals ping-pong between the *_a and
// *_b buffers; the result lands in (keys_out, vals_out).
size_t radix_workspace(int64_t n_cap);
gs_status launch_radix_sort(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                            uint32_t* keys_out, uint32_t* vals_out, const uint32_t* n_dev,
                            int64_t n_cap, int bits, void* ws, cudaStream_t s);

gs_status launch_render_fwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, float* image, float* alpha, cudaStream_t s);
gs_status launch_render_stats(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                              unsigned long long* stats, cudaStream_t s);
// Persistent fused composite + image loss + single-pass backward (see
// gs_render_fused); queue: 2 device words, tile_loss: [tiles] device floats.
gs_status launch_render_fused(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                              const gs_raster_cfg& cfg, const float* target, int loss_kind, float* image,
                              float* alpha, float* loss, float* partials, float* tile_loss, uint32_t* queue,
                              cudaStream_t s);
gs_status launch_render_bwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, const float* dimage, const float* dalpha,
                            const float* image, float* partials, cudaStream_t s);
gs_status launch_project_bwd(const gs_params& p, const float* poses, const ViewTable& vt,
                             const gs_raster_cfg& cfg, const gs_splats& sp, const gs_bins& bins,
                             const float* partials, const gs_grads& g, float* pose_partials, float* dpose,
                             float* drgb, cudaStream_t s);
// warps of the per-Gaussian backward (pose partials are kept per warp)
int64_t pose_partial_warps(int64_t n);
gs_status launch_adam(float* p, const float* g, float* m, float* v, int64_t n,
                      const gs_adam_cfg& cfg, int step, cudaStream_t s);

size_t loss_workspace_bytes();
gs_status launch_loss(const float* img, const float* tgt, int64_t count, int kind, float* grad,
                      float* loss, void* ws, cudaStream_t s);

// Per (tile, splat) pair as stored: dmx, dmy, dA, dB, dC, dopacity, dr, dg, db.
// Inside the blend kernels values 0-4 hold the moments of dL/dpower until
// store_pair applies the splat's conic.
constexpr int kPartialValues = 9;
constexpr int kPartialStride = 12;      // floats per (tile, splat) pair: 3 float4, last 3 unused
constexpr int kGradBlock = 256;         // threads per block of the per-Gaussian backward

}  // namespace gs
