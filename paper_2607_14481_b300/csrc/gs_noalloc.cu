// gs_bin_sort_noalloc: gs_bin_sort with its workspace in a static device
// array inside libgs instead of a caller buffer.  It allocates nothing: no
// cudaMalloc / cudaFree, no allocating library.
//
// Who cannot allocate, and why:
//   - a C host (or a plugin inside another application) that receives its
//     device buffers from an owner with its own pool and has no device
//     allocator of its own for temporaries;
//   - a latency-critical thread, where cudaMalloc / cudaFree may synchronise
//     the whole device and stall every other stream;
//   - a caller held to a fixed device-memory budget (such as an admission
//     budget), which must not grow its footprint per call.
// For those, small scenes (see the limit below) can be binned with no
// workspace at all.  The scratch costs GS_NOALLOC_SCRATCH_BYTES of device
// memory per device once libgs is loaded on it.
#include <mutex>

#include "gs_internal.h"

namespace {

// The whole workspace of one gs_bin_sort call.  Nothing in it has to start
// at zero: every word the sort reads is written earlier in the same call (its
// scalar block by the first kernel it launches).
static __device__ __align__(256) unsigned char g_sort_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  Outside stream
// capture it is looked up on every call (cheap), so a device reset or a
// re-created context never leaves a stale address behind; under capture the
// address cached by an earlier call on this device is used (the lookup may
// load the module, which must not happen inside a capture).
gs_status scratch_address(cudaStream_t stream, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return gs::check_launch("gs_bin_sort_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return gs::fail(GS_ERR_INVALID, "gs_bin_sort_noalloc: device %d unsupported", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return gs::fail(GS_ERR_CUDA, "gs_bin_sort_noalloc: cudaStreamIsCapturing failed");
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap != cudaStreamCaptureStatusNone) {
    if (!g_scratch_ptr[dev])
      return gs::fail(GS_ERR_INVALID, "gs_bin_sort_noalloc: the first call on a device must come before any "
                                      "stream capture");
    *out = g_scratch_ptr[dev];
    return GS_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return gs::fail(GS_ERR_CUDA, "gs_bin_sort_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
  }
  g_scratch_ptr[dev] = p;
  *out = p;
  return GS_OK;
}

}  // namespace

// The scratch size as a data symbol, so that bindings read it from the library
// instead of repeating the constant.
extern "C" GS_API const uint64_t gs_noalloc_scratch_bytes = GS_NOALLOC_SCRATCH_BYTES;

// Validation beyond the size check, and the launches, are gs_bin_sort's own:
// the scratch is handed to it as the workspace.
extern "C" gs_status gs_bin_sort_noalloc(const gs_splats* splats, const gs_camera* cams, int32_t views,
                                         const gs_raster_cfg* cfg, gs_bins* out, gs_stream stream) {
  GS_NVTX("gs_bin_sort_noalloc");
  if (!splats || !out) return gs::fail(GS_ERR_INVALID, "gs_bin_sort_noalloc: NULL splats or bins");
  const size_t need = gs_bin_sort_workspace(splats->n, views, out->capacity);
  if (need > (size_t)GS_NOALLOC_SCRATCH_BYTES)
    return gs::fail(GS_ERR_OOM,
                    "gs_bin_sort_noalloc: n*views = %lld with capacity %lld needs %zu bytes of scratch, the "
                    "static scratch holds %zu (e.g. 65536 items with 262144 pairs); use gs_bin_sort with a "
                    "workspace",
                    (long long)splats->n * views, (long long)out->capacity, need,
                    (size_t)GS_NOALLOC_SCRATCH_BYTES);
  void* ws = nullptr;
  const gs_status st = scratch_address((cudaStream_t)stream, &ws);
  if (st != GS_OK) return st;
  return gs_bin_sort(splats, cams, views, cfg, out, ws, (size_t)GS_NOALLOC_SCRATCH_BYTES, stream);
}
