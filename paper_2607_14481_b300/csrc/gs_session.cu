// Streaming session: a persistent loop that admits render and train requests
// as frames arrive (the live-capture mode of §5.2, where optimisation runs
// asynchronously until the next keyframe), batches them continuously, keeps
// the Gaussians, their Adam state and the tile lists resident on the device,
// admits work by an HBM budget and reports latency percentiles beside
// throughput.
//
// Threads.  gs_session_submit appends to a queue.  A worker thread forms a
// batch of up to max_batch_views queued requests as soon as a batch context is
// free and enqueues the batch without waiting for earlier batches: a request
// that arrives while batches run joins the next batch (continuous batching).
// A completion thread polls the events of every batch in flight (bounded
// waits), finishes whichever completes first, copies rendered images to the
// callers' buffers and records per-request latency.
//
// Streams.  Everything that writes the parameters (train parts, adds of
// Gaussians, loop closures, hierarchy builds) runs in issue order on the
// session's stream.  Render parts run on their own batch context's stream:
// a render part first waits for the event of the last write issued before it
// (it sees every update issued earlier), and a later write waits, on the
// device, for the render parts issued before it (its Adam step, or the add,
// does not change what they read).  So render parts run beside one another
// and beside the forward and backward of a train part issued after them.
//
// Within a batch, render views are rasterised first (they see the parameters
// before this batch's update), then the train views run the fused forward,
// loss and per-pixel backward, the per-Gaussian backward and one fused Adam
// step over every active Gaussian.  If a batch overflows its pair capacity
// the Adam step is skipped on the device, the capacity grows (within the
// budget) and the batch is issued again.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gs_internal.h"

namespace gs {

size_t bin_sort_workspace_bytes(int64_t m, int64_t cap);
gs_status launch_bin_sort(const gs_splats& sp, const ViewTable& vt, const gs_bins& bins, void* ws,
                          cudaStream_t s);
size_t render_bwd_ws_bytes(int64_t n, int32_t views, int64_t capacity);
void render_bwd_ws_layout(int64_t n, int32_t views, int64_t capacity, void* ws, float** partials,
                          float** pose_partials, float** drgb);

namespace {

double steady_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Runs f(lo, hi) over [0, n) in contiguous ranges of at least `grain`
// elements on the calling thread and up to seven helper threads: the host
// staging of a request (a target image of up to 25 MB) or of an add (the SH
// planes of 50k Gaussians) is memory-bound, and one core copies a fraction
// of what the host memory delivers.  Without helpers (one range, or a
// thread that cannot be started) the caller runs the rest itself.
template <class F>
void host_parallel(int64_t n, int64_t grain, F&& f) {
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  const int64_t T = std::max<int64_t>(1, std::min<int64_t>({8, hw, n / std::max<int64_t>(1, grain)}));
  if (T <= 1) {
    f((int64_t)0, n);
    return;
  }
  const int64_t step = (n + T - 1) / T;
  std::vector<std::thread> helpers;
  int64_t done_by_helpers = step;  // range [step, ...) goes to helpers while they start
  for (int64_t t = 1; t < T; ++t) {
    const int64_t lo = t * step, hi = std::min(n, lo + step);
    if (lo >= hi) break;
    try {
      helpers.emplace_back([&f, lo, hi] { f(lo, hi); });
      done_by_helpers = hi;
    } catch (...) {
      break;
    }
  }
  f((int64_t)0, std::min(n, step));
  if (done_by_helpers < n) f(done_by_helpers, n);
  for (auto& h : helpers) h.join();
}

struct Req {
  int64_t id = 0;
  int32_t kind = 0;
  gs_camera cam{};
  float pose[12]{};
  float* target = nullptr;       // pinned copy of a train target (from the session's pool), or the caller's
  size_t target_bytes = 0;
  bool target_borrowed = false;  // the caller's pinned target (not the pool's)
  float* image_out = nullptr;
  double arrival = 0.0;
  double done_at = 0.0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  gs_status status = GS_OK;
};

struct Dev {
  void* p = nullptr;
  size_t bytes = 0;
};

// Device and pinned buffers of one batch in flight.
struct Ctx {
  cudaEvent_t done = nullptr;
  cudaStream_t rs = nullptr;     // stream of the batch's render part
  cudaEvent_t rdone = nullptr;   // the render part's last work
  double issued_at = 0.0;
  bool dead = false;             // lost its pair buffers (allocation failure): never used again
  Dev splat_buf, pair_off, ranges, order, counts, vals, ws_bin, ws_bwd, img, tgt, loss, poses, dpose;
  float* h_img = nullptr;       // pinned staging of rendered images
  float* h_poses = nullptr;     // pinned poses [2][max views][12]
  uint32_t* h_counts = nullptr; // pinned [8]: counts of the render and train sub-batches
  int64_t pair_cap = 0;
  size_t bytes = 0;             // device bytes held
  std::vector<std::shared_ptr<Req>> reqs;
  bool busy = false;
  bool has_train = false;
};

}  // namespace
}  // namespace gs

struct gs_session {
  gs_session_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  gs::Dev arena[4];  // parameters, gradients, first and second moments (stride = capacity)
  gs::Dev status_word, step_dev;
  // progressive hierarchy (cfg.lod): leaf rows [0, max_gaussians), merged
  // nodes appended from row max_gaussians on; two active-set buffers: renders
  // and trains read the front one while an analysis writes the other
  gs::Dev h_parent, h_child, h_active[2], h_n, h_info, h_ws, h_pose;
  int front = 0;
  bool h_pending = false;       // an analysis was issued; its buffer becomes the front when it completes
  cudaEvent_t h_done = nullptr;
  uint32_t* h_read = nullptr;   // pinned [8]: summary words of the pending analysis (node rows first)
  float* h_pose_host = nullptr; // pinned [12]
  int64_t h_rows = 0;           // node rows in use after the last swap
  gs::Dev kf_of;               // int32 [arena rows]: keyframe that added each Gaussian (-1: none)
  gs::Dev sim3, sim3_status;   // loop-closure corrections [num_kf][8], status word
  cudaEvent_t mut_done = nullptr;  // the last write of the parameters issued (session stream)
  int64_t fail_allocs = 0;     // host-side fault injection: device allocations still to fail
  int64_t train_beside_render = 0;  // train parts issued while a render part was in flight
  int32_t keyframe = -1;       // tag of the Gaussians added next
  int64_t lod_builds = 0;      // hierarchy analyses completed (their buffers swapped in)
  int64_t capacity = 0;
  int64_t n_active = 0;
  int nc = 1;
  size_t fixed_bytes = 0, ctx_bytes = 0, in_use = 0;
  std::vector<std::unique_ptr<gs::Ctx>> ctxs;
  float* h_add = nullptr;  // pinned staging of added Gaussians
  int64_t h_add_cap = 0;
  cudaEvent_t add_done = nullptr;
  std::mutex add_mu;       // serialises adds (one staging buffer)
  // pinned buffers for train targets, recycled by size once a request ends
  std::mutex pool_mu;
  std::multimap<size_t, float*> pinned_free;
  std::vector<float*> pinned_all;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_ctx;
  std::deque<std::shared_ptr<gs::Req>> queue;
  std::deque<gs::Ctx*> inflight;
  std::vector<std::shared_ptr<gs::Req>> all;  // index = id - 1
  std::vector<double> latencies;
  int64_t iterations = 0, batches = 0, retries = 0, completed = 0, failed = 0;
  double pixels = 0.0, created_at = 0.0;
  bool stop = false;
  bool hold = false;  // admission paused: requests queue up, no batch is formed
  gs_status fatal = GS_OK;
  std::thread worker, completer;
};

namespace gs {
namespace {

constexpr double kWaitTimeout = 30.0;  // seconds a batch may take before the session gives up

size_t arena_floats(int64_t cap, int nc) { return (size_t)(12 + 3 * nc) * (size_t)cap; }

int64_t max_pixels(const gs_session_config& c) { return (int64_t)c.max_width * c.max_height; }
int64_t max_tiles(const gs_session_config& c) {
  const int tw = c.raster.tile_w, th = c.raster.tile_h;
  return (int64_t)((c.max_width + tw - 1) / tw) * ((c.max_height + th - 1) / th);
}

// Device bytes of one batch context at a given pair capacity.
size_t ctx_device_bytes(const gs_session_config& c, int64_t cap_n, int64_t pair_cap) {
  const int64_t V = c.max_batch_views;
  size_t b = 0;
  auto add = [&](size_t x) { b += align_up(std::max<size_t>(x, 16), 256); };
  add(gs_splats_bytes(cap_n, (int32_t)V));
  add(4 * (size_t)cap_n * V);                     // pair_off
  add(8 * (size_t)max_tiles(c) * V);              // ranges
  add(4 * (size_t)max_tiles(c) * V);              // tile order
  add(32);                                        // counts of both sub-batches
  add(4 * (size_t)pair_cap);                      // vals
  add(bin_sort_workspace_bytes(cap_n * V, pair_cap));
  add(gs_render_fused_workspace(cap_n, (int32_t)V, pair_cap, max_tiles(c) * V));
  add(12 * (size_t)max_pixels(c) * V);            // images
  add(12 * (size_t)max_pixels(c) * V);            // targets
  add(8);                                         // loss
  add(48 * 2 * (size_t)V);                        // poses
  add(24 * (size_t)V);                            // pose gradient
  return b;
}

// Rows of the parameter arenas: the leaves, and with a hierarchy its coarse
// nodes after them.
int64_t arena_rows(const gs_session_config& c) {
  return c.lod ? 2 * c.max_gaussians : c.max_gaussians;  // merged nodes: fewer than the leaves
}

size_t fixed_device_bytes(const gs_session_config& c) {
  const int nc = (c.sh_degree + 1) * (c.sh_degree + 1);
  size_t b = 4 * align_up(4 * arena_floats(arena_rows(c), nc), 256) + 2 * 256;
  if (c.lod) {
    const size_t r = (size_t)arena_rows(c);
    b += align_up(4 * r, 256) + align_up(16 * r, 256) + 2 * align_up(r, 256) + align_up(hier_workspace_bytes(r), 256) +
         3 * 256;
  }
  b += align_up(4 * (size_t)arena_rows(c), 256);  // keyframe tags
  return b;
}

int64_t initial_pair_cap(const gs_session_config& c) {
  const double f = c.pair_factor > 0.0 ? c.pair_factor : 4.0;
  return std::max<int64_t>(4096, (int64_t)(f * (double)c.max_gaussians));
}

gs_status dalloc(Dev& d, size_t bytes, size_t& counter, int64_t* fail_next = nullptr) {
  d.bytes = align_up(std::max<size_t>(bytes, 16), 256);
  if (fail_next && *fail_next > 0) {  // injected failure (tests): as if the device were out of memory
    --*fail_next;
    d.p = nullptr;
    d.bytes = 0;
    return fail(GS_ERR_OOM, "session: device allocation of %zu bytes failed (injected)", align_up(bytes, 256));
  }
  if (cudaMalloc(&d.p, d.bytes) != cudaSuccess) {
    cudaGetLastError();
    d.p = nullptr;
    return fail(GS_ERR_OOM, "session: cudaMalloc of %zu bytes failed", d.bytes);
  }
  counter += d.bytes;
  return GS_OK;
}

void dfree(Dev& d, size_t& counter) {
  if (d.p) {
    cudaFree(d.p);
    counter -= d.bytes;
  }
  d.p = nullptr;
  d.bytes = 0;
}

void free_pair_buffers(gs_session* S, Ctx& c) {
  dfree(c.vals, S->in_use);
  dfree(c.ws_bin, S->in_use);
  dfree(c.ws_bwd, S->in_use);
}

size_t fused_ws_bytes(gs_session* S, int64_t pair_cap) {
  const int64_t V = S->cfg.max_batch_views;
  return gs_render_fused_workspace(S->capacity, (int32_t)V, pair_cap, max_tiles(S->cfg) * V);
}

// All three or none: on failure nothing stays allocated.
gs_status alloc_pair_buffers(gs_session* S, Ctx& c, int64_t pair_cap) {
  const auto& cf = S->cfg;
  const int64_t V = cf.max_batch_views;
  gs_status st;
  if ((st = dalloc(c.vals, 4 * (size_t)pair_cap, S->in_use, &S->fail_allocs)) == GS_OK &&
      (st = dalloc(c.ws_bin, bin_sort_workspace_bytes(S->capacity * V, pair_cap), S->in_use, &S->fail_allocs)) ==
          GS_OK &&
      (st = dalloc(c.ws_bwd, fused_ws_bytes(S, pair_cap), S->in_use, &S->fail_allocs)) == GS_OK) {
    c.pair_cap = pair_cap;
    return GS_OK;
  }
  free_pair_buffers(S, c);
  c.pair_cap = 0;
  return st;
}

gs_status alloc_ctx(gs_session* S, Ctx& c) {
  const auto& cf = S->cfg;
  const int64_t V = cf.max_batch_views, px = max_pixels(cf);
  size_t& u = S->in_use;
  int64_t* fa = &S->fail_allocs;
  gs_status st;
  if ((st = dalloc(c.splat_buf, gs_splats_bytes(S->capacity, (int32_t)V), u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.pair_off, 4 * (size_t)S->capacity * V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.ranges, 8 * (size_t)max_tiles(cf) * V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.order, 4 * (size_t)max_tiles(cf) * V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.counts, 32, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.img, 12 * (size_t)px * V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.tgt, 12 * (size_t)px * V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.loss, 8, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.poses, 48 * 2 * (size_t)V, u, fa)) != GS_OK) return st;
  if ((st = dalloc(c.dpose, 24 * (size_t)V, u, fa)) != GS_OK) return st;
  if ((st = alloc_pair_buffers(S, c, initial_pair_cap(cf))) != GS_OK) return st;
  if (cudaStreamCreateWithFlags(&c.rs, cudaStreamNonBlocking) != cudaSuccess) return check_launch("stream");
  if (cudaEventCreateWithFlags(&c.rdone, cudaEventDisableTiming) != cudaSuccess) return check_launch("event");
  if (cudaMallocHost(&c.h_img, 12 * (size_t)px * V) != cudaSuccess ||
      cudaMallocHost(&c.h_poses, 48 * 2 * (size_t)V) != cudaSuccess ||
      cudaMallocHost(&c.h_counts, 32) != cudaSuccess) {
    cudaGetLastError();
    return fail(GS_ERR_OOM, "session: pinned host allocation failed");
  }
  if (cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) return check_launch("event");
  return GS_OK;
}

void free_ctx(gs_session* S, Ctx& c) {
  Dev* devs[] = {&c.splat_buf, &c.pair_off, &c.ranges, &c.order, &c.counts, &c.vals, &c.ws_bin, &c.ws_bwd, &c.img,
                 &c.tgt, &c.loss, &c.poses, &c.dpose};
  for (Dev* d : devs) dfree(*d, S->in_use);
  if (c.h_img) cudaFreeHost(c.h_img);
  if (c.h_poses) cudaFreeHost(c.h_poses);
  if (c.h_counts) cudaFreeHost(c.h_counts);
  if (c.done) cudaEventDestroy(c.done);
  if (c.rdone) cudaEventDestroy(c.rdone);
  if (c.rs) cudaStreamDestroy(c.rs);
  c = Ctx();
}

void free_hier(gs_session* S) {
  for (Dev* d : {&S->h_parent, &S->h_child, &S->h_active[0], &S->h_active[1], &S->h_n, &S->h_info, &S->h_ws,
                 &S->h_pose})
    dfree(*d, S->in_use);
  if (S->h_done) cudaEventDestroy(S->h_done);
  if (S->h_read) cudaFreeHost(S->h_read);
  if (S->h_pose_host) cudaFreeHost(S->h_pose_host);
  S->h_done = nullptr;
  S->h_read = nullptr;
  S->h_pose_host = nullptr;
}

float* arena_ptr(gs_session* S, int k) { return static_cast<float*>(S->arena[k].p); }

gs_params params_of(gs_session* S, int k) {
  float* a = arena_ptr(S, k);
  const int64_t cap = S->capacity;
  gs_params p;
  p.means4 = a;
  p.scale_opa = a + 4 * cap;
  p.quat = a + 8 * cap;
  p.sh = a + 12 * cap;
  p.n = S->n_active;
  p.sh_degree = S->cfg.sh_degree;
  p.sh_stride = cap;
  return p;
}

void wait_renders(gs_session* S, cudaStream_t s);
void mark_write(gs_session* S);

// Adam groups over the rows in use of the capacity-strided arena: the active
// leaf slots and, with a hierarchy, the merged nodes (rows from
// max_gaussians on).
int adam_groups(gs_session* S, gs_adam_group* g) {
  const auto& c = S->cfg;
  const int64_t cap = S->capacity;
  int k = 0;
  auto set = [&](int64_t b, int64_t e, float l0, float l1, float l2, float l3) {
    g[k].begin = b; g[k].end = e;
    g[k].lr[0] = l0; g[k].lr[1] = l1; g[k].lr[2] = l2; g[k].lr[3] = l3;
    ++k;
  };
  auto rows = [&](int64_t r0, int64_t r1) {
    if (r1 <= r0) return;
    set(4 * r0, 4 * r1, c.lr_means, c.lr_means, c.lr_means, 0.f);
    set(4 * cap + 4 * r0, 4 * cap + 4 * r1, c.lr_scale, c.lr_scale, c.lr_scale, c.lr_opacity);
    set(8 * cap + 4 * r0, 8 * cap + 4 * r1, c.lr_quat, c.lr_quat, c.lr_quat, c.lr_quat);
    for (int p = 0; p < 3 * S->nc; ++p) {
      const float lr = (p % S->nc == 0) ? c.lr_sh_dc : c.lr_sh_rest;
      const int64_t b = 12 * cap + (int64_t)p * cap;
      set(b + r0, b + r1, lr, lr, lr, lr);
    }
  };
  // with a hierarchy, one range over the leaf slots and the merged nodes:
  // the unused leaf slots between them have zero gradients and moments, so
  // their update is zero (two ranges would need more groups than allowed)
  rows(0, c.lod ? S->h_rows : S->n_active);
  return k;
}

gs_hier hier_of(gs_session* S, int buf) {
  gs_hier h;
  h.parent = static_cast<int32_t*>(S->h_parent.p);
  h.child = static_cast<int32_t*>(S->h_child.p);
  h.active = static_cast<uint8_t*>(S->h_active[buf].p);
  h.n_nodes = static_cast<uint32_t*>(S->h_n.p);
  h.info = static_cast<uint32_t*>(S->h_info.p);
  h.capacity = S->capacity;
  return h;
}

// At a swap: the Adam moments of the rows whose active flag changed are zeroed
// (a node entering or leaving the active set starts afresh), and every new
// merged node takes the keyframe tag most common among its children (ties:
// the first child's), so a loop closure moves it with them.
__global__ void k_hier_swap(const uint8_t* __restrict__ before, const uint8_t* __restrict__ after, int64_t rows,
                            int64_t new_from, const int32_t* __restrict__ child, int32_t* __restrict__ kf, float* m,
                            float* v, int64_t cap, int nc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  if (before[i] != after[i]) {
    for (float* A : {m, v}) {
      reinterpret_cast<float4*>(A)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(A + 4 * cap)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(A + 8 * cap)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int p = 0; p < 3 * nc; ++p) A[12 * cap + (int64_t)p * cap + i] = 0.f;
    }
  }
  if (i >= new_from) {
    int32_t best = -1;
    int bc = 0;
    for (int a = 0; a < 4; ++a) {
      const int32_t ca = child[4 * i + a];
      if (ca < 0) continue;
      int cnt = 0;
      for (int b = 0; b < 4; ++b)
        if (child[4 * i + b] >= 0 && kf[child[4 * i + b]] == kf[ca]) ++cnt;
      if (cnt > bc) {
        bc = cnt;
        best = kf[ca];
      }
    }
    kf[i] = best;
  }
}

// The pending analysis's buffer becomes the front one once it has completed
// (S->mu held).  Its swap work is a write on the session stream.
void try_swap(gs_session* S) {
  if (!S->h_pending) return;
  const cudaError_t e = cudaEventQuery(S->h_done);
  if (e == cudaErrorNotReady) return;
  S->h_pending = false;
  if (e != cudaSuccess) {
    cudaGetLastError();
    S->fatal = fail(GS_ERR_CUDA, "session: hierarchy analysis failed: %s", cudaGetErrorString(e));
    return;
  }
  const int back = S->front ^ 1;
  const int64_t rows = std::min<int64_t>(S->capacity, (int64_t)S->h_read[0]);
  const unsigned grid = (unsigned)std::max<int64_t>(1, (rows + 255) / 256);
  k_hier_swap<<<grid, 256, 0, S->stream>>>(static_cast<const uint8_t*>(S->h_active[S->front].p),
                                           static_cast<const uint8_t*>(S->h_active[back].p), rows, S->h_rows,
                                           static_cast<const int32_t*>(S->h_child.p),
                                           static_cast<int32_t*>(S->kf_of.p), arena_ptr(S, 2), arena_ptr(S, 3),
                                           S->capacity, S->nc);
  mark_write(S);
  S->front = back;
  S->h_rows = rows;
  S->lod_builds++;
}

// The session stream waits, on the device, for every render part issued so
// far (a write must not change what they read).
void wait_renders(gs_session* S, cudaStream_t s) {
  for (auto& c : S->ctxs)
    if (c->rdone) cudaStreamWaitEvent(s, c->rdone, 0);
}

// A write of the parameters was issued on the session stream: later render
// parts wait for it.
void mark_write(gs_session* S) { cudaEventRecord(S->mut_done, S->stream); }

// Enqueue one batch: its render part on the context's stream, its train part
// on the session stream (S->mu held).
gs_status issue_batch(gs_session* S, Ctx& c) {
  cudaStream_t s = S->stream;
  const auto& cf = S->cfg;
  const int64_t n = S->n_active;
  std::vector<Req*> R, T;
  std::vector<gs_camera> cR, cT;
  for (auto& r : c.reqs) {
    if (r->kind == GS_REQUEST_TRAIN) { T.push_back(r.get()); cT.push_back(r->cam); }
    else { R.push_back(r.get()); cR.push_back(r->cam); }
  }
  c.has_train = !T.empty();
  c.issued_at = steady_now();
  gs_params P = params_of(S, 0);
  uint32_t* counts = static_cast<uint32_t*>(c.counts.p);
  float* img = static_cast<float*>(c.img.p);
  float* poses = static_cast<float*>(c.poses.p);
  const int V = cf.max_batch_views;
  const int tw = cf.raster.tile_w, th = cf.raster.tile_h;
  gs_status st;
  int64_t off = 0;
  if (!R.empty()) {
    GS_NVTX("session render part");
    cudaStream_t rs = c.rs;
    ViewTable vt;
    if (!make_view_table(cR.data(), (int)R.size(), &vt, tw, th)) return GS_ERR_INVALID;
    for (size_t i = 0; i < R.size(); ++i) std::memcpy(c.h_poses + 12 * i, R[i]->pose, 48);
    if (cudaMemcpyAsync(poses, c.h_poses, 48 * R.size(), cudaMemcpyHostToDevice, rs) != cudaSuccess)
      return check_launch("session poses");
    gs_params PR = P;
    gs_hier hf;
    if (cf.lod) {
      // every node row in use (the render cut does not read the active set)
      PR.n = S->h_rows;
      hf = hier_of(S, S->front);
    }
    // every write issued before this render part
    if (cudaStreamWaitEvent(rs, S->mut_done, 0) != cudaSuccess) return check_launch("session wait");
    gs_splats sp;
    gs_splats_carve(c.splat_buf.p, PR.n, (int32_t)R.size(), &sp);
    gs_bins b{static_cast<uint32_t*>(c.vals.p), static_cast<uint32_t*>(c.ranges.p),
              static_cast<uint32_t*>(c.pair_off.p), nullptr, counts, c.pair_cap, vt.total_tiles,
              static_cast<uint32_t*>(c.order.p)};
    // renders draw the hierarchy's render cut (descent from the roots, Sec. 6.2)
    if ((st = launch_project(PR, poses, vt, cf.raster, sp, rs, nullptr, 0, cf.lod_tau, cf.lod ? &hf : nullptr,
                             true)) != GS_OK)
      return st;
    if ((st = launch_bin_sort(sp, vt, b, c.ws_bin.p, rs)) != GS_OK) return st;
    if ((st = launch_render_fwd(sp, b, vt, cf.raster, img, nullptr, rs)) != GS_OK) return st;
    for (Req* r : R) off += 3 * (int64_t)r->cam.width * r->cam.height;
    if (cudaMemcpyAsync(c.h_img, img, 4 * off, cudaMemcpyDeviceToHost, rs) != cudaSuccess)
      return check_launch("session images");
    if (cudaMemcpyAsync(c.h_counts, counts, 16, cudaMemcpyDeviceToHost, rs) != cudaSuccess)
      return check_launch("session counts");
    if (cudaEventRecord(c.rdone, rs) != cudaSuccess) return check_launch("session event");
  } else {
    std::memset(c.h_counts, 0, 16);
  }
  if (!T.empty()) {
    GS_NVTX("session train part");
    // the render part of this batch (on the context's stream) uses the same
    // splat, pair and workspace buffers: the train part runs after it
    if (!R.empty() && cudaStreamWaitEvent(s, c.rdone, 0) != cudaSuccess) return check_launch("session wait");
    for (auto& o : S->ctxs)
      if (o.get() != &c && o->busy && !o->reqs.empty() && o->reqs.front()->kind == GS_REQUEST_RENDER) {
        S->train_beside_render++;  // its forward and backward run beside that render part
        break;
      }
    ViewTable vt;
    if (!make_view_table(cT.data(), (int)T.size(), &vt, tw, th)) return GS_ERR_INVALID;
    float* tgt = static_cast<float*>(c.tgt.p);
    int64_t tpx = 0;
    for (Req* r : T) {  // straight from each request's pinned copy
      const int64_t k = 3 * (int64_t)r->cam.width * r->cam.height;
      if (cudaMemcpyAsync(tgt + tpx, r->target, 4 * k, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return check_launch("session targets");
      tpx += k;
    }
    for (size_t i = 0; i < T.size(); ++i) std::memcpy(c.h_poses + 12 * (V + i), T[i]->pose, 48);
    float* tposes = poses + 12 * V;
    if (cudaMemcpyAsync(tposes, c.h_poses + 12 * V, 48 * T.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return check_launch("session poses");
    // with a hierarchy the train views render (and train) the cut of the
    // front active set: merged nodes in it are optimised like leaves
    const int64_t rows = cf.lod ? S->h_rows : n;
    gs_params PT = P;
    PT.n = rows;
    gs_hier hf = cf.lod ? hier_of(S, S->front) : gs_hier{};
    gs_splats sp;
    gs_splats_carve(c.splat_buf.p, rows, (int32_t)T.size(), &sp);
    gs_bins b{static_cast<uint32_t*>(c.vals.p), static_cast<uint32_t*>(c.ranges.p),
              static_cast<uint32_t*>(c.pair_off.p), nullptr, counts + 4, c.pair_cap, vt.total_tiles,
              static_cast<uint32_t*>(c.order.p)};
    float* timg = img + off;
    if ((st = launch_project(PT, tposes, vt, cf.raster, sp, s, nullptr, 0, cf.lod_tau, cf.lod ? &hf : nullptr)) !=
        GS_OK)
      return st;
    if ((st = launch_bin_sort(sp, vt, b, c.ws_bin.p, s)) != GS_OK) return st;
    // composite, loss and per-pixel backward in one persistent launch
    float *partials, *pose_partials, *drgb;
    render_bwd_ws_layout(rows, (int32_t)T.size(), c.pair_cap, c.ws_bwd.p, &partials, &pose_partials, &drgb);
    char* wsb = static_cast<char*>(c.ws_bwd.p);
    const size_t bwd_bytes = render_bwd_ws_bytes(rows, (int32_t)T.size(), c.pair_cap);
    gs_raster_cfg rc = cf.raster;
    rc.schedule &= ~GS_SCHED_FUSED_LONGEST_FIRST;  // the session bins without a tile order
    if ((st = launch_render_fused(sp, b, vt, rc, tgt, cf.loss_kind, timg, nullptr, static_cast<float*>(c.loss.p),
                                  partials, reinterpret_cast<float*>(wsb + bwd_bytes + 256),
                                  reinterpret_cast<uint32_t*>(wsb + bwd_bytes), s)) != GS_OK)
      return st;
    gs_params G = params_of(S, 1);
    gs_grads g{const_cast<float*>(G.means4), const_cast<float*>(G.scale_opa), const_cast<float*>(G.quat),
               const_cast<float*>(G.sh), rows, G.sh_degree, G.sh_stride};
    if ((st = launch_project_bwd(PT, tposes, vt, cf.raster, sp, b, partials, g, pose_partials, nullptr, drgb,
                                 s)) != GS_OK)
      return st;
    gs_adam_group groups[GS_MAX_ADAM_GROUPS];
    gs_adam_cfg ac{};
    ac.groups = groups;
    ac.num_groups = adam_groups(S, groups);
    ac.beta1 = cf.beta1; ac.beta2 = cf.beta2; ac.eps = cf.eps;
    ac.status = static_cast<uint32_t*>(S->status_word.p);
    ac.step_dev = static_cast<int32_t*>(S->step_dev.p);
    ac.skip_dev = counts + 6;  // the train sub-batch's bins status: skip on overflow
    const int64_t arena_n = (int64_t)arena_floats(S->capacity, S->nc);
    // the update waits for the render parts issued before it (this batch's included)
    wait_renders(S, s);
    if ((st = launch_adam(arena_ptr(S, 0), arena_ptr(S, 1), arena_ptr(S, 2), arena_ptr(S, 3), arena_n, ac, 0,
                          s)) != GS_OK)
      return st;
    mark_write(S);
    if (cudaMemcpyAsync(c.h_counts + 4, counts + 4, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return check_launch("session counts");
  }
  if (cudaEventRecord(c.done, T.empty() ? c.rs : s) != cudaSuccess) return check_launch("session event");
  return GS_OK;
}

Ctx* free_ctx_of(gs_session* S) {
  for (auto& c : S->ctxs)
    if (!c->busy && !c->dead) return c.get();
  return nullptr;
}

// A pinned buffer of at least `bytes` from the pool (allocated on demand).
float* acquire_pinned(gs_session* S, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(S->pool_mu);
    auto it = S->pinned_free.lower_bound(bytes);
    if (it != S->pinned_free.end() && it->first <= 2 * bytes) {
      float* p = it->second;
      S->pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(S->pool_mu);
  S->pinned_all.push_back(static_cast<float*>(p));
  return static_cast<float*>(p);
}

void release_target(gs_session* S, Req* r) {
  if (!r->target) return;
  if (r->target_borrowed) {  // the caller's memory: nothing to return to the pool
    r->target = nullptr;
    return;
  }
  std::lock_guard<std::mutex> lk(S->pool_mu);
  S->pinned_free.emplace(r->target_bytes, r->target);
  r->target = nullptr;
}

void finish_req(gs_session* S, Req* r, gs_status st) {
  r->done_at = steady_now();
  r->status = st;
  r->state = st == GS_OK ? 2 : 3;
  release_target(S, r);  // the pinned copy of a target is not needed once finished
  if (st == GS_OK) {
    S->completed++;
    S->latencies.push_back(1e3 * (r->done_at - r->arrival));
    S->pixels += (double)r->cam.width * r->cam.height;
  } else {
    S->failed++;
  }
}

void worker_main(gs_session* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // exit only once nothing is queued or in flight: a batch in flight may
    // still send its requests back (pair capacity retry)
    S->cv_work.wait(lk, [&] {
      return (S->stop && S->queue.empty() && S->inflight.empty()) ||
             (!S->queue.empty() && (!S->hold || S->stop) && free_ctx_of(S) != nullptr);
    });
    if (S->queue.empty()) break;  // stop requested and drained
    try_swap(S);  // a completed hierarchy analysis becomes the front active set
    Ctx* c = free_ctx_of(S);
    c->busy = true;
    c->reqs.clear();
    while (!S->queue.empty() && (int)c->reqs.size() < S->cfg.max_batch_views) {
      c->reqs.push_back(S->queue.front());
      S->queue.pop_front();
      c->reqs.back()->state = 1;
    }
    const gs_status st = issue_batch(S, *c);
    if (st != GS_OK) {
      for (auto& r : c->reqs) finish_req(S, r.get(), st);
      c->reqs.clear();
      c->busy = false;
      S->cv_done.notify_all();
      continue;
    }
    S->batches++;
    S->inflight.push_back(c);
    S->cv_done.notify_all();
  }
  S->cv_done.notify_all();
}

void completer_main(gs_session* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_done.wait(lk, [&] { return !S->inflight.empty() || (S->stop && S->queue.empty()); });
    if (S->inflight.empty()) break;
    // the first batch in flight to complete (render-only batches may finish
    // before a train batch issued earlier); a batch still running
    // kWaitTimeout seconds after its issue is given up
    Ctx* c = nullptr;
    cudaError_t e = cudaErrorNotReady;
    for (;;) {
      std::vector<Ctx*> snap(S->inflight.begin(), S->inflight.end());
      lk.unlock();
      double oldest = 1e300;
      Ctx* old_c = nullptr;
      for (Ctx* x : snap) {
        const cudaError_t q = cudaEventQuery(x->done);
        if (q != cudaErrorNotReady) {
          c = x;
          e = q;
          break;
        }
        if (x->issued_at < oldest) { oldest = x->issued_at; old_c = x; }
      }
      if (!c && old_c && steady_now() - oldest > kWaitTimeout) c = old_c;  // e stays NotReady: timeout
      if (c) break;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
    // The render and train parts of a batch have their own tile lists and
    // status: an overflowing part is issued again on its own (a train part
    // that overflowed skipped its update on the device), the other completes.
    uint32_t sr = 0, strn = 0;
    if (e == cudaSuccess) {
      sr = c->h_counts[2];
      strn = c->has_train ? c->h_counts[6] : 0u;
      if (!(sr & 3u)) {  // copy rendered images out before taking the lock
        int64_t off = 0;
        for (auto& r : c->reqs) {
          if (r->kind != GS_REQUEST_RENDER) continue;
          const int64_t k = 3 * (int64_t)r->cam.width * r->cam.height;
          if (r->image_out) std::memcpy(r->image_out, c->h_img + off, 4 * k);
          off += k;
        }
      }
    }
    const bool retry = ((sr | strn) & 1u) != 0, bad_index = ((sr | strn) & 2u) != 0;
    lk.lock();
    S->inflight.erase(std::find(S->inflight.begin(), S->inflight.end(), c));
    if (e == cudaErrorNotReady) {
      S->fatal = GS_ERR_TIMEOUT;
      for (auto& r : c->reqs) finish_req(S, r.get(), GS_ERR_TIMEOUT);
    } else if (e != cudaSuccess) {
      cudaGetLastError();
      S->fatal = GS_ERR_CUDA;
      for (auto& r : c->reqs) finish_req(S, r.get(), GS_ERR_CUDA);
    } else if (bad_index) {
      for (auto& r : c->reqs) {
        const uint32_t part = r->kind == GS_REQUEST_TRAIN ? strn : sr;
        finish_req(S, r.get(), (part & 2u) ? gs::fail(GS_ERR_CUDA, "session: internal index error") : GS_OK);
      }
      if (c->has_train && !(strn & 3u)) S->iterations++;
    } else if (retry) {
      const uint32_t K = std::max(c->h_counts[1], c->has_train ? c->h_counts[5] : 0u);
      const int64_t want = (int64_t)(1.25 * (double)K) + 4096;
      const size_t old = c->vals.bytes + c->ws_bin.bytes + c->ws_bwd.bytes;
      const int64_t V = S->cfg.max_batch_views;
      const size_t grow = align_up(4 * (size_t)want, 256) + bin_sort_workspace_bytes(S->capacity * V, want) +
                          fused_ws_bytes(S, want);
      gs_status st = GS_OK;
      if (S->in_use - old + grow > S->cfg.hbm_budget_bytes) {
        st = fail(GS_ERR_OOM, "session: pair capacity %lld exceeds the HBM budget", (long long)want);
      } else {
        const int64_t old_cap = c->pair_cap;
        free_pair_buffers(S, *c);
        st = alloc_pair_buffers(S, *c, want);
        if (st != GS_OK) {
          // keep the context serving at its old capacity if that still fits
          char msg[512];
          gs_last_error(msg, sizeof(msg));
          if (alloc_pair_buffers(S, *c, old_cap) != GS_OK) c->dead = true;
          st = fail(GS_ERR_OOM, "%s", msg);
        }
      }
      if (c->has_train && !(strn & 1u)) S->iterations++;
      if (st == GS_OK) S->retries++;
      for (auto it = c->reqs.rbegin(); it != c->reqs.rend(); ++it) {
        Req* r = it->get();
        const bool over = ((r->kind == GS_REQUEST_TRAIN ? strn : sr) & 1u) != 0;
        if (!over) {
          finish_req(S, r, GS_OK);
        } else if (st != GS_OK) {
          finish_req(S, r, st);
        } else {
          r->state = 0;  // issued again, ahead of everything queued
          S->queue.push_front(*it);
        }
      }
    } else {
      if (c->has_train) S->iterations++;
      for (auto& r : c->reqs) finish_req(S, r.get(), GS_OK);
    }
    c->reqs.clear();
    c->busy = false;
    if (S->fatal == GS_OK && free_ctx_of(S) == nullptr && S->inflight.empty()) {
      // every context lost its buffers: nothing can be served any more
      S->fatal = fail(GS_ERR_OOM, "session: no batch context left after allocation failures");
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    if (S->fatal != GS_OK) {
      // a batch that does not finish (or a CUDA error) leaves the stream unusable:
      // fail everything queued and stop
      for (auto& r : S->queue) finish_req(S, r.get(), S->fatal);
      S->queue.clear();
      S->stop = true;
      S->cv_work.notify_all();
    }
  }
}

gs_status wait_idle(gs_session* S, std::unique_lock<std::mutex>& lk, int timeout_ms) {
  const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [&] { return S->queue.empty() && S->inflight.empty(); });
  if (!ok) return fail(GS_ERR_TIMEOUT, "session: not idle after %d ms", timeout_ms);
  return S->fatal;
}

gs_status sync_stream(gs_session* S, double timeout_s) {
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return check_launch("event");
  cudaEventRecord(ev, S->stream);
  const double t0 = steady_now();
  cudaError_t e;
  while ((e = cudaEventQuery(ev)) == cudaErrorNotReady) {
    if (steady_now() - t0 > timeout_s) break;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  if (e == cudaErrorNotReady) return fail(GS_ERR_TIMEOUT, "session: stream did not finish");
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, "session: %s", cudaGetErrorString(e));
  return GS_OK;
}

// Waits (bounded) for a pending hierarchy analysis and swaps its buffer in
// (S->mu held).
gs_status finish_analysis(gs_session* S, double timeout_s) {
  if (!S->h_pending) return GS_OK;
  const double t0 = steady_now();
  while (cudaEventQuery(S->h_done) == cudaErrorNotReady) {
    if (steady_now() - t0 > timeout_s) return fail(GS_ERR_TIMEOUT, "session: hierarchy analysis did not finish");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  try_swap(S);  // reads the event's status (an error is fatal)
  return S->fatal;
}

}  // namespace
}  // namespace gs

using gs::Ctx;
using gs::Req;

extern "C" {

double gs_session_now(void) { return gs::steady_now(); }

gs_status gs_session_plan(const gs_session_config* cfg, gs_session_plan_info* out) {
  GS_NVTX("gs_session_plan");
  if (!cfg || !out) return gs::fail(GS_ERR_INVALID, "NULL config or plan");
  if (cfg->max_gaussians <= 0 || cfg->max_gaussians >= (1ll << 31) || cfg->sh_degree < 0 || cfg->sh_degree > 3)
    return gs::fail(GS_ERR_INVALID, "session: bad max_gaussians or sh_degree");
  if (cfg->max_batch_views < 1 || cfg->max_batch_views > GS_MAX_VIEWS)
    return gs::fail(GS_ERR_INVALID, "session: max_batch_views must be 1..%d", GS_MAX_VIEWS);
  if (cfg->max_width <= 0 || cfg->max_height <= 0 || cfg->max_width > 16 * 4096 || cfg->max_height > 16 * 4096)
    return gs::fail(GS_ERR_INVALID, "session: bad maximum resolution");
  if ((uint64_t)gs::arena_rows(*cfg) * (uint64_t)cfg->max_batch_views >= (1ull << 32))
    return gs::fail(GS_ERR_INVALID, "session: max_gaussians * max_batch_views must be < 2^32");
  if (cfg->lod != 0 && cfg->lod != 1) return gs::fail(GS_ERR_INVALID, "session: lod must be 0 or 1");
  if (cfg->lod && !(cfg->lod_tau > 0.f)) return gs::fail(GS_ERR_INVALID, "session: lod_tau must be > 0");
  out->fixed_bytes = gs::fixed_device_bytes(*cfg);
  out->context_bytes = gs::ctx_device_bytes(*cfg, gs::arena_rows(*cfg), gs::initial_pair_cap(*cfg));
  out->initial_pair_capacity = gs::initial_pair_cap(*cfg);
  const uint64_t budget = cfg->hbm_budget_bytes;
  int64_t k = 0;
  if (budget > out->fixed_bytes) k = (int64_t)((budget - out->fixed_bytes) / std::max<size_t>(1, out->context_bytes));
  out->contexts = (int32_t)std::min<int64_t>(k, std::max(1, cfg->max_inflight));
  return out->contexts >= 1 ? GS_OK
                            : gs::fail(GS_ERR_OOM, "session: budget %llu B holds no batch context (fixed %zu B, "
                                                   "context %zu B)",
                                       (unsigned long long)budget, out->fixed_bytes, out->context_bytes);
}

gs_status gs_session_create(const gs_session_config* cfg, gs_session** out) {
  GS_NVTX("gs_session_create");
  if (!out) return gs::fail(GS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  gs_session_plan_info plan;
  gs_status st = gs_session_plan(cfg, &plan);
  if (st != GS_OK) return st;
  if (!gs::tile_shape_ok(cfg->raster.tile_w, cfg->raster.tile_h) || !(cfg->raster.znear > 0.f))
    return gs::fail(GS_ERR_INVALID, "session: raster config needs a 16x16, 32x8 or 8x32 tile and znear > 0");
  if (cfg->loss_kind != 0 && cfg->loss_kind != 1) return gs::fail(GS_ERR_INVALID, "session: loss_kind 0 or 1");
  auto S = std::make_unique<gs_session>();
  S->cfg = *cfg;
  S->nc = (cfg->sh_degree + 1) * (cfg->sh_degree + 1);
  S->capacity = gs::arena_rows(*cfg);
  S->created_at = gs::steady_now();
  cudaGetDevice(&S->device);
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return gs::check_launch("stream");
  auto cleanup = [&](gs_status e) {
    for (auto& c : S->ctxs) gs::free_ctx(S.get(), *c);
    for (auto& a : S->arena) gs::dfree(a, S->in_use);
    gs::dfree(S->status_word, S->in_use);
    gs::dfree(S->step_dev, S->in_use);
    gs::free_hier(S.get());
    gs::dfree(S->kf_of, S->in_use);
    gs::dfree(S->sim3_status, S->in_use);
    if (S->h_add) cudaFreeHost(S->h_add);
    if (S->add_done) cudaEventDestroy(S->add_done);
    if (S->mut_done) cudaEventDestroy(S->mut_done);
    cudaStreamDestroy(S->stream);
    return e;
  };
  if (cudaEventCreateWithFlags(&S->mut_done, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(gs::check_launch("event"));
  const size_t af = gs::arena_floats(S->capacity, S->nc);
  for (auto& a : S->arena) {
    if ((st = gs::dalloc(a, 4 * af, S->in_use)) != GS_OK) return cleanup(st);
    cudaMemsetAsync(a.p, 0, a.bytes, S->stream);
  }
  if ((st = gs::dalloc(S->status_word, 16, S->in_use)) != GS_OK) return cleanup(st);
  if ((st = gs::dalloc(S->step_dev, 16, S->in_use)) != GS_OK) return cleanup(st);
  cudaMemsetAsync(S->status_word.p, 0, 16, S->stream);
  cudaMemsetAsync(S->step_dev.p, 0, 16, S->stream);
  if ((st = gs::dalloc(S->kf_of, 4 * (size_t)S->capacity, S->in_use)) != GS_OK) return cleanup(st);
  if ((st = gs::launch_fill_i32(static_cast<int32_t*>(S->kf_of.p), -1, S->capacity, S->stream)) != GS_OK)
    return cleanup(st);
  if ((st = gs::dalloc(S->sim3_status, 16, S->in_use)) != GS_OK) return cleanup(st);
  cudaMemsetAsync(S->sim3_status.p, 0, 16, S->stream);
  if (cfg->lod) {
    const size_t r = (size_t)S->capacity;
    if ((st = gs::dalloc(S->h_parent, 4 * r, S->in_use)) != GS_OK) return cleanup(st);
    if ((st = gs::dalloc(S->h_child, 16 * r, S->in_use)) != GS_OK) return cleanup(st);
    for (auto& a : S->h_active) {
      if ((st = gs::dalloc(a, r, S->in_use)) != GS_OK) return cleanup(st);
      cudaMemsetAsync(a.p, 0, r, S->stream);
    }
    if ((st = gs::dalloc(S->h_n, 16, S->in_use)) != GS_OK) return cleanup(st);
    if ((st = gs::dalloc(S->h_info, 32, S->in_use)) != GS_OK) return cleanup(st);
    if ((st = gs::dalloc(S->h_pose, 48, S->in_use)) != GS_OK) return cleanup(st);
    if ((st = gs::dalloc(S->h_ws, gs::hier_workspace_bytes(S->capacity), S->in_use)) != GS_OK) return cleanup(st);
    // leaf slots hold no node until Gaussians are added to them (-2)
    if ((st = gs::launch_fill_i32(static_cast<int32_t*>(S->h_parent.p), -2, cfg->max_gaussians, S->stream)) !=
            GS_OK ||
        (st = gs::launch_fill_i32(static_cast<int32_t*>(S->h_parent.p) + cfg->max_gaussians, -1,
                                  S->capacity - cfg->max_gaussians, S->stream)) != GS_OK ||
        (st = gs::launch_fill_i32(static_cast<int32_t*>(S->h_child.p), -1, 4 * S->capacity, S->stream)) != GS_OK)
      return cleanup(st);
    // the leaf slots count as node rows (inactive until added); merged nodes follow
    const uint32_t rows0 = (uint32_t)cfg->max_gaussians;
    cudaMemcpyAsync(S->h_n.p, &rows0, 4, cudaMemcpyHostToDevice, S->stream);
    S->h_rows = cfg->max_gaussians;
    if (cudaEventCreateWithFlags(&S->h_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&S->h_read, 16 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&S->h_pose_host, 12 * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(gs::fail(GS_ERR_OOM, "session: hierarchy event or pinned buffers"));
    }
  }
  for (int k = 0; k < plan.contexts; ++k) {
    S->ctxs.push_back(std::make_unique<Ctx>());
    if ((st = gs::alloc_ctx(S.get(), *S->ctxs.back())) != GS_OK) return cleanup(st);
  }
  S->h_add_cap = 1 << 16;
  if (cudaMallocHost(&S->h_add, sizeof(float) * (12 + 3 * S->nc) * S->h_add_cap) != cudaSuccess)
    return cleanup(gs::fail(GS_ERR_OOM, "session: pinned staging"));
  cudaEventCreateWithFlags(&S->add_done, cudaEventDisableTiming);
  cudaEventRecord(S->add_done, S->stream);
  gs::mark_write(S.get());  // the zeroed arenas
  if ((st = gs::sync_stream(S.get(), 30.0)) != GS_OK) return cleanup(st);
  gs_session* raw = S.release();
  raw->worker = std::thread(gs::worker_main, raw);
  raw->completer = std::thread(gs::completer_main, raw);
  *out = raw;
  return GS_OK;
}

gs_status gs_session_add_gaussians(gs_session* S, int64_t count, const float* means, const float* log_scales,
                                   const float* quats, const float* opa_logits, const float* sh) {
  GS_NVTX("gs_session_add_gaussians");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  if (count < 0) return gs::fail(GS_ERR_INVALID, "count < 0");
  if (count == 0) return GS_OK;
  if (!means || !log_scales || !quats || !opa_logits || !sh) return gs::fail(GS_ERR_INVALID, "NULL array");
  // Adds are serialised; the host-side staging runs without the session lock,
  // the device copies are enqueued under it together with the new count (so
  // a batch never sees rows that are being filled).
  std::lock_guard<std::mutex> add_lk(S->add_mu);
  int64_t n0;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->fatal != GS_OK) return gs::fail(S->fatal, "session failed earlier");
    if (S->n_active + count > S->cfg.max_gaussians)
      return gs::fail(GS_ERR_OOM, "session: %lld + %lld Gaussians exceed the capacity %lld",
                      (long long)S->n_active, (long long)count, (long long)S->cfg.max_gaussians);
    n0 = S->n_active;  // only adds change it, and they are serialised
  }
  const int nc = S->nc;
  const int64_t cap = S->capacity;
  // the staging buffer is free once the previous add's copies finished
  const double t0 = gs::steady_now();
  cudaError_t e;
  while ((e = cudaEventQuery(S->add_done)) == cudaErrorNotReady) {
    if (gs::steady_now() - t0 > 30.0) return gs::fail(GS_ERR_TIMEOUT, "session: add staging busy");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  if (e != cudaSuccess) return gs::fail(GS_ERR_CUDA, "session: %s", cudaGetErrorString(e));
  if (count > S->h_add_cap) {
    cudaFreeHost(S->h_add);
    S->h_add = nullptr;
    if (cudaMallocHost(&S->h_add, sizeof(float) * (12 + 3 * nc) * count) != cudaSuccess) {
      cudaGetLastError();
      S->h_add_cap = 0;
      return gs::fail(GS_ERR_OOM, "session: pinned staging of %lld Gaussians", (long long)count);
    }
    S->h_add_cap = count;
  }
  const int64_t k = count;
  float* h = S->h_add;
  float* hm = h;
  float* hs = h + 4 * k;
  float* hq = h + 8 * k;
  float* hsh = h + 12 * k;
  // Gaussian by Gaussian (the source read in order; a plane-by-plane sweep
  // re-read it once per plane, 3x slower at 50k Gaussians), in ranges of
  // Gaussians on several threads
  gs::host_parallel(k, 2048, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      hm[4 * i] = means[3 * i]; hm[4 * i + 1] = means[3 * i + 1]; hm[4 * i + 2] = means[3 * i + 2];
      hm[4 * i + 3] = 0.f;
      hs[4 * i] = log_scales[3 * i]; hs[4 * i + 1] = log_scales[3 * i + 1]; hs[4 * i + 2] = log_scales[3 * i + 2];
      hs[4 * i + 3] = opa_logits[i];
      for (int c = 0; c < 4; ++c) hq[4 * i + c] = quats[4 * i + c];
      const float* src = sh + i * 3 * nc;
      for (int p = 0; p < 3 * nc; ++p) hsh[(int64_t)p * k + i] = src[p];
    }
  });
  std::unique_lock<std::mutex> lk(S->mu);
  float* A = gs::arena_ptr(S, 0);
  cudaStream_t s = S->stream;
  gs::wait_renders(S, s);  // the active flags change under render parts issued earlier
  cudaMemcpyAsync(A + 4 * n0, hm, 16 * k, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(A + 4 * cap + 4 * n0, hs, 16 * k, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(A + 8 * cap + 4 * n0, hq, 16 * k, cudaMemcpyHostToDevice, s);
  cudaMemcpy2DAsync(A + 12 * cap + n0, 4 * cap, hsh, 4 * k, 4 * k, 3 * nc, cudaMemcpyHostToDevice, s);
  for (int a = 2; a < 4; ++a) {  // fresh Adam moments for the new slots
    float* M = gs::arena_ptr(S, a);
    cudaMemsetAsync(M + 4 * n0, 0, 16 * k, s);
    cudaMemsetAsync(M + 4 * cap + 4 * n0, 0, 16 * k, s);
    cudaMemsetAsync(M + 8 * cap + 4 * n0, 0, 16 * k, s);
    cudaMemset2DAsync(M + 12 * cap + n0, 4 * cap, 0, 4 * k, 3 * nc, s);
  }
  gs_status st = gs::launch_fill_i32(static_cast<int32_t*>(S->kf_of.p) + n0, S->keyframe, k, s);
  if (st != GS_OK) return st;
  if (S->cfg.lod) {  // new leaves: roots, active in both buffers (the pending analysis did not see them)
    st = gs::launch_fill_i32(static_cast<int32_t*>(S->h_parent.p) + n0, -1, k, s);
    if (st != GS_OK) return st;
    for (auto& a : S->h_active) cudaMemsetAsync(static_cast<uint8_t*>(a.p) + n0, 1, (size_t)k, s);
  }
  cudaEventRecord(S->add_done, s);
  gs::mark_write(S);
  st = gs::check_launch("session add");
  if (st != GS_OK) return st;
  S->n_active += count;
  return GS_OK;
}

gs_status gs_session_set_keyframe(gs_session* S, int32_t kf) {
  GS_NVTX("gs_session_set_keyframe");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  std::lock_guard<std::mutex> add_lk(S->add_mu);
  S->keyframe = kf < 0 ? -1 : kf;
  return GS_OK;
}

gs_status gs_session_loop_closure(gs_session* S, int32_t num_kf, const float* sim3) {
  GS_NVTX("gs_session_loop_closure");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  if (num_kf < 0 || (num_kf > 0 && !sim3)) return gs::fail(GS_ERR_INVALID, "bad corrections");
  for (int32_t k = 0; k < num_kf; ++k)
    if (!(sim3[8 * k + 7] > 0.f)) return gs::fail(GS_ERR_INVALID, "keyframe %d: scale must be > 0", k);
  std::lock_guard<std::mutex> add_lk(S->add_mu);
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal != GS_OK) return gs::fail(S->fatal, "session failed earlier");
  const size_t bytes = 32 * (size_t)std::max(1, num_kf);
  if (S->sim3.bytes < bytes) {
    // the corrections of an earlier closure may still be read by the stream
    gs_status st = gs::sync_stream(S, 30.0);
    if (st != GS_OK) return st;
    gs::dfree(S->sim3, S->in_use);
    if ((st = gs::dalloc(S->sim3, bytes, S->in_use)) != GS_OK) return st;
  }
  cudaStream_t s = S->stream;
  gs::wait_renders(S, s);  // the update moves what render parts issued earlier read
  if (num_kf > 0 && cudaMemcpyAsync(S->sim3.p, sim3, 32 * (size_t)num_kf, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return gs::check_launch("session sim3");
  gs_params P = gs::params_of(S, 0);
  // every row in use: leaves and merged nodes (tagged with their children's keyframe)
  gs_grads rw{const_cast<float*>(P.means4), const_cast<float*>(P.scale_opa), const_cast<float*>(P.quat),
              const_cast<float*>(P.sh), S->cfg.lod ? S->h_rows : S->n_active, P.sh_degree, P.sh_stride};
  gs_status st = gs::launch_sim3_update(rw, static_cast<const int32_t*>(S->kf_of.p),
                                        static_cast<const float*>(S->sim3.p), num_kf,
                                        static_cast<uint32_t*>(S->sim3_status.p), s);
  if (st != GS_OK) return st;
  gs::mark_write(S);
  return GS_OK;
}

gs_status gs_session_keyframe_weights(gs_session* S, int32_t num_kf, int32_t min_keep, float frac, double* p_out,
                                      uint32_t* counts_out, uint8_t* kept_out) {
  GS_NVTX("gs_session_keyframe_weights");
  if (!S || !p_out) return gs::fail(GS_ERR_INVALID, "NULL session or output");
  if (num_kf <= 0 || min_keep < 0 || !(frac >= 0.f && frac <= 1.f))
    return gs::fail(GS_ERR_INVALID, "bad num_kf, min_keep or frac");
  std::vector<uint32_t> c((size_t)num_kf);
  {
    std::lock_guard<std::mutex> add_lk(S->add_mu);
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->fatal != GS_OK) return gs::fail(S->fatal, "session failed earlier");
    gs::Dev counts;
    gs_status st = gs::dalloc(counts, sizeof(uint32_t) * (size_t)num_kf, S->in_use);
    if (st != GS_OK) return st;
    // after everything enqueued so far (adds, closures), on the session stream
    // the leaf Gaussians (rows [0, n_active)) each keyframe generated that
    // are still in the active set (all of them without a hierarchy)
    st = gs::launch_keyframe_counts(static_cast<const int32_t*>(S->kf_of.p), S->n_active, num_kf,
                                    static_cast<uint32_t*>(counts.p), S->stream,
                                    S->cfg.lod ? static_cast<const uint8_t*>(S->h_active[S->front].p) : nullptr);
    if (st == GS_OK &&
        cudaMemcpyAsync(c.data(), counts.p, sizeof(uint32_t) * (size_t)num_kf, cudaMemcpyDeviceToHost, S->stream) !=
            cudaSuccess)
      st = gs::check_launch("keyframe counts");
    if (st == GS_OK) st = gs::sync_stream(S, 30.0);
    gs::dfree(counts, S->in_use);
    if (st != GS_OK) return st;
  }
  // Sec. 6.2: probability proportional to the leaf count; keyframes below
  // frac of the largest count are offloaded, but the min_keep largest stay
  uint32_t cmax = 0;
  for (uint32_t v : c) cmax = std::max(cmax, v);
  std::vector<uint8_t> kept((size_t)num_kf, 0);
  for (int32_t k = 0; k < num_kf; ++k) kept[k] = cmax > 0 && (double)c[k] >= (double)frac * (double)cmax;
  std::vector<int32_t> order((size_t)num_kf);
  for (int32_t k = 0; k < num_kf; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return c[a] > c[b]; });
  for (int32_t i = 0; i < std::min(min_keep, num_kf); ++i) kept[order[i]] = 1;
  double total = 0;
  for (int32_t k = 0; k < num_kf; ++k)
    if (kept[k]) total += c[k];
  for (int32_t k = 0; k < num_kf; ++k) {
    p_out[k] = (kept[k] && total > 0) ? c[k] / total : 0.0;
    if (counts_out) counts_out[k] = c[k];
    if (kept_out) kept_out[k] = kept[k];
  }
  return GS_OK;
}

gs_status gs_session_submit(gs_session* S, const gs_request* req, int64_t* id) {
  GS_NVTX("gs_session_submit");
  if (!S || !req) return gs::fail(GS_ERR_INVALID, "NULL session or request");
  if (req->kind != GS_REQUEST_RENDER && req->kind != GS_REQUEST_TRAIN)
    return gs::fail(GS_ERR_INVALID, "request kind must be render or train");
  const gs_camera& c = req->cam;
  if (c.width <= 0 || c.height <= 0 || c.width > S->cfg.max_width || c.height > S->cfg.max_height ||
      !(c.fx > 0.f) || !(c.fy > 0.f))
    return gs::fail(GS_ERR_INVALID, "request camera %dx%d outside the session limits %dx%d", c.width, c.height,
                    S->cfg.max_width, S->cfg.max_height);
  if (req->kind == GS_REQUEST_TRAIN && !req->target) return gs::fail(GS_ERR_INVALID, "train request needs a target");
  if (req->flags & ~GS_REQUEST_BORROW_TARGET) return gs::fail(GS_ERR_INVALID, "unknown request flags %d", req->flags);
  auto r = std::make_shared<Req>();
  r->kind = req->kind;
  r->cam = c;
  std::memcpy(r->pose, req->pose, sizeof(r->pose));
  r->image_out = req->image_out;
  r->arrival = req->arrival_s > 0.0 ? req->arrival_s : gs::steady_now();
  if (req->kind == GS_REQUEST_TRAIN) {
    r->target_bytes = sizeof(float) * 3 * (size_t)c.width * c.height;
    if (req->flags & GS_REQUEST_BORROW_TARGET) {
      r->target = const_cast<float*>(req->target);
      r->target_borrowed = true;
    } else {
      r->target = gs::acquire_pinned(S, r->target_bytes);
      if (!r->target) return gs::fail(GS_ERR_OOM, "session: pinned host memory for a target");
      char* dst = reinterpret_cast<char*>(r->target);
      const char* src = reinterpret_cast<const char*>(req->target);
      gs::host_parallel((int64_t)r->target_bytes, (int64_t)1 << 20,
                        [&](int64_t lo, int64_t hi) { std::memcpy(dst + lo, src + lo, (size_t)(hi - lo)); });
    }
  }
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal != GS_OK || S->stop) {
    gs::release_target(S, r.get());
    if (S->fatal != GS_OK) return gs::fail(S->fatal, "session failed earlier");
    return gs::fail(GS_ERR_BUSY, "session is stopping");
  }
  r->id = (int64_t)S->all.size() + 1;
  S->all.push_back(r);
  S->queue.push_back(r);
  if (id) *id = r->id;
  S->cv_work.notify_one();
  return GS_OK;
}

gs_status gs_session_poll(gs_session* S, int64_t id, int32_t* done) {
  GS_NVTX("gs_session_poll");
  if (!S || !done) return gs::fail(GS_ERR_INVALID, "NULL session or output");
  std::unique_lock<std::mutex> lk(S->mu);
  if (id < 1 || id > (int64_t)S->all.size()) return gs::fail(GS_ERR_INVALID, "unknown request id %lld", (long long)id);
  const Req& r = *S->all[id - 1];
  *done = r.state >= 2 ? 1 : 0;
  return r.state == 3 ? r.status : GS_OK;
}

gs_status gs_session_wait(gs_session* S, int64_t id, int32_t timeout_ms) {
  GS_NVTX("gs_session_wait");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (id < 1 || id > (int64_t)S->all.size()) return gs::fail(GS_ERR_INVALID, "unknown request id %lld", (long long)id);
  auto r = S->all[id - 1];
  if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state >= 2; }))
    return gs::fail(GS_ERR_TIMEOUT, "request %lld not done after %d ms", (long long)id, timeout_ms);
  return r->state == 3 ? gs::fail(r->status, "request %lld failed", (long long)id) : GS_OK;
}

gs_status gs_session_times(gs_session* S, int64_t id, double* arrival_s, double* done_s) {
  GS_NVTX("gs_session_times");
  if (!S || !arrival_s || !done_s) return gs::fail(GS_ERR_INVALID, "NULL session or output");
  std::unique_lock<std::mutex> lk(S->mu);
  if (id < 1 || id > (int64_t)S->all.size()) return gs::fail(GS_ERR_INVALID, "unknown request id %lld", (long long)id);
  const Req& r = *S->all[id - 1];
  if (r.state < 2) return GS_ERR_BUSY;
  *arrival_s = r.arrival;
  *done_s = r.done_at;
  return GS_OK;
}

gs_status gs_session_hold(gs_session* S, int32_t on) {
  GS_NVTX("gs_session_hold");
  if (!S) return gs::fail(GS_ERR_INVALID, "NULL session");
  std::lock_guard<std::mutex> lk(S->mu);
  S->hold = on != 0;
  S->cv_work.notify_all();
  return GS_OK;
}

gs_status gs_session_drain(gs_session* S, int32_t timeout_ms) {
  GS_NVTX("gs_session_drain");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_status st = gs::wait_idle(S, lk, timeout_ms);
  if (st != GS_OK) return st;
  return gs::finish_analysis(S, 1e-3 * timeout_ms);
}

gs_status gs_session_stats(gs_session* S, gs_stats* out) {
  GS_NVTX("gs_session_stats");
  if (!S || !out) return gs::fail(GS_ERR_INVALID, "NULL session or stats");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_stats st{};
  st.submitted = (int64_t)S->all.size();
  st.completed = S->completed;
  st.failed = S->failed;
  st.queued = (int64_t)S->queue.size();
  int64_t inflight = 0;
  for (auto* c : S->inflight) inflight += (int64_t)c->reqs.size();
  st.inflight = inflight;
  st.iterations = S->iterations;
  st.batches = S->batches;
  st.retries = S->retries;
  st.lod_builds = S->lod_builds;
  st.gaussians = S->n_active;
  st.pixels = S->pixels;
  st.wall_s = gs::steady_now() - S->created_at;
  st.hbm_in_use = S->in_use;
  st.hbm_budget = S->cfg.hbm_budget_bytes;
  st.contexts = (int32_t)S->ctxs.size();
  st.train_beside_render = S->train_beside_render;
  if (!S->latencies.empty()) {
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      // nearest rank
      const size_t k = (size_t)std::min<double>((double)l.size() - 1, std::ceil(q * (double)l.size()) - 1);
      return l[std::max<size_t>(0, k)];
    };
    st.p50_ms = pct(0.50);
    st.p99_ms = pct(0.99);
    st.max_ms = l.back();
    double s = 0;
    for (double x : l) s += x;
    st.mean_ms = s / (double)l.size();
  }
  *out = st;
  return GS_OK;
}

// Checkpoint: parameters, Adam moments, the step counter and the active count.
gs_status gs_session_save(gs_session* S, const char* path) {
  GS_NVTX("gs_session_save");
  if (!S || !path) return gs::fail(GS_ERR_INVALID, "NULL session or path");
  if (S->cfg.lod) return gs::fail(GS_ERR_INVALID, "session: checkpoints of a session with a hierarchy are not supported");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_status st = gs::wait_idle(S, lk, 60000);
  if (st != GS_OK) return st;
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  const int64_t n = S->n_active, cap = S->capacity;
  const int nc = S->nc;
  int32_t step = 0;
  cudaMemcpyAsync(&step, S->step_dev.p, 4, cudaMemcpyDeviceToHost, S->stream);
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return gs::fail(GS_ERR_INVALID, "cannot open %s", path);
  const int64_t hdr[4] = {0x3153534553534723ll, (int64_t)S->cfg.sh_degree, n, (int64_t)step};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
  std::vector<float> buf((size_t)(12 + 3 * nc) * std::max<int64_t>(n, 1));
  for (int a : {0, 2, 3}) {
    const float* A = gs::arena_ptr(S, a);
    cudaStream_t s = S->stream;
    cudaMemcpyAsync(buf.data(), A, 16 * n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(buf.data() + 4 * n, A + 4 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(buf.data() + 8 * n, A + 8 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
    cudaMemcpy2DAsync(buf.data() + 12 * n, 4 * n, A + 12 * cap, 4 * cap, 4 * n, 3 * nc, cudaMemcpyDeviceToHost, s);
    if ((st = gs::sync_stream(S, 30.0)) != GS_OK) break;
    ok = ok && std::fwrite(buf.data(), sizeof(float), (size_t)(12 + 3 * nc) * n, f) == (size_t)(12 + 3 * nc) * n;
  }
  if (st != GS_OK) {
    std::fclose(f);
    return st;
  }
  ok = (std::fclose(f) == 0) && ok;
  if ((st = gs::check_launch("session save")) != GS_OK) return st;
  return ok ? GS_OK : gs::fail(GS_ERR_INVALID, "write to %s failed", path);
}

gs_status gs_session_load(gs_session* S, const char* path) {
  GS_NVTX("gs_session_load");
  if (!S || !path) return gs::fail(GS_ERR_INVALID, "NULL session or path");
  if (S->cfg.lod) return gs::fail(GS_ERR_INVALID, "session: checkpoints of a session with a hierarchy are not supported");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_status st = gs::wait_idle(S, lk, 60000);
  if (st != GS_OK) return st;
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  FILE* f = std::fopen(path, "rb");
  if (!f) return gs::fail(GS_ERR_INVALID, "cannot open %s", path);
  int64_t hdr[4];
  if (std::fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 0x3153534553534723ll || hdr[1] != S->cfg.sh_degree ||
      hdr[2] < 0 || hdr[2] > S->cfg.max_gaussians) {
    std::fclose(f);
    return gs::fail(GS_ERR_INVALID, "%s is not a checkpoint of this session's layout", path);
  }
  const int64_t n = hdr[2], cap = S->capacity;
  const int nc = S->nc;
  std::vector<float> buf((size_t)(12 + 3 * nc) * std::max<int64_t>(n, 1));
  bool ok = true;
  for (int a : {0, 2, 3}) {
    ok = ok && std::fread(buf.data(), sizeof(float), (size_t)(12 + 3 * nc) * n, f) == (size_t)(12 + 3 * nc) * n;
    if (!ok) break;
    // on the session stream, then waited for: a copy from pageable memory may
    // return before its data lands, and the session stream does not wait for
    // the legacy default stream
    float* A = gs::arena_ptr(S, a);
    cudaStream_t s = S->stream;
    cudaMemcpyAsync(A, buf.data(), 16 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(A + 4 * cap, buf.data() + 4 * n, 16 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(A + 8 * cap, buf.data() + 8 * n, 16 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpy2DAsync(A + 12 * cap, 4 * cap, buf.data() + 12 * n, 4 * n, 4 * n, 3 * nc, cudaMemcpyHostToDevice, s);
    if ((st = gs::sync_stream(S, 30.0)) != GS_OK) break;
  }
  std::fclose(f);
  if (st != GS_OK) return st;
  if (!ok) return gs::fail(GS_ERR_INVALID, "%s is truncated", path);
  const int32_t step = (int32_t)hdr[3];
  cudaMemcpyAsync(S->step_dev.p, &step, 4, cudaMemcpyHostToDevice, S->stream);
  gs::mark_write(S);
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  S->n_active = n;
  return gs::check_launch("session load");
}

gs_status gs_session_read_params(gs_session* S, float* means4, float* scale_opa, float* quat, float* sh) {
  GS_NVTX("gs_session_read_params");
  if (!S) return gs::fail(GS_ERR_INVALID, "session is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_status st = gs::wait_idle(S, lk, 60000);
  if (st != GS_OK) return st;
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  const int64_t n = S->n_active, cap = S->capacity;
  const float* A = gs::arena_ptr(S, 0);
  cudaStream_t s = S->stream;
  if (means4) cudaMemcpyAsync(means4, A, 16 * n, cudaMemcpyDeviceToHost, s);
  if (scale_opa) cudaMemcpyAsync(scale_opa, A + 4 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
  if (quat) cudaMemcpyAsync(quat, A + 8 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
  if (sh) cudaMemcpy2DAsync(sh, 4 * n, A + 12 * cap, 4 * cap, 4 * n, 3 * S->nc, cudaMemcpyDeviceToHost, s);
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  return gs::check_launch("session read");
}

gs_status gs_session_read_hierarchy(gs_session* S, int64_t max_rows, int64_t* rows, float* means4,
                                    float* scale_opa, float* quat, float* sh, int32_t* parent, int32_t* child,
                                    uint8_t* active) {
  GS_NVTX("gs_session_read_hierarchy");
  if (!S || !rows) return gs::fail(GS_ERR_INVALID, "NULL session or rows");
  if (!S->cfg.lod) return gs::fail(GS_ERR_INVALID, "session: no hierarchy (lod = 0)");
  std::unique_lock<std::mutex> lk(S->mu);
  gs_status st = gs::wait_idle(S, lk, 60000);
  if (st != GS_OK) return st;
  if ((st = gs::finish_analysis(S, 30.0)) != GS_OK) return st;
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  const int64_t n = S->h_rows, cap = S->capacity;
  *rows = n;
  const bool any = means4 || scale_opa || quat || sh || parent || child || active;
  if (!any) return GS_OK;
  if (max_rows < n) return gs::fail(GS_ERR_INVALID, "session: %lld node rows, arrays hold %lld", (long long)n,
                                    (long long)max_rows);
  const float* A = gs::arena_ptr(S, 0);
  cudaStream_t s = S->stream;
  if (means4) cudaMemcpyAsync(means4, A, 16 * n, cudaMemcpyDeviceToHost, s);
  if (scale_opa) cudaMemcpyAsync(scale_opa, A + 4 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
  if (quat) cudaMemcpyAsync(quat, A + 8 * cap, 16 * n, cudaMemcpyDeviceToHost, s);
  if (sh) cudaMemcpy2DAsync(sh, 4 * n, A + 12 * cap, 4 * cap, 4 * n, 3 * S->nc, cudaMemcpyDeviceToHost, s);
  if (parent) cudaMemcpyAsync(parent, S->h_parent.p, 4 * n, cudaMemcpyDeviceToHost, s);
  if (child) cudaMemcpyAsync(child, S->h_child.p, 16 * n, cudaMemcpyDeviceToHost, s);
  if (active) cudaMemcpyAsync(active, S->h_active[S->front].p, (size_t)n, cudaMemcpyDeviceToHost, s);
  if ((st = gs::sync_stream(S, 30.0)) != GS_OK) return st;
  return gs::check_launch("session read hierarchy");
}

gs_status gs_session_analyze(gs_session* S, const gs_camera* cam, const float* pose12) {
  GS_NVTX("gs_session_analyze");
  if (!S || !cam || !pose12) return gs::fail(GS_ERR_INVALID, "NULL session, camera or pose");
  if (!S->cfg.lod) return gs::fail(GS_ERR_INVALID, "session: no hierarchy (lod = 0)");
  if (cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
    return gs::fail(GS_ERR_INVALID, "session: bad camera");
  std::lock_guard<std::mutex> add_lk(S->add_mu);
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->fatal != GS_OK) return gs::fail(S->fatal, "session failed earlier");
  gs::try_swap(S);
  if (S->h_pending) return gs::fail(GS_ERR_BUSY, "session: the previous analysis has not completed");
  cudaStream_t s = S->stream;
  const int back = S->front ^ 1;
  // the back buffer may still be read by render parts issued before the last swap
  gs::wait_renders(S, s);
  cudaMemcpyAsync(S->h_active[back].p, S->h_active[S->front].p, (size_t)S->capacity, cudaMemcpyDeviceToDevice, s);
  std::memcpy(S->h_pose_host, pose12, 48);
  cudaMemcpyAsync(S->h_pose.p, S->h_pose_host, 48, cudaMemcpyHostToDevice, s);
  gs_params P = gs::params_of(S, 0);
  gs_grads rw{const_cast<float*>(P.means4), const_cast<float*>(P.scale_opa), const_cast<float*>(P.quat),
              const_cast<float*>(P.sh), S->capacity, P.sh_degree, P.sh_stride};
  gs_hier h = gs::hier_of(S, back);
  const float tau_h = S->cfg.lod_tau, tau_l = 0.5f * S->cfg.lod_tau;
  const float* pose = static_cast<const float*>(S->h_pose.p);
  gs_status st = gs::launch_hier_analyze(rw, h, nullptr, nullptr, pose, *cam, S->cfg.raster.znear, tau_l, S->h_ws.p, s);
  if (st == GS_OK) cudaMemcpyAsync(S->h_read + 1, S->h_info.p, 32, cudaMemcpyDeviceToHost, s);
  // the reload for the same view: nodes too coarse for it go back to their children
  if (st == GS_OK)
    st = gs::launch_hier_refine(rw, h, nullptr, nullptr, pose, *cam, S->cfg.raster.znear, tau_h, 16, S->h_ws.p, s);
  if (st != GS_OK) return st;
  cudaMemcpyAsync(S->h_read, S->h_n.p, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(S->h_read + 9, S->h_info.p, 4, cudaMemcpyDeviceToHost, s);
  if (cudaEventRecord(S->h_done, s) != cudaSuccess) return gs::check_launch("session analysis event");
  S->h_pending = true;
  return gs::check_launch("session analyze");
}

gs_status gs_session_inject_alloc_failures(gs_session* S, int32_t count) {
  GS_NVTX("gs_session_inject_alloc_failures");
  if (!S || count < 0) return gs::fail(GS_ERR_INVALID, "NULL session or count < 0");
  std::lock_guard<std::mutex> lk(S->mu);
  S->fail_allocs = count;
  return GS_OK;
}

gs_status gs_session_destroy(gs_session* S) {
  GS_NVTX("gs_session_destroy");
  if (!S) return GS_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.notify_all();
  }
  if (S->completer.joinable()) S->completer.join();
  gs::sync_stream(S, 30.0);
  for (auto& c : S->ctxs) gs::free_ctx(S, *c);
  for (auto& a : S->arena) gs::dfree(a, S->in_use);
  gs::dfree(S->status_word, S->in_use);
  gs::dfree(S->step_dev, S->in_use);
  gs::free_hier(S);
  gs::dfree(S->kf_of, S->in_use);
  gs::dfree(S->sim3, S->in_use);
  gs::dfree(S->sim3_status, S->in_use);
  if (S->h_add) cudaFreeHost(S->h_add);
  if (S->add_done) cudaEventDestroy(S->add_done);
  for (auto& r : S->all) r->target = nullptr;  // pooled buffers are freed below
  for (float* p : S->pinned_all) cudaFreeHost(p);
  cudaStreamDestroy(S->stream);
  delete S;
  return GS_OK;
}

}  // extern "C"
