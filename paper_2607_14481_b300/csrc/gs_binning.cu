// Tile binning: per-tile duplication of the visible splats and the
// (tile, depth) sort that orders every tile's list front to back, then the
// [start, end) range of each tile.
//
// The 64-bit (global tile << 32 | depth bits) order is produced by two stable
// LSD radix sorts instead of one sort of 64-bit keys:
//   1. the visible (view, Gaussian) items are sorted by their 32-bit depth key
//      (items are compacted in (view, id) order, so equal depths stay in id
//      order);
//   2. every item, in that depth order, emits one pair per tile of its rect;
//      the pairs are sorted stably by global tile id on its significant bits
//      only (12 bits at 720p, 17 for 16 views at 1080p).
// Within one tile the pairs then sit in (depth, id) order: the same result as
// the 64-bit sort, with about a third of the bytes moved.
//
// Every count (visible items, pairs) stays in device memory: kernels are
// launched for the capacity and read the live count, so the whole stage runs
// without a host synchronisation and can be captured in a CUDA graph.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 8;                      // items per thread
constexpr int kItemsPerBlock = kThreads * kIPT;
constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;

__device__ __forceinline__ uint32_t num_blocks(uint32_t n) {
  return (n + kItemsPerBlock - 1) / kItemsPerBlock;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kThreads / 32 ? s_warp[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < kThreads / 32) s_warp[lane] = wi - w;
    if (lane == kThreads / 32 - 1) s_warp[kThreads / 32] = wi;
  }
  __syncthreads();
  uint32_t r = s_warp[warp] + inc - x;
  *total = s_warp[kThreads / 32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan (reduce, scan block sums, scan + add)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                          const uint32_t* __restrict__ n_dev,
                                                          uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t s_warp[kThreads / 32 + 1];
  const uint32_t n = *n_dev;
  const uint32_t b = blockIdx.x;
  if (b >= num_blocks(n)) return;
  const uint64_t base = (uint64_t)b * kItemsPerBlock;
  uint32_t sum = 0;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    uint64_t idx = base + (uint64_t)r * kThreads + threadIdx.x;
    if (idx < n) sum += in[idx];
  }
  uint32_t total;
  block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) block_sums[b] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* __restrict__ block_sums,
                                                   const uint32_t* __restrict__ n_dev,
                                                   uint32_t* __restrict__ total_dev) {
  __shared__ uint32_t s_part[1024];
  const uint32_t nb = num_blocks(*n_dev);
  const uint32_t per = (nb + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(nb, lo + per);
  uint32_t sum = 0;
  for (uint32_t k = lo; k < hi; ++k) sum += block_sums[k];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partial sums
  for (int d = 1; d < 1024; d <<= 1) {
    uint32_t y = threadIdx.x >= (unsigned)d ? s_part[threadIdx.x - d] : 0u;
    __syncthreads();
    s_part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = s_part[threadIdx.x] - sum;
  for (uint32_t k = lo; k < hi; ++k) {
    uint32_t x = block_sums[k];
    block_sums[k] = run;
    run += x;
  }
  if (threadIdx.x == 1023) *total_dev = s_part[1023];
}

// in and out may alias (in-place scan): each thread reads its items before the
// block barrier and writes only those items afterwards.
__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t* in, uint32_t* out,
                                                        const uint32_t* __restrict__ block_sums,
                                                        const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t s_warp[kThreads / 32 + 1];
  const uint32_t n = *n_dev;
  const uint32_t b = blockIdx.x;
  if (b >= num_blocks(n)) return;
  // thread t owns the contiguous items [base + t*kIPT, base + (t+1)*kIPT)
  const uint64_t base = (uint64_t)b * kItemsPerBlock + (uint64_t)threadIdx.x * kIPT;
  uint32_t x[kIPT];
  uint32_t sum = 0;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    x[r] = (base + r < n) ? in[base + r] : 0u;
    sum += x[r];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, s_warp, &total) + block_sums[b];
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    if (base + r < n) out[base + r] = run;
    run += x[r];
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ n_dev,
                                                         int shift, uint32_t* __restrict__ hist,
                                                         uint32_t* __restrict__ hist_n_dev) {
  __shared__ uint32_t s_h[kRadixDigits];
  const uint32_t n = *n_dev;
  const uint32_t nb = num_blocks(n);
  const uint32_t b = blockIdx.x;
  if (b == 0 && threadIdx.x == 0) *hist_n_dev = kRadixDigits * nb;
  if (b >= nb) return;
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)b * kItemsPerBlock;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    uint64_t idx = base + (uint64_t)r * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&s_h[(keys[idx] >> shift) & (kRadixDigits - 1)], 1u);
  }
  __syncthreads();
  // digit-major layout: all blocks of digit 0, then digit 1, ...
  hist[(uint64_t)threadIdx.x * nb + b] = s_h[threadIdx.x];
}

// Each warp ranks 256 consecutive items (8 rounds of 32) with __match_any_sync;
// the block's offset for a digit is the scanned histogram entry, the warp's
// offset is the count of that digit in earlier warps: order is preserved.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
    const uint32_t* __restrict__ n_dev, int shift, const uint32_t* __restrict__ hist_scanned,
    uint32_t n_cap) {
  __shared__ uint32_t s_wh[kThreads / 32][kRadixDigits];
  __shared__ uint32_t s_bo[kRadixDigits];
  const uint32_t n = *n_dev;
  const uint32_t nb = num_blocks(n);
  const uint32_t b = blockIdx.x;
  if (b >= nb) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) s_wh[w][threadIdx.x] = 0;
  s_bo[threadIdx.x] = hist_scanned[(uint64_t)threadIdx.x * nb + b];
  __syncthreads();
  const uint64_t wbase = (uint64_t)b * kItemsPerBlock + (uint64_t)warp * (32 * kIPT);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kIPT], val[kIPT], rank[kIPT], dig[kIPT];
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
    const bool ok = idx < n;
    key[r] = ok ? keys_in[idx] : 0u;
    val[r] = ok ? vals_in[idx] : 0u;
    dig[r] = ok ? ((key[r] >> shift) & (kRadixDigits - 1)) : (uint32_t)kRadixDigits;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
    uint32_t prev = 0;
    if (ok) prev = s_wh[warp][dig[r]];
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) s_wh[warp][dig[r]] = prev + __popc(peers);
    __syncwarp();
    rank[r] = prev + __popc(peers & lt_mask);
  }
  __syncthreads();
  {
    // exclusive scan over warps for digit threadIdx.x
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      uint32_t c = s_wh[w][threadIdx.x];
      s_wh[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    if (dig[r] < (uint32_t)kRadixDigits) {
      const uint32_t pos = s_bo[dig[r]] + s_wh[warp][dig[r]] + rank[r];
      if (pos < n_cap) {  // always true for a consistent histogram
        keys_out[pos] = key[r];
        vals_out[pos] = val[r];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Item and pair kernels
// ---------------------------------------------------------------------------
__global__ void k_visible_flags(const uint32_t* __restrict__ touched, int64_t m,
                                uint32_t* __restrict__ flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) flags[i] = touched[i] > 0u ? 1u : 0u;
}

__global__ void k_compact(const uint32_t* __restrict__ touched, const float* __restrict__ depth,
                          const uint32_t* __restrict__ offs, int64_t m,
                          uint32_t* __restrict__ dkeys, uint32_t* __restrict__ items) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || touched[i] == 0u) return;
  const uint32_t o = offs[i];
  dkeys[o] = __float_as_uint(depth[i]);  // positive floats order like their bits
  items[o] = (uint32_t)i;
}

// Status bits written to counts[2]: 1 = pair capacity exceeded, 2 = an index
// read from an earlier stage was out of range (the access was skipped).
constexpr uint32_t kStatusCapacity = 1u, kStatusIndex = 2u;

__global__ void k_pair_counts(const uint32_t* __restrict__ items, const uint32_t* __restrict__ touched,
                              const uint32_t* __restrict__ n_dev, int64_t m, uint32_t* __restrict__ cnt,
                              uint32_t* __restrict__ counts) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= *n_dev || (int64_t)j >= m) return;
  const uint32_t it = items[j];
  if ((int64_t)it >= m) {
    cnt[j] = 0;
    atomicOr(&counts[2], kStatusIndex);
    return;
  }
  cnt[j] = touched[it];
}

__global__ void k_init_counts(uint32_t* counts, uint32_t* m_dev, uint32_t m) {
  *m_dev = m;  // live length of the first (item) scan; its total goes to counts[0]
  counts[0] = 0; counts[1] = 0; counts[2] = 0; counts[3] = 0;
}

__global__ void k_pair_status(uint32_t* counts, int64_t cap) {
  const uint32_t K = counts[1];
  if ((int64_t)K > cap) counts[2] |= kStatusCapacity;
  counts[3] = (int64_t)K > cap ? (uint32_t)cap : K;
}

struct EmitArgs {
  const uint32_t* items;
  const uint32_t* poff;
  const uint2* rect;
  const uint32_t* counts;
  int64_t n;
  int64_t cap;
  uint32_t* pair_off;
  uint32_t* tkeys;
  uint32_t* tvals;
};

// Warp-cooperative emission: each warp takes 32 consecutive items (in depth
// order); lane l loads item l's record, then the warp emits the items one
// after another with its 32 lanes striding over the item's tiles, so a splat
// covering hundreds of tiles is written by 32 lanes and consecutive pairs are
// written by consecutive lanes (coalesced).
__global__ void __launch_bounds__(256) k_emit(const EmitArgs a, const ViewTable vt) {
  const uint32_t M = a.counts[0];
  const int lane = threadIdx.x & 31;
  const uint32_t j0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
  if (j0 >= M || (int64_t)j0 >= a.n * vt.views) return;
  const uint32_t j = j0 + lane;
  const int64_t total = a.n * vt.views;
  bool ok = j < M && (int64_t)j < total;
  uint32_t item = 0, off = 0, rx = 1u, ry = 0u;
  int v = 0;
  if (ok) {
    item = a.items[j];
    if ((int64_t)item >= total) {
      atomicOr(const_cast<uint32_t*>(&a.counts[2]), kStatusIndex);
      ok = false;
    } else {
      v = (int)(item / (uint64_t)a.n);
      off = a.poff[j];
      a.pair_off[item] = off;
      const uint2 rc = a.rect[item];
      rx = rc.x;
      ry = rc.y;
      if ((int)(ry & 0xffff) >= vt.v[v].TX || (int)(ry >> 16) >= vt.v[v].TY) {
        atomicOr(const_cast<uint32_t*>(&a.counts[2]), kStatusIndex);
        ok = false;
      }
    }
  }
  for (int src = 0; src < 32; ++src) {
    const bool sok = __shfl_sync(0xffffffffu, ok, src);
    const uint32_t sitem = __shfl_sync(0xffffffffu, item, src);
    const uint32_t soff = __shfl_sync(0xffffffffu, off, src);
    const uint32_t sx = __shfl_sync(0xffffffffu, rx, src);
    const uint32_t sy = __shfl_sync(0xffffffffu, ry, src);
    const int sv = __shfl_sync(0xffffffffu, v, src);
    if (!sok) continue;
    const int x0 = sx & 0xffff, y0 = sx >> 16, x1 = sy & 0xffff, y1 = sy >> 16;
    const int w = x1 - x0 + 1;
    const int cnt = w * (y1 - y0 + 1);
    const int TX = vt.v[sv].TX;
    const uint32_t tb = (uint32_t)vt.v[sv].tile_base;
    const uint32_t g = (uint32_t)(sitem - (uint64_t)sv * a.n);
    for (int t = lane; t < cnt; t += 32) {
      const uint64_t k = (uint64_t)soff + t;
      if ((int64_t)k >= a.cap) break;
      const int ty = y0 + t / w, tx = x0 + t % w;
      a.tkeys[k] = tb + (uint32_t)(ty * TX + tx);
      a.tvals[k] = g;
    }
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ tkeys, uint32_t* __restrict__ counts,
                         uint2* __restrict__ ranges, uint32_t num_tiles) {
  const uint32_t K = counts[3];
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const uint32_t g = tkeys[k];
  if (g >= num_tiles) {
    atomicOr(&counts[2], kStatusIndex);
    return;
  }
  if (k == 0 || tkeys[k - 1] != g) ranges[g].x = k;
  if (k == K - 1 || tkeys[k + 1] != g) ranges[g].y = k + 1;
}

__global__ void k_full_keys(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ vals,
                            const uint32_t* __restrict__ counts, const float* __restrict__ depth,
                            int64_t n, uint64_t* __restrict__ keys, const ViewTable vt) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= counts[3]) return;
  const uint32_t g = tkeys[k];
  const int v = view_of_tile(vt, (int)g);
  const uint32_t gid = vals[k];
  keys[k] = ((uint64_t)g << 32) | (gid < n ? __float_as_uint(depth[(int64_t)v * n + gid]) : 0u);
}

inline unsigned grid_for(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads);
}

}  // namespace

// ---------------------------------------------------------------------------
size_t scan_workspace(int64_t n_cap) {
  return align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(1, (n_cap + kItemsPerBlock - 1) / kItemsPerBlock), 256);
}

gs_status launch_scan(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, int64_t n_cap,
                      uint32_t* total_dev, void* ws, cudaStream_t s) {
  uint32_t* block_sums = static_cast<uint32_t*>(ws);
  const unsigned nb = grid_for(n_cap, kItemsPerBlock);
  k_scan_reduce<<<nb, kThreads, 0, s>>>(in, n_dev, block_sums);
  k_scan_top<<<1, 1024, 0, s>>>(block_sums, n_dev, total_dev);
  k_scan_down<<<nb, kThreads, 0, s>>>(in, out, block_sums, n_dev);
  return check_launch("scan");
}

size_t radix_workspace(int64_t n_cap) {
  const int64_t nb = std::max<int64_t>(1, (n_cap + kItemsPerBlock - 1) / kItemsPerBlock);
  return align_up(sizeof(uint32_t) * kRadixDigits * nb, 256) + scan_workspace(kRadixDigits * nb) + 256;
}

gs_status launch_radix_sort(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b,
                            uint32_t* keys_out, uint32_t* vals_out, const uint32_t* n_dev,
                            int64_t n_cap, int bits, void* ws, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>(1, (n_cap + kItemsPerBlock - 1) / kItemsPerBlock);
  char* w = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w);
  w += align_up(sizeof(uint32_t) * kRadixDigits * nb, 256);
  void* scan_ws = w;
  w += scan_workspace(kRadixDigits * nb);
  uint32_t* hist_n = reinterpret_cast<uint32_t*>(w);
  uint32_t* hist_total = hist_n + 1;
  const int passes = std::max(1, (bits + kRadixBits - 1) / kRadixBits);
  const uint32_t* ksrc = keys_a;
  const uint32_t* vsrc = vals_a;
  for (int p = 0; p < passes; ++p) {
    uint32_t* kdst = (p == passes - 1) ? keys_out : ((p & 1) == 0 ? keys_b : keys_a);
    uint32_t* vdst = (p == passes - 1) ? vals_out : ((p & 1) == 0 ? vals_b : vals_a);
    const int shift = p * kRadixBits;
    k_radix_hist<<<(unsigned)nb, kThreads, 0, s>>>(ksrc, n_dev, shift, hist, hist_n);
    gs_status st = launch_scan(hist, hist, hist_n, kRadixDigits * nb, hist_total, scan_ws, s);
    if (st != GS_OK) return st;
    k_radix_scatter<<<(unsigned)nb, kThreads, 0, s>>>(ksrc, vsrc, kdst, vdst, n_dev, shift, hist,
                                                       (uint32_t)n_cap);
    ksrc = kdst;
    vsrc = vdst;
  }
  return check_launch("radix_sort");
}

// ---------------------------------------------------------------------------
// Workspace of gs_bin_sort: item arrays sized n*V, pair arrays sized capacity.
// ---------------------------------------------------------------------------
struct BinWs {
  uint32_t* scalars;  // [0] = item count m (input length of the first scan)
  uint32_t *offs, *dk_a, *it_a, *dk_b, *it_b, *dk_s, *it_s, *cnt;
  uint32_t *tk_a, *tv_a, *tk_b, *tv_b, *tk_s;
  void* radix;
  void* scan;
  size_t bytes;
};

static BinWs bin_layout(char* base, int64_t m, int64_t cap) {
  BinWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes, 256);
    return p;
  };
  const size_t mi = sizeof(uint32_t) * (size_t)std::max<int64_t>(1, m);
  const size_t ci = sizeof(uint32_t) * (size_t)std::max<int64_t>(1, cap);
  w.scalars = (uint32_t*)take(16);
  w.offs = (uint32_t*)take(mi);
  w.dk_a = (uint32_t*)take(mi); w.it_a = (uint32_t*)take(mi);
  w.dk_b = (uint32_t*)take(mi); w.it_b = (uint32_t*)take(mi);
  w.dk_s = (uint32_t*)take(mi); w.it_s = (uint32_t*)take(mi);
  w.cnt = (uint32_t*)take(mi);
  w.tk_a = (uint32_t*)take(ci); w.tv_a = (uint32_t*)take(ci);
  w.tk_b = (uint32_t*)take(ci); w.tv_b = (uint32_t*)take(ci);
  w.tk_s = (uint32_t*)take(ci);
  w.radix = take(radix_workspace(std::max(m, cap)));
  w.scan = take(scan_workspace(std::max(m, cap)));
  w.bytes = off;
  return w;
}

size_t bin_sort_workspace_bytes(int64_t m, int64_t cap) { return bin_layout(nullptr, m, cap).bytes; }

gs_status launch_bin_sort(const gs_splats& sp, const ViewTable& vt, const gs_bins& bins, void* ws,
                          cudaStream_t s) {
  const int64_t m = sp.n * vt.views;
  const int64_t cap = bins.capacity;
  BinWs w = bin_layout(static_cast<char*>(ws), m, cap);
  uint32_t* counts = bins.counts;
  const int T = 256;
  k_init_counts<<<1, 1, 0, s>>>(counts, w.scalars, (uint32_t)m);
  if (cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)bins.num_tiles, s) != cudaSuccess)
    return check_launch("memset ranges");
  if (m == 0) return check_launch("bin_sort");
  // 1. compact the visible items in (view, id) order with their depth keys
  k_visible_flags<<<grid_for(m, T), T, 0, s>>>(sp.touched, m, w.offs);
  // the scan's length (m) and its total (visible items -> counts[0]) must not alias
  gs_status st = launch_scan(w.offs, w.offs, w.scalars, m, counts, w.scan, s);
  if (st != GS_OK) return st;
  k_compact<<<grid_for(m, T), T, 0, s>>>(sp.touched, sp.depth, w.offs, m, w.dk_a, w.it_a);
  // 2. stable sort of the visible items by depth
  st = launch_radix_sort(w.dk_a, w.it_a, w.dk_b, w.it_b, w.dk_s, w.it_s, counts, m, 32, w.radix, s);
  if (st != GS_OK) return st;
  // 3. pair offsets in depth order, emission, pair count status
  k_pair_counts<<<grid_for(m, T), T, 0, s>>>(w.it_s, sp.touched, counts, m, w.cnt, counts);
  st = launch_scan(w.cnt, w.cnt, counts, m, counts + 1, w.scan, s);
  if (st != GS_OK) return st;
  k_pair_status<<<1, 1, 0, s>>>(counts, cap);
  EmitArgs ea{w.it_s, w.cnt, reinterpret_cast<const uint2*>(sp.rect), counts, sp.n, cap,
              bins.pair_off, w.tk_a, w.tv_a};
  k_emit<<<grid_for(m, T), T, 0, s>>>(ea, vt);
  // 4. stable sort of the pairs by global tile on its significant bits
  int bits = 1;
  while ((1ll << bits) < (int64_t)vt.total_tiles) ++bits;
  if (cap > 0) {
    st = launch_radix_sort(w.tk_a, w.tv_a, w.tk_b, w.tv_b, w.tk_s, bins.vals, counts + 3, cap, bits,
                           w.radix, s);
    if (st != GS_OK) return st;
    k_ranges<<<grid_for(cap, T), T, 0, s>>>(w.tk_s, counts, reinterpret_cast<uint2*>(bins.ranges),
                                            (uint32_t)bins.num_tiles);
    if (bins.keys)
      k_full_keys<<<grid_for(cap, T), T, 0, s>>>(w.tk_s, bins.vals, counts, sp.depth, sp.n, bins.keys, vt);
  }
  return check_launch("bin_sort");
}

}  // namespace gs
