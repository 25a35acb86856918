// Tile binning: per-tile duplication of the visible splats and the
// (tile, depth) sort that orders every tile's list front to back, then the
// [start, end) range of each tile.
//
// A counting sort by tile followed by a sort of each tile's own list:
//   1. a single-pass exclusive scan (decoupled look-back) of the
//      per-(view, Gaussian) tile counts gives every visible splat a
//      contiguous block of pair slots (pair_off, emission order: what the
//      backward indexes its per-pair gradients by), and
//   2. in the same launch every pair is counted in its tile (a reduction
//      into the ranges array, nothing waits for it);
//   3. one CTA scans the tiles' counts into list starts, sets each tile's
//      cursor to its start and groups the tiles by list length (and, when
//      asked, orders them longest list first); beyond 8192 tiles a
//      device-wide scan and two ordering kernels do it;
//   4. every pair takes the next place of its tile's cursor and writes its
//      (depth bits, Gaussian id) key there (splats of >= 128 tiles in
//      128-pair chunks by extra blocks of the same launch);
//   5. each tile's list is sorted: lists of fewer than 256 keys by one warp
//      in registers (eight tiles per CTA), up to 2048 by a CTA merging warp-
//      sorted runs of 256 in shared memory, up to 4096 by a CTA bitonic
//      network, the few beyond by stable radix passes through global
//      memory; the sort writes the ids.
// A first launch zeroes the counters, the ranges and the scan's look-back
// words; the five launches are chained as programmatic dependent launches.
// Within a tile every Gaussian appears once, so (depth bits, id) keys are
// distinct and the sorted list is unique: the atomics' order never shows.
// This is the order of one sort of 64-bit (tile, depth) keys with depth ties
// in id order, with ~30 bytes moved per pair.
//
// Every count (visible items, pairs) stays in device memory: kernels are
// launched for the capacity and read the live count, so the whole stage runs
// without a host synchronisation and can be captured in a CUDA graph.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 8;                      // items per thread (scans)
constexpr int kItemsPerBlock = kThreads * kIPT;
constexpr int kRadixBits = 8;                // long-list fallback sort
constexpr int kRadixDigits = 1 << kRadixBits;
constexpr int64_t kMaxScanTiles = 1ll << 25; // bound of the tile scan's workspace

__device__ __forceinline__ uint32_t num_blocks(uint32_t n) {
  return (n + kItemsPerBlock - 1) / kItemsPerBlock;
}

// Lanes of the warp that are `ok` and hold the same 8-bit digit as this lane
// (a multi-split by one ballot per digit bit; lanes not ok get no meaningful
// result).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool ok) {
  uint32_t m = __ballot_sync(0xffffffffu, ok);
#pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const uint32_t bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit != 0u);
    m &= bit ? bal : ~bal;
  }
  return m;
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
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ in, int in_stride,
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
    if (idx < n) sum += in[idx * in_stride];
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
// block barrier and writes only those items afterwards.  Strides are in
// elements (2 for the tile counts that sit in the ranges array).
__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t* in, int in_stride, uint32_t* out,
                                                        int out_stride, const uint32_t* __restrict__ block_sums,
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
    x[r] = (base + r < n) ? in[(base + r) * in_stride] : 0u;
    sum += x[r];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, s_warp, &total) + block_sums[b];
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    if (base + r < n) out[(base + r) * out_stride] = run;
    run += x[r];
  }
}


// ---------------------------------------------------------------------------
// Stable LSD radix sort of (u32 key, u32 value) pairs, 8-bit digits (used by
// the level-of-detail grouping)
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
// Pair kernels
// ---------------------------------------------------------------------------
// Status bits written to counts[2]: 1 = pair capacity exceeded, 2 = an index
// read from an earlier stage was out of range (the access was skipped).
constexpr uint32_t kStatusCapacity = 1u, kStatusIndex = 2u;

// Zeroes what a binning accumulates into, in one launch: the scalars and
// counters (block 0), the tiles' range words and the look-back words of the
// item scan (grid-stride).
__global__ void k_init_bins(uint32_t* counts, uint32_t* scalars, uint32_t m, uint32_t tiles, uint32_t* ranges,
                            int64_t range_words, unsigned long long* state, int64_t parts) {
  chain_enter();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < 128; i += blockDim.x) scalars[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      scalars[0] = m;      // live length of the item scan
      scalars[1] = tiles;  // live length of the tile scan
      counts[0] = 0; counts[1] = 0; counts[2] = 0; counts[3] = 0;
    }
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < range_words; i += stride) ranges[i] = 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < parts; i += stride) state[i] = 0ull;
}

// Items with at least kWide pairs (splats covering many tiles) are keyed in
// chunks of kWideChunk pairs, one warp per chunk, so that no warp walks a
// long item alone.
constexpr uint32_t kWide = 128, kWideChunk = 128;

struct PairArgs {
  const uint32_t* touched;
  const uint2* rect;
  const float* depth;
  uint32_t* pair_off;        // emission offset of every (view, Gaussian)
  uint32_t* counts;
  int64_t n;
  int64_t cap;
  uint32_t* ranges;          // [tiles][2]: word 1 counts the tile's pairs, then (start, cursor), then (start, end)
  uint64_t* keys;            // [cap] (depth bits << 32 | id) at the pair's list position
  unsigned long long* wide_count;  // (chunks << 32 | items) of the wide items, zero at launch
  uint2* wide_chunks;        // [wide_cap] (item, first pair of the chunk)
  uint32_t wide_cap;
};

// The next place in the tile's list (the tile's cursor).
__device__ __forceinline__ uint32_t take_place(const PairArgs& a, uint32_t tile) {
  return atomicAdd(&a.ranges[2 * (uint64_t)tile + 1], 1u);
}

// Warp-cooperative walk over the pairs of 32 consecutive (view, Gaussian)
// items starting at j0: the warp scans the items' pair counts and its lanes
// take the pairs 32 at a time, each finding its item by a binary search over
// the scan, so the lanes stay busy whatever the mix of small and large splats.
// Pairs of an item are its rect's tiles in row-major order; `off` is the
// lane's item's first pair slot (its pair_off), tch its tile count, rc its
// rect and dep its depth (loaded by the caller).  Pairs at slots >= cap
// (capacity overflow) are skipped by both passes.  Returns the visible items
// of the group (touched > 0).
// KEYS = false: count every pair in its tile (a reduction without return, no
// wait); true: take the next place of the tile's cursor and write the pair's
// key there.
template <bool KEYS>
__device__ __forceinline__ uint32_t warp_pairs(const PairArgs& a, const ViewTable& vt, int64_t j0, uint32_t off,
                                               uint32_t tch, uint2 rc, float dep) {
  const int64_t m = a.n * vt.views;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t j = j0 + lane;
  bool ok = j < m && tch > 0u;
  const uint32_t vis = (uint32_t)__popc(__ballot_sync(full, ok));
  if (KEYS && tch >= kWide) ok = false;  // keyed by the wide pass, in balanced chunks
  uint32_t x0y0 = 0, w = 1, cnt = 0, key_hi = 0, tb = 0, tx_n = 1, gid = 0;
  if (ok) {
    const int v = (int)(j / a.n);
    const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
    if (x1 >= vt.v[v].TX || y1 >= vt.v[v].TY || x0 > x1 || y0 > y1) {
      atomicOr(&a.counts[2], kStatusIndex);
      ok = false;
    } else {
      x0y0 = rc.x;
      w = (uint32_t)(x1 - x0 + 1);
      // never beyond the item's own block of slots
      cnt = min(w * (uint32_t)(y1 - y0 + 1), tch);
      tb = (uint32_t)vt.v[v].tile_base;
      tx_n = (uint32_t)vt.v[v].TX;
      if (KEYS) {
        key_hi = __float_as_uint(dep);  // positive floats order like their bits
        gid = (uint32_t)(j - (int64_t)v * a.n);
      }
    }
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(full, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t total = __shfl_sync(full, incl, 31);
  const uint32_t excl = incl - cnt;
  // rounds of 32 pairs, kRounds at a time: the key pass issues the rounds'
  // cursor atomics together and only then waits for their places
  constexpr int kRounds = KEYS ? 4 : 1;
  for (uint32_t base = 0; base < total; base += 32 * kRounds) {
    uint32_t pos[kRounds];
    uint64_t key[kRounds];
#pragma unroll
    for (int rr = 0; rr < kRounds; ++rr) {
      pos[rr] = 0xffffffffu;
      key[rr] = 0ull;
    }
#pragma unroll
    for (int rr = 0; rr < kRounds; ++rr) {
      const uint32_t q = base + 32 * rr + lane;
      if (base + 32 * rr >= total) break;  // warp-uniform
      // owner: the number of lanes whose inclusive count is <= q
      int o = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(full, incl, o + step - 1) <= q) o += step;
      const uint32_t so = __shfl_sync(full, off, o), se = __shfl_sync(full, excl, o);
      const uint32_t sxy = __shfl_sync(full, x0y0, o), sw = __shfl_sync(full, w, o);
      const uint32_t stb = __shfl_sync(full, tb, o), stx = __shfl_sync(full, tx_n, o);
      const uint32_t skey = KEYS ? __shfl_sync(full, key_hi, o) : 0u;
      const uint32_t sg = KEYS ? __shfl_sync(full, gid, o) : 0u;
      if (q >= total) continue;
      const uint32_t t = q - se;
      if ((int64_t)so + t >= a.cap) continue;
      const uint32_t tile = stb + ((sxy >> 16) + t / sw) * stx + (sxy & 0xffff) + t % sw;
      if (!KEYS) {
        atomicAdd(&a.ranges[2 * (uint64_t)tile + 1], 1u);  // result unused: a reduction
      } else {
        pos[rr] = take_place(a, tile);
        key[rr] = ((uint64_t)skey << 32) | sg;
      }
    }
    if (KEYS) {
#pragma unroll
      for (int rr = 0; rr < kRounds; ++rr) {
        if (pos[rr] == 0xffffffffu) continue;
        if ((int64_t)pos[rr] < a.cap) {
          a.keys[pos[rr]] = key[rr];
        } else {
          atomicOr(&a.counts[2], kStatusIndex);
        }
      }
    }
  }
  return vis;
}

// The wide items' keys: warps w, w + warps, ... take chunks of kWideChunk
// pairs; the lanes of a round take 32 consecutive pairs of the chunk, with
// the cursor atomics of the chunk's rounds issued together.
__device__ __forceinline__ void keys_wide(const PairArgs& a, const ViewTable& vt, uint32_t w, uint32_t warps) {
  const int lane = threadIdx.x & 31;
  const uint32_t nchunks = min((uint32_t)(*a.wide_count >> 32), a.wide_cap);
  for (uint32_t c = w; c < nchunks; c += warps) {
    const uint2 wc = a.wide_chunks[c];
    const int64_t j = wc.x;
    const uint32_t tch = a.touched[j], off = a.pair_off[j];
    const uint2 rc = a.rect[j];
    const float dep = a.depth[j];
    const int v = (int)(j / a.n);
    const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
    if (x1 >= vt.v[v].TX || y1 >= vt.v[v].TY || x0 > x1 || y0 > y1) {
      if (lane == 0) atomicOr(&a.counts[2], kStatusIndex);
      continue;
    }
    const uint32_t wd = (uint32_t)(x1 - x0 + 1);
    const uint32_t cnt = min(wd * (uint32_t)(y1 - y0 + 1), tch);
    const uint32_t tb = (uint32_t)vt.v[v].tile_base, tx_n = (uint32_t)vt.v[v].TX;
    const uint64_t key = ((uint64_t)__float_as_uint(dep) << 32) | (uint32_t)(j - (int64_t)v * a.n);
    constexpr int kR = kWideChunk / 32;
    uint32_t pos[kR];
#pragma unroll
    for (int rr = 0; rr < kR; ++rr) {
      pos[rr] = 0xffffffffu;
      const uint32_t t = wc.y + 32 * rr + lane;
      if (t >= cnt || (int64_t)off + t >= a.cap) continue;
      const uint32_t tile = tb + ((uint32_t)y0 + t / wd) * tx_n + (uint32_t)x0 + t % wd;
      pos[rr] = take_place(a, tile);
    }
#pragma unroll
    for (int rr = 0; rr < kR; ++rr) {
      if (pos[rr] == 0xffffffffu) continue;
      if ((int64_t)pos[rr] < a.cap) {
        a.keys[pos[rr]] = key;
      } else {
        atomicOr(&a.counts[2], kStatusIndex);
      }
    }
  }
}

// The key pass: blocks below item_blocks take 32 items per warp (offsets
// from pair_off); the blocks after them key the wide items' chunks, so that
// one launch covers both and the chunks fill the item blocks' tail.
__global__ void __launch_bounds__(256) k_keys(const PairArgs a, const ViewTable vt, uint32_t item_blocks) {
  chain_enter();
  if (blockIdx.x >= item_blocks) {
    const uint32_t wb = blockIdx.x - item_blocks, nwb = gridDim.x - item_blocks;
    keys_wide(a, vt, wb * (blockDim.x >> 5) + (threadIdx.x >> 5), nwb * (blockDim.x >> 5));
    return;
  }
  const int64_t m = a.n * vt.views;
  const int64_t j0 = ((int64_t)(blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
  if (j0 >= m) return;  // warp-uniform
  const int64_t j = j0 + (threadIdx.x & 31);
  // every load of the item at once (not waiting for its count)
  const bool in = j < m;
  const uint32_t tch = in ? a.touched[j] : 0u;
  const uint32_t off = in ? a.pair_off[j] : 0u;
  const uint2 rc = in ? a.rect[j] : make_uint2(0u, 0u);
  const float dep = in ? a.depth[j] : 0.f;
  warp_pairs<true>(a, vt, j0, off, tch, rc, dep);
}

// ---------------------------------------------------------------------------
// Single-pass scan of the items' tile counts with decoupled look-back, fused
// with the count pass.  Each CTA takes the next partition of 2048 items from
// a counter (so a CTA only ever waits for partitions taken before it, whose
// CTAs are already running), scans its counts, publishes its total, finds
// its prefix from the published words of the partitions before it (a warp
// reads 32 of them at a time), publishes its inclusive prefix, writes the
// pair offsets and then counts its items' pairs in their tiles.  The waits
// are bounded (kLookbackNs of %globaltimer): on expiry the CTA sets status
// bit 4 in counts[2] and carries on with a wrong prefix (the result is then
// flagged invalid, the launch still ends).
// ---------------------------------------------------------------------------
constexpr unsigned long long kFlagAgg = 1ull << 32, kFlagInc = 2ull << 32;
constexpr uint32_t kStatusTimeout = 16u;
constexpr unsigned long long kLookbackNs = 2000000000ull;  // 2 s

struct ScanCountArgs {
  PairArgs p;
  unsigned long long* state;  // [parts] look-back words (flag << 32 | value), zero at launch
  uint32_t* ticket;           // partition counter, zero at launch
  uint32_t parts;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreads) k_scan_count(const ScanCountArgs a, const ViewTable vt) {
  chain_enter();
  __shared__ uint32_t s_warp[kThreads / 32 + 1];
  __shared__ uint32_t s_part, s_prefix, s_vis;
  __shared__ uint32_t s_off[kItemsPerBlock], s_cnt[kItemsPerBlock];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t m = a.p.n * vt.views;
  if (threadIdx.x == 0) {
    s_part = atomicAdd(a.ticket, 1u);
    s_vis = 0;
  }
  __syncthreads();
  const uint32_t part = s_part;
  const uint64_t pbase = (uint64_t)part * kItemsPerBlock;
  // thread t owns the contiguous items [pbase + t*kIPT, pbase + (t+1)*kIPT)
  const uint64_t base = pbase + (uint64_t)threadIdx.x * kIPT;
  uint32_t x[kIPT];
  uint32_t sum = 0;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    x[r] = (int64_t)(base + r) < m ? a.p.touched[base + r] : 0u;
    sum += x[r];
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan(sum, s_warp, &total);
  if (warp == 0) {
    uint32_t prefix = 0;
    if (part == 0) {
      if (lane == 0) *(volatile unsigned long long*)&a.state[0] = kFlagInc | total;
    } else {
      if (lane == 0) *(volatile unsigned long long*)&a.state[part] = kFlagAgg | total;
      int64_t p = (int64_t)part - 1;
      const unsigned long long t0 = global_ns();
      for (;;) {
        const int64_t idx = p - lane;
        const unsigned long long wd =
            idx >= 0 ? *(volatile const unsigned long long*)&a.state[idx] : kFlagInc;  // none before the first
        const uint32_t flag = (uint32_t)(wd >> 32);
        const unsigned inc = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned ready = __ballot_sync(0xffffffffu, flag != 0u);
        const int first = inc ? __ffs(inc) - 1 : 31;            // the closest inclusive word, else all 32
        const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
        if ((ready & need) != need) {  // a partition before this one has not published yet
          if (global_ns() - t0 > kLookbackNs) {
            if (lane == 0) atomicOr(&a.p.counts[2], kStatusTimeout);
            break;
          }
          __nanosleep(64);
          continue;
        }
        uint32_t v = lane <= first ? (uint32_t)wd : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (inc) break;
        p -= 32;
      }
      if (lane == 0) *(volatile unsigned long long*)&a.state[part] = kFlagInc | (prefix + total);
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  uint32_t run = s_prefix + excl;
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    s_off[threadIdx.x * kIPT + r] = run;
    s_cnt[threadIdx.x * kIPT + r] = x[r];
    if ((int64_t)(base + r) < m) a.p.pair_off[base + r] = run;
    run += x[r];
  }
  // wide items: reserve their chunks (one atomic for the item and its chunks)
#pragma unroll
  for (int r = 0; r < kIPT; ++r) {
    if (x[r] < kWide) continue;
    const uint32_t nch = (x[r] + kWideChunk - 1) / kWideChunk;
    const unsigned long long old = atomicAdd(a.p.wide_count, ((unsigned long long)nch << 32) | 1ull);
    const uint32_t c0 = (uint32_t)(old >> 32);
    for (uint32_t c = 0; c < nch; ++c)
      if (c0 + c < a.p.wide_cap) a.p.wide_chunks[c0 + c] = make_uint2((uint32_t)(base + r), c * kWideChunk);
  }
  if (part == a.parts - 1 && threadIdx.x == kThreads - 1) {
    // the last partition knows the number of pairs
    const uint32_t K = run;
    a.p.counts[1] = K;
    if ((int64_t)K > a.p.cap) atomicOr(&a.p.counts[2], kStatusCapacity);
    a.p.counts[3] = (int64_t)K > a.p.cap ? (uint32_t)a.p.cap : K;
  }
  __syncthreads();
  // count pass: warp w takes the partition's 32-item groups w, w + 8, ...;
  // the rects of all its visible items are loaded first
  constexpr int kGroups = kItemsPerBlock / 32 / (kThreads / 32);
  uint2 rc[kGroups];
#pragma unroll
  for (int i = 0; i < kGroups; ++i) {
    const int g = warp + i * (kThreads / 32);
    const uint64_t jj = pbase + (uint64_t)g * 32 + lane;
    rc[i] = s_cnt[g * 32 + lane] ? a.p.rect[jj] : make_uint2(0u, 0u);
  }
  uint32_t vis = 0;
#pragma unroll
  for (int i = 0; i < kGroups; ++i) {
    const int g = warp + i * (kThreads / 32);
    const int64_t j0 = (int64_t)(pbase + (uint64_t)g * 32);
    if (j0 >= m) break;
    vis += warp_pairs<false>(a.p, vt, j0, s_off[g * 32 + lane], s_cnt[g * 32 + lane], rc[i], 0.f);
  }
  if (lane == 0 && vis) atomicAdd(&s_vis, vis);
  __syncthreads();
  if (threadIdx.x == 0 && s_vis) atomicAdd(&a.p.counts[0], s_vis);
}

// ---------------------------------------------------------------------------
// Tile scan: counts -> list starts, the cursors of the key pass, and the
// tiles grouped by list length.  Tiles go into power-of-two buckets: bucket 0
// holds lists of >= 2^15 pairs, bucket 15 single pairs, bucket 16 the empty
// tiles.  The order within a bucket follows the atomics and does not matter.
// Bucket counts go to bucket_count[17]; the non-empty tiles in bucket order
// to `work` (what the tile sort takes its work from), and, when asked, all
// tiles in bucket order (longest list first, empty tiles last) to `order`.
// An empty tile's range becomes (0, 0).
// ---------------------------------------------------------------------------
constexpr int kTileScanThreads = 1024;
// one CTA walks its threads' runs of tiles serially: quicker than the five
// launches of the device-wide form up to a few thousand tiles per thread
// block, slower beyond (80k tiles of a 16-view batch: 0.13 ms)
constexpr int64_t kTileScanMax = 1ll << 13;
constexpr int kOrderBuckets = 17;
constexpr int kShortBucket = 8;  // buckets >= 8 (lists of < 256 pairs) are sorted by one warp

__device__ __forceinline__ int order_bucket(uint32_t len) {
  return len == 0 ? kOrderBuckets - 1 : 15 - min(15, 31 - __clz(len));
}

// One CTA of 1024 threads (thread t takes a contiguous run of tiles), for up
// to kTileScanMax tiles; more go through the multi-kernel form below.
__global__ void __launch_bounds__(kTileScanThreads) k_tile_scan(uint32_t* __restrict__ ranges, uint32_t tiles,
                                                                 uint32_t* __restrict__ bucket_count,
                                                                 uint32_t* __restrict__ work,
                                                                 uint32_t* __restrict__ order) {
  chain_enter();
  constexpr int NW = kTileScanThreads / 32;
  __shared__ uint32_t s_warp[NW + 1];
  __shared__ uint32_t s_count[kOrderBuckets], s_base[kOrderBuckets];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t per = (tiles + kTileScanThreads - 1) / kTileScanThreads;
  const uint32_t lo = min(tiles, threadIdx.x * per), hi = min(tiles, lo + per);
  if (threadIdx.x < kOrderBuckets) s_count[threadIdx.x] = 0;
  __syncthreads();
  uint32_t sum = 0;
  for (uint32_t t = lo; t < hi; ++t) {
    const uint32_t c = ranges[2 * (uint64_t)t + 1];
    sum += c;
    atomicAdd(&s_count[order_bucket(c)], 1u);
  }
  // block-wide exclusive scan of the per-thread sums
  uint32_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < NW ? s_warp[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < NW) s_warp[lane] = wi - w;
  }
  if (threadIdx.x == 0) {
    uint32_t b0 = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      bucket_count[b] = s_count[b];
      s_base[b] = b0;
      b0 += s_count[b];
      s_count[b] = 0;
    }
  }
  __syncthreads();
  const uint32_t nonempty = s_base[kOrderBuckets - 1];
  uint32_t run = s_warp[warp] + inc - sum;
  for (uint32_t t = lo; t < hi; ++t) {
    const uint32_t c = ranges[2 * (uint64_t)t + 1];
    const int b = order_bucket(c);
    const uint32_t pos = s_base[b] + atomicAdd(&s_count[b], 1u);
    if (order) order[pos] = t;
    if (pos < nonempty) work[pos] = t;
    // the start, and the key pass's cursor; (0, 0) when empty
    const uint32_t st = c ? run : 0u;
    ranges[2 * (uint64_t)t] = st;
    ranges[2 * (uint64_t)t + 1] = st;
    run += c;
  }
}

// The multi-kernel form, for more tiles (after a device-wide scan has put
// the starts in ranges[2t], the counts still in ranges[2t + 1]): bucket
// counts, then placement (which also sets the cursors and empty ranges).
__global__ void __launch_bounds__(kThreads) k_order_count(const uint32_t* __restrict__ ranges, uint32_t tiles,
                                                          uint32_t* __restrict__ bucket_count) {
  __shared__ uint32_t s[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) s[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x)
    atomicAdd(&s[order_bucket(ranges[2 * (uint64_t)t + 1])], 1u);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets && s[threadIdx.x]) atomicAdd(&bucket_count[threadIdx.x], s[threadIdx.x]);
}

__global__ void __launch_bounds__(kThreads) k_order_place(uint32_t* __restrict__ ranges, uint32_t tiles,
                                                          const uint32_t* __restrict__ bucket_count,
                                                          uint32_t* __restrict__ cursor, uint32_t* __restrict__ work,
                                                          uint32_t* __restrict__ order) {
  __shared__ uint32_t s_base[kOrderBuckets];
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      s_base[b] = run;
      run += bucket_count[b];
    }
  }
  __syncthreads();
  const uint32_t nonempty = s_base[kOrderBuckets - 1];
  const int lane = threadIdx.x & 31;
  // grid-stride rounds are uniform per warp (the stride is a multiple of 32),
  // so the whole warp takes each round together: the lanes of one bucket
  // take their places with one atomic (most rounds hold a few buckets)
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < tiles; t0 += stride) {
    const uint32_t t = t0 + (uint32_t)lane;
    const bool in = t < tiles;
    const uint32_t c = in ? ranges[2 * (uint64_t)t + 1] : 0u;
    const int b = in ? order_bucket(c) : kOrderBuckets;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    uint32_t first = 0;
    if (in && lane == leader) first = atomicAdd(&cursor[b], (uint32_t)__popc(peers));
    first = __shfl_sync(0xffffffffu, first, leader);
    if (!in) continue;
    const uint32_t pos = s_base[b] + first + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (order && pos < tiles) order[pos] = t;
    if (pos < nonempty) work[pos] = t;
    const uint32_t st = c ? ranges[2 * (uint64_t)t] : 0u;
    ranges[2 * (uint64_t)t] = st;
    ranges[2 * (uint64_t)t + 1] = st;
  }
}

// One stable CTA-wide LSD radix pass over src[0, cnt) on key bits
// [lo, lo + 8), writing dst (shared or global memory).  A digit histogram of
// the whole list gives each digit's base; then, chunk by chunk (2048 keys),
// warp w ranks its contiguous share of the chunk with __match_any_sync and
// the keys go after everything of the same digit in earlier warps and chunks.
// Returns false (and writes nothing) when every key has the same digit: the
// pass would not move anything.
__device__ bool cta_radix_pass(const uint64_t* src, uint64_t* dst, uint32_t cnt, int lo, uint32_t* s_base,
                               uint32_t (*s_wh)[kRadixDigits]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t i0 = 0; i0 < cnt; i0 += kThreads) {
    const uint32_t i = i0 + threadIdx.x;
    const bool ok = i < cnt;
    const uint32_t d = ok ? (uint32_t)(src[i] >> lo) & (kRadixDigits - 1) : 0u;
    const uint32_t peers = digit_peers(d, ok);
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_base[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  {
    uint32_t total;
    const uint32_t c = s_base[threadIdx.x];
    const int uniform = __syncthreads_or(c == cnt);
    if (uniform) return false;
    s_base[threadIdx.x] = block_exclusive_scan(c, &s_wh[0][0], &total);
    __syncthreads();
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (uint32_t c0 = 0; c0 < cnt; c0 += kItemsPerBlock) {
    const uint32_t cc = min((uint32_t)kItemsPerBlock, cnt - c0);
    const uint32_t per = (cc + kThreads / 32 - 1) / (kThreads / 32);  // keys per warp
    const uint32_t w0 = c0 + (uint32_t)warp * per, w1 = c0 + min(cc, (uint32_t)(warp + 1) * per);
    const int rounds = (int)((per + 31) / 32);
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s_wh[w][threadIdx.x] = 0;
    __syncthreads();
    uint64_t key[kIPT];
    uint32_t rank[kIPT], dig[kIPT];
#pragma unroll
    for (int r = 0; r < kIPT; ++r) {
      dig[r] = (uint32_t)kRadixDigits;
      if (r < rounds) {
        const uint32_t idx = w0 + (uint32_t)r * 32 + lane;
        const bool ok = idx < w1;
        key[r] = ok ? src[idx] : 0ull;
        dig[r] = ok ? ((uint32_t)(key[r] >> lo) & (kRadixDigits - 1)) : (uint32_t)kRadixDigits;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        uint32_t prev = 0;
        if (ok) prev = s_wh[warp][dig[r]];
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) s_wh[warp][dig[r]] = prev + __popc(peers);
        __syncwarp();
        rank[r] = prev + __popc(peers & lt_mask);
      }
    }
    __syncthreads();
    uint32_t chunk_total = 0;
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t c = s_wh[w][threadIdx.x];
        s_wh[w][threadIdx.x] = run;
        run += c;
      }
      chunk_total = run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kIPT; ++r)
      if (dig[r] < (uint32_t)kRadixDigits) dst[s_base[dig[r]] + s_wh[warp][dig[r]] + rank[r]] = key[r];
    __syncthreads();
    s_base[threadIdx.x] += chunk_total;
    __syncthreads();
  }
  return true;
}

// Stable radix passes over key bits [lo0, lo1) in steps of 8; returns the
// buffer holding the result.
__device__ uint64_t* cta_radix_sort(uint64_t* a, uint64_t* b, uint32_t cnt, int lo0, int lo1, uint32_t* s_base,
                                    uint32_t (*s_wh)[kRadixDigits]) {
  for (int lo = lo0; lo < lo1; lo += kRadixBits) {
    if (!cta_radix_pass(a, b, cnt, lo, s_base, s_wh)) continue;
    uint64_t* t = a;
    a = b;
    b = t;
  }
  return a;
}

struct TileSortArgs {
  uint64_t* keys;       // [cap] tile lists, unsorted
  uint64_t* keys_b;     // [cap] ping-pong buffer of lists too long for shared memory
  const uint32_t* ranges;  // [tiles][2]: (start, end); (0, 0) when empty
  uint32_t* vals;       // [cap] Gaussian ids in list order
  uint64_t* full_keys;  // optional: (tile << 32 | depth bits) in list order
  const uint32_t* work;          // non-empty tiles grouped by list length, longest first
  const uint32_t* bucket_count;  // [17] tiles per length bucket
  int id_bits;          // significant bits of the id (low word)
};

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int j) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, j);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), j);
  return ((uint64_t)hi << 32) | lo;
}

// One exchange across lanes at distance J: the lane keeps the smaller key
// when it is the lower of the pair in an ascending run (or the upper in a
// descending one), else the larger.  Equal keys (padding) may go either way.
template <int J>
__device__ __forceinline__ void cx_lanes(uint64_t& x, bool up, int lane) {
  const uint64_t o = shfl_xor64(x, J);
  const bool keep_min = ((lane & J) == 0) == up;
  x = (keep_min == (o < x)) ? o : x;
}

// One exchange of two keys held by the same thread (x at the lower index).
__device__ __forceinline__ void cx_regs(uint64_t& x, uint64_t& y, bool up) {
  const bool swap = (y < x) == up;
  const uint64_t t = swap ? y : x;
  y = swap ? x : y;
  x = t;
}

// Stages J, J / 2, ..., 1 across lanes for one register (compile-time J).
template <int J>
__device__ __forceinline__ void lane_stages(uint64_t& x, bool up, int lane) {
  cx_lanes<J>(x, up, lane);
  if constexpr (J > 1) lane_stages<J / 2>(x, up, lane);
}

// Bitonic sorting network over 32 * E keys held by one warp in registers
// (element r * 32 + lane in v[r]); ascending.  Exchanges across lanes take a
// shuffle, the others stay in the thread.
template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[E]) {
  const int lane = threadIdx.x & 31;
  // stage blocks k = 2 .. 32: within each register
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t e = (uint32_t)(r * 32 + lane);
    cx_lanes<1>(v[r], (e & 2) == 0, lane);
    lane_stages<2>(v[r], (e & 4) == 0, lane);
    lane_stages<4>(v[r], (e & 8) == 0, lane);
    lane_stages<8>(v[r], (e & 16) == 0, lane);
    lane_stages<16>(v[r], (e & 32) == 0, lane);
  }
  // stage blocks k = 64 .. 32 E: distances >= 32 in registers, then lanes
#pragma unroll
  for (int k = 64; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int jr = k / 64; jr >= 1; jr >>= 1) {
#pragma unroll
      for (int r = 0; r < E; ++r)
        if (!(r & jr)) cx_regs(v[r], v[r | jr], ((r * 32) & k) == 0);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) lane_stages<16>(v[r], ((r * 32) & k) == 0, lane);
  }
}

template <int E>
__device__ __forceinline__ void warp_sort_list(const TileSortArgs& a, uint32_t t, uint32_t start, uint32_t cnt) {
  const int lane = threadIdx.x & 31;
  uint64_t v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t i = (uint32_t)(r * 32 + lane);
    v[r] = i < cnt ? a.keys[start + i] : ~0ull;
  }
  warp_bitonic<E>(v);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t i = (uint32_t)(r * 32 + lane);
    if (i < cnt) {
      a.vals[start + i] = (uint32_t)v[r];
      if (a.full_keys) a.full_keys[start + i] = ((uint64_t)t << 32) | (v[r] >> 32);
    }
  }
}

// Bitonic stages with partner distances 32, 16, ..., 1 of stage block k
// (k >= 64) over one 64-key block held by a warp in registers: x0 is key
// e0 = 64 b + lane, x1 key e0 + 32.  Distance 32 pairs a lane's own two keys,
// smaller ones pair lanes (shuffles).  Both keys share the direction.
__device__ __forceinline__ void block_run(uint64_t& x0, uint64_t& x1, uint32_t e0, uint32_t k) {
  const int lane = threadIdx.x & 31;
  const bool up = (e0 & k) == 0;
  cx_regs(x0, x1, up);
  lane_stages<16>(x0, up, lane);
  lane_stages<16>(x1, up, lane);
}

// Bitonic sort of a tile's list of cnt keys (N = a power of two >= cnt, 256
// .. kBitonicMax) by the CTA, ascending, writing the ids out.  Warp w owns
// the 64-key blocks w, w + 8, ...: every stage with a partner distance of at
// most 32 stays inside a block and runs in registers (stage blocks k <= 64
// entirely, straight from the global list), the others go through shared
// memory (contiguous, conflict-free pairs).
__device__ void cta_bitonic(const TileSortArgs& a, uint32_t t, uint32_t start, uint32_t cnt, uint32_t N,
                            uint64_t* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t bb = (uint32_t)warp; bb < N / 64; bb += kThreads / 32) {
    const uint32_t e0 = 64 * bb + (uint32_t)lane;
    uint64_t x0 = e0 < cnt ? a.keys[start + e0] : ~0ull;
    uint64_t x1 = e0 + 32 < cnt ? a.keys[start + e0 + 32] : ~0ull;
    // stage blocks 2 .. 32 inside each 32-key half, then 64
    cx_lanes<1>(x0, (e0 & 2) == 0, lane);
    lane_stages<2>(x0, (e0 & 4) == 0, lane);
    lane_stages<4>(x0, (e0 & 8) == 0, lane);
    lane_stages<8>(x0, (e0 & 16) == 0, lane);
    lane_stages<16>(x0, true, lane);
    cx_lanes<1>(x1, (e0 & 2) == 0, lane);
    lane_stages<2>(x1, (e0 & 4) == 0, lane);
    lane_stages<4>(x1, (e0 & 8) == 0, lane);
    lane_stages<8>(x1, (e0 & 16) == 0, lane);
    lane_stages<16>(x1, false, lane);
    block_run(x0, x1, e0, 64);
    s[e0] = x0;
    s[e0 + 32] = x1;
  }
  __syncthreads();
  for (uint32_t k = 128; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j >= 64; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < N / 2; i += kThreads) {
        const uint32_t x = 2 * i - (i & (j - 1)), y = x + j;
        const bool up = (x & k) == 0;
        const uint64_t p = s[x], q = s[y];
        if ((p > q) == up) {
          s[x] = q;
          s[y] = p;
        }
      }
      __syncthreads();
    }
    for (uint32_t bb = (uint32_t)warp; bb < N / 64; bb += kThreads / 32) {
      const uint32_t e0 = 64 * bb + (uint32_t)lane;
      uint64_t x0 = s[e0], x1 = s[e0 + 32];
      block_run(x0, x1, e0, k);
      if (k == N) {
        if (e0 < cnt) {
          a.vals[start + e0] = (uint32_t)x0;
          if (a.full_keys) a.full_keys[start + e0] = ((uint64_t)t << 32) | (x0 >> 32);
        }
        if (e0 + 32 < cnt) {
          a.vals[start + e0 + 32] = (uint32_t)x1;
          if (a.full_keys) a.full_keys[start + e0 + 32] = ((uint64_t)t << 32) | (x1 >> 32);
        }
      } else {
        s[e0] = x0;
        s[e0 + 32] = x1;
      }
    }
    if (k < N) __syncthreads();
  }
}

constexpr uint32_t kBitonicMax = 4096;  // longest list sorted in shared memory

constexpr uint32_t kMergeMax = 2048;     // longest list sorted by runs and merges (two buffers of s_keys)

// Sort of a tile's list of 256 < cnt <= kMergeMax keys by the CTA: warp w
// sorts runs w, w + 8, ... of 256 keys in registers (the warp's bitonic
// network; the last run padded with ~0 keys, which sort last), then passes of
// merges double the sorted runs up to the whole list, ping-ponging between
// the two halves of s (each thread finds where its share of a merged run
// starts by a binary search along the merge path, then merges its share in
// order).  Keys of a tile are distinct, so the result is the one order; the
// ids (and optionally the full keys) are written out.
__device__ void cta_merge_sort(const TileSortArgs& a, uint32_t t, uint32_t start, uint32_t cnt, uint64_t* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t npad = (cnt + 255u) & ~255u;  // whole runs of 256
  uint64_t* src = s;
  uint64_t* dst = s + kMergeMax;
  for (uint32_t r = (uint32_t)warp; r * 256u < npad; r += kThreads / 32) {
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const uint32_t i = r * 256u + (uint32_t)(e * 32 + lane);
      v[e] = i < cnt ? a.keys[start + i] : ~0ull;
    }
    warp_bitonic<8>(v);
#pragma unroll
    for (int e = 0; e < 8; ++e) src[r * 256u + (uint32_t)(e * 32 + lane)] = v[e];
  }
  __syncthreads();
  // each merged run is cut into chunks of kChunk outputs (kChunk divides
  // every run length 2 * width, so no chunk straddles two runs)
  constexpr uint32_t kChunk = 4;
  for (uint32_t width = 256; width < npad; width <<= 1) {
    for (uint32_t o = threadIdx.x * kChunk; o < npad; o += kThreads * kChunk) {
      const uint32_t seg = o / (2 * width) * (2 * width);
      const uint32_t la = min(width, npad - seg);       // run A = [seg, seg + la)
      const uint32_t lb = min(width, npad - seg - la);  // run B follows it (may be empty)
      const uint64_t* A = src + seg;
      const uint64_t* B = A + la;
      const uint32_t k = o - seg;  // position within the merged run
      // merge path: i keys of A and k - i of B precede output k
      uint32_t lo = k > lb ? k - lb : 0u, hi = min(k, la);
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[k - mid - 1]) lo = mid + 1; else hi = mid;
      }
      uint32_t i = lo, j = k - lo;
#pragma unroll
      for (uint32_t q = 0; q < kChunk; ++q) {
        const bool take_a = j >= lb || (i < la && A[i] <= B[j]);
        dst[o + q] = take_a ? A[i] : B[j];
        i += take_a ? 1u : 0u;
        j += take_a ? 0u : 1u;
      }
    }
    __syncthreads();
    uint64_t* tmp = src;
    src = dst;
    dst = tmp;
  }
  for (uint32_t i = threadIdx.x; i < cnt; i += kThreads) {
    const uint64_t key = src[i];
    a.vals[start + i] = (uint32_t)key;
    if (a.full_keys) a.full_keys[start + i] = ((uint64_t)t << 32) | (key >> 32);
  }
}



// The tile sort.  Work unit u < L (L = tiles of >= 256 pairs) is the u-th
// longest such tile, sorted by the whole CTA: a bitonic network in shared
// memory up to kBitonicMax keys, stable LSD radix passes through global
// memory beyond (a tile in which two keys share a depth is sorted again over
// id and depth bits, which leaves equal depths in id order).  Later units
// take eight shorter tiles, one per warp, each sorted in registers.  Keys
// (depth bits, id) are distinct within a tile, so every network gives the
// same list.  The CTA writes the ids (and optionally the full keys); the
// ranges are already (start, end).
__global__ void __launch_bounds__(kThreads, 4) k_tile_sort(const TileSortArgs a) {
  chain_enter();
  __shared__ __align__(16) uint64_t s_keys[kBitonicMax];
  __shared__ uint32_t s_base[kRadixDigits];
  __shared__ uint32_t s_wh[kThreads / 32][kRadixDigits];
  uint32_t L = 0, S = 0;
#pragma unroll
  for (int b = 0; b < kOrderBuckets - 1; ++b) (b < kShortBucket ? L : S) += a.bucket_count[b];
  const uint32_t u = blockIdx.x;
  const int warp = threadIdx.x >> 5;
  if (u >= L) {
    const uint32_t k = (u - L) * (kThreads / 32) + (uint32_t)warp;
    if (k >= S) return;
    const uint32_t t = a.work[L + k];
    const uint32_t start = a.ranges[2 * (uint64_t)t], cnt = a.ranges[2 * (uint64_t)t + 1] - start;
    if (cnt <= 32) warp_sort_list<1>(a, t, start, cnt);
    else if (cnt <= 64) warp_sort_list<2>(a, t, start, cnt);
    else if (cnt <= 128) warp_sort_list<4>(a, t, start, cnt);
    else warp_sort_list<8>(a, t, start, cnt);
    return;
  }
  const uint32_t t = a.work[u];
  const uint32_t start = a.ranges[2 * (uint64_t)t], cnt = a.ranges[2 * (uint64_t)t + 1] - start;
  if (cnt <= kMergeMax) {
    cta_merge_sort(a, t, start, cnt, s_keys);
    return;
  }
  if (cnt <= kBitonicMax) {
    uint32_t N = 256;
    while (N < cnt) N <<= 1;
    cta_bitonic(a, t, start, cnt, N, s_keys);
    return;
  }
  const uint64_t* sorted;
  {
    uint64_t* buf_a = a.keys + start;
    uint64_t* buf_b = a.keys_b + start;
    uint64_t* out = cta_radix_sort(buf_a, buf_b, cnt, 32, 64, s_base, s_wh);
    bool tie = false;
    for (uint32_t i = threadIdx.x; i + 1 < cnt; i += kThreads)
      tie |= (uint32_t)(out[i] >> 32) == (uint32_t)(out[i + 1] >> 32);
    if (__syncthreads_or(tie)) {
      uint64_t* other = out == buf_a ? buf_b : buf_a;
      out = cta_radix_sort(out, other, cnt, 0, (a.id_bits + kRadixBits - 1) / kRadixBits * kRadixBits, s_base,
                           s_wh);
      other = out == buf_a ? buf_b : buf_a;
      out = cta_radix_sort(out, other, cnt, 32, 64, s_base, s_wh);
    }
    __syncthreads();
    sorted = out;
  }
  for (uint32_t i = threadIdx.x; i < cnt; i += kThreads) {
    const uint64_t k = sorted[i];
    a.vals[start + i] = (uint32_t)k;
    if (a.full_keys) a.full_keys[start + i] = ((uint64_t)t << 32) | (k >> 32);
  }
}

inline unsigned grid_for(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads);
}

}  // namespace

// ---------------------------------------------------------------------------
size_t scan_workspace(int64_t n_cap) {
  return align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(1, (n_cap + kItemsPerBlock - 1) / kItemsPerBlock), 256);
}

gs_status launch_scan(const uint32_t* in, int in_stride, uint32_t* out, int out_stride, const uint32_t* n_dev,
                      int64_t n_cap, uint32_t* total_dev, void* ws, cudaStream_t s) {
  uint32_t* block_sums = static_cast<uint32_t*>(ws);
  const unsigned nb = grid_for(n_cap, kItemsPerBlock);
  k_scan_reduce<<<nb, kThreads, 0, s>>>(in, in_stride, n_dev, block_sums);
  k_scan_top<<<1, 1024, 0, s>>>(block_sums, n_dev, total_dev);
  k_scan_down<<<nb, kThreads, 0, s>>>(in, in_stride, out, out_stride, block_sums, n_dev);
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
    gs_status st = launch_scan(hist, 1, hist, 1, hist_n, kRadixDigits * nb, hist_total, scan_ws, s);
    if (st != GS_OK) return st;
    k_radix_scatter<<<(unsigned)nb, kThreads, 0, s>>>(ksrc, vsrc, kdst, vdst, n_dev, shift, hist,
                                                       (uint32_t)n_cap);
    ksrc = kdst;
    vsrc = vdst;
  }
  return check_launch("radix_sort");
}

// ---------------------------------------------------------------------------
// Workspace of gs_bin_sort: pair arrays sized capacity, one scan workspace.
// ---------------------------------------------------------------------------
struct BinWs {
  uint32_t* scalars;  // [0] = item count, [1] = tile count, [2] = scanned tile total,
                      // [3] = partition counter of the item scan, [4, 6) = the wide items'
                      // (chunks << 32 | items) counter, [32, 49) tiles per length bucket,
                      // [64, 81) their cursors
  unsigned long long* state;  // look-back words of the item scan, one per 2048 items
  uint32_t* work;             // [cap] non-empty tiles grouped by list length (at most one per pair)
  uint64_t *keys_a, *keys_b;
  void* scan;
  size_t bytes;
};

static int64_t scan_parts(int64_t m) { return (m + kItemsPerBlock - 1) / kItemsPerBlock; }

static BinWs bin_layout(char* base, int64_t m, int64_t cap) {
  BinWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes, 256);
    return p;
  };
  const size_t c = (size_t)std::max<int64_t>(1, cap);
  w.scalars = (uint32_t*)take(128 * sizeof(uint32_t));
  w.state = (unsigned long long*)take(sizeof(unsigned long long) * (size_t)std::max<int64_t>(1, scan_parts(m)));
  w.work = (uint32_t*)take(sizeof(uint32_t) * c);
  w.keys_a = (uint64_t*)take(sizeof(uint64_t) * c);
  w.keys_b = (uint64_t*)take(sizeof(uint64_t) * c);
  w.scan = take(scan_workspace(kMaxScanTiles));
  w.bytes = off;
  return w;
}

size_t bin_sort_workspace_bytes(int64_t m, int64_t cap) { return bin_layout(nullptr, m, cap).bytes; }

int64_t bin_sort_max_tiles() { return kMaxScanTiles; }

gs_status launch_bin_sort(const gs_splats& sp, const ViewTable& vt, const gs_bins& bins, void* ws,
                          cudaStream_t s) {
  const int64_t m = sp.n * vt.views;
  const int64_t cap = bins.capacity;
  BinWs w = bin_layout(static_cast<char*>(ws), m, cap);
  uint32_t* counts = bins.counts;
  const uint32_t tiles = (uint32_t)vt.total_tiles;
  // counters, scalars, the ranges (each tile's pair count, then (start,
  // cursor)) and the scan's look-back words, zeroed by one launch
  const int64_t parts = m > 0 ? scan_parts(m) : 0;
  const int64_t range_words = 2 * (int64_t)bins.num_tiles;
  const unsigned igrid =
      (unsigned)std::min<int64_t>(592, std::max<int64_t>(1, (std::max(range_words, parts) + 255) / 256));
  launch_dependent(k_init_bins, igrid, 256, s, counts, w.scalars, (uint32_t)m, tiles, bins.ranges, range_words,
                   w.state, parts);
  // the wide items' chunk table borrows keys_b (the sort's ping-pong buffer,
  // not used before the key passes end): cap entries, more than the
  // cap / 64 chunks that pairs within the capacity can need
  const uint32_t wide_cap = (uint32_t)std::min<int64_t>((int64_t)UINT32_MAX, std::max<int64_t>(1, cap));
  PairArgs pa{sp.touched, reinterpret_cast<const uint2*>(sp.rect), sp.depth, bins.pair_off, counts, sp.n, cap,
              bins.ranges, w.keys_a, reinterpret_cast<unsigned long long*>(w.scalars + 4),
              reinterpret_cast<uint2*>(w.keys_b), wide_cap};
  // 1. + 2. pair slots per (view, Gaussian) (single-pass scan of the tile
  // counts) and every pair counted in its tile, in one launch
  if (m > 0) {
    ScanCountArgs sa{pa, w.state, w.scalars + 3, (uint32_t)parts};
    launch_dependent(k_scan_count, (unsigned)parts, kThreads, s, sa, vt);
  }
  if (tiles == 0) return check_launch("bin_sort");
  // 3. list starts, the key pass's cursors and the tiles grouped by length
  if (vt.total_tiles <= kTileScanMax) {
    launch_dependent(k_tile_scan, 1, kTileScanThreads, s, bins.ranges, tiles, w.scalars + 32, w.work,
                     bins.tile_order);
  } else {
    gs_status st = launch_scan(bins.ranges + 1, 2, bins.ranges, 2, w.scalars + 1, vt.total_tiles, w.scalars + 2,
                               w.scan, s);
    if (st != GS_OK) return st;
    const unsigned og = (unsigned)std::min<int64_t>(592, ((int64_t)tiles + kThreads - 1) / kThreads);
    k_order_count<<<og, kThreads, 0, s>>>(bins.ranges, tiles, w.scalars + 32);
    k_order_place<<<og, kThreads, 0, s>>>(bins.ranges, tiles, w.scalars + 32, w.scalars + 64, w.work,
                                          bins.tile_order);
  }
  if (m == 0 || cap == 0) return check_launch("bin_sort");
  // 4. every key at its place in its tile's list
  const unsigned pgrid = (unsigned)std::max<int64_t>(1, (m + 255) / 256);  // 8 warps of 32 items per block
  const unsigned wgrid = (unsigned)std::min<int64_t>(1184, pgrid);         // the wide items' chunks
  launch_dependent(k_keys, pgrid + wgrid, 256, s, pa, vt, pgrid);
  // 5. every tile's list by (depth bits, id)
  int id_bits = 1;
  while (id_bits < 32 && (1ll << id_bits) < sp.n) ++id_bits;
  TileSortArgs ta{w.keys_a, w.keys_b, bins.ranges, bins.vals, reinterpret_cast<uint64_t*>(bins.keys), w.work,
                  w.scalars + 32, id_bits};
  const unsigned sgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(vt.total_tiles, cap));
  launch_dependent(k_tile_sort, sgrid, kThreads, s, ta);
  return check_launch("bin_sort");
}

}  // namespace gs
