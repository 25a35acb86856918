// Front-to-back alpha compositing per 16x16 tile and its backward (the
// per-pixel stages of the splat renderer of Sec. 5.2).
//
// One CTA per (view, tile), one thread per pixel.  Each batch of the tile's
// sorted splat list is staged in shared memory by the CTA's threads with
// coalesced float4 loads; the whole CTA leaves the list as soon as every pixel
// has saturated (__syncthreads_count, the block-wide ballot).
//
// The splat test is written once (splat_alpha) with explicit round-to-nearest
// intrinsics so that the forward, the backward's replay and the backward's
// reverse walk take bit-identical decisions.
#include "gs_internal.h"

namespace gs {

namespace {

struct Eval {
  float dx, dy, power, ex, raw, alpha;
};

// Alpha of one splat at pixel (px, py): false when the splat is skipped
// (centre outside [m-r, m+r]^2, power > 0 or alpha < 1/255).
__device__ __forceinline__ bool splat_alpha(const float4 m, const float4 co, float r, float px,
                                            float py, Eval& e) {
  e.dx = __fadd_rn(__fsub_rn(m.x, px), __fsub_rn(m.z, 0.5f));
  e.dy = __fadd_rn(__fsub_rn(m.y, py), __fsub_rn(m.w, 0.5f));
  if (fabsf(e.dx) > r || fabsf(e.dy) > r) return false;
  const float q = __fmaf_rn(co.x, __fmul_rn(e.dx, e.dx), __fmul_rn(co.z, __fmul_rn(e.dy, e.dy)));
  e.power = __fmaf_rn(-0.5f, q, __fmul_rn(-co.y, __fmul_rn(e.dx, e.dy)));
  if (e.power > 0.f) return false;
  e.ex = __expf(e.power);
  e.raw = __fmul_rn(co.w, e.ex);
  e.alpha = fminf(kAlphaMax, e.raw);
  return e.alpha >= kAlphaMin;
}

// A splat that never passes the test (radius -1): stands in for an
// out-of-range id, which is reported through counts[2] bit 2.
__device__ __forceinline__ void null_splat(float4& m, float4& co, float4& col) {
  m = make_float4(0.f, 0.f, 0.f, 0.f);
  co = make_float4(0.f, 0.f, 0.f, 0.f);
  col = make_float4(0.f, 0.f, 0.f, -1.f);
}

struct FwdArgs {
  const float4* xy;
  const float4* conic;
  const float4* rgb;
  const uint32_t* vals;
  const uint2* ranges;
  uint32_t* counts;
  int64_t n;
  float bg[3];
  float* image;
  float* alpha;
};

constexpr int kFwdBatch = kTilePixels;

// COUNT = true is the diagnostic instantiation behind gs_render_stats: the
// same loop, also counting per pixel the splats tested (up to and including
// the one that stops it) and blended, and per tile the backward's walk length.
template <bool COUNT>
__global__ void __launch_bounds__(kTilePixels) k_render_fwd(const FwdArgs a, const ViewTable vt,
                                                            unsigned long long* stats) {
  __shared__ float4 s_xy[kFwdBatch], s_co[kFwdBatch], s_rgb[kFwdBatch];
  __shared__ int s_last;
  uint32_t n_tested = 0, n_blended = 0;
  int last = -1;
  if (COUNT && threadIdx.x == 0) s_last = -1;
  const int gt = blockIdx.x;
  const int v = view_of_tile(vt, gt);
  const ViewInfo& vi = vt.v[v];
  const int lt = gt - vi.tile_base;
  const int tx = lt % vi.TX, ty = lt / vi.TX;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < vi.W && py < vi.H;
  const float pxf = (float)px, pyf = (float)py;
  const uint2 rg = a.ranges[gt];
  const int64_t vbase = (int64_t)v * a.n;
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += kFwdBatch) {
    if (__syncthreads_count(done) == kTilePixels) break;
    const uint32_t j = start + threadIdx.x;
    if (j < rg.y) {
      const uint32_t g = a.vals[j];
      if (g < a.n) {
        const int64_t gi = vbase + g;
        s_xy[threadIdx.x] = a.xy[gi];
        s_co[threadIdx.x] = a.conic[gi];
        s_rgb[threadIdx.x] = a.rgb[gi];
      } else {
        null_splat(s_xy[threadIdx.x], s_co[threadIdx.x], s_rgb[threadIdx.x]);
        atomicOr(&a.counts[2], 2u);
      }
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kFwdBatch, rg.y - start);
    for (int k = 0; !done && k < cnt; ++k) {
      const float4 col = s_rgb[k];
      Eval e;
      if (COUNT) ++n_tested;
      if (!splat_alpha(s_xy[k], s_co[k], col.w, pxf, pyf, e)) continue;
      const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
      if (Tn < kTransMin) { done = true; break; }
      const float w = e.alpha * T;
      c0 += col.x * w; c1 += col.y * w; c2 += col.z * w;
      T = Tn;
      if (COUNT) { ++n_blended; last = (int)(start + k); }
    }
  }
  if (COUNT) {
    __syncthreads();
    if (last >= 0) atomicMax(&s_last, last);
    unsigned long long t = n_tested, b = n_blended;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], t);
      atomicAdd(&stats[1], b);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_last >= 0) atomicAdd(&stats[2], (unsigned long long)(s_last + 1 - (int)rg.x));
    if (threadIdx.x == 0) atomicAdd(&stats[3], (unsigned long long)(rg.y - rg.x));
    return;
  }
  if (inside) {
    const int64_t np = (int64_t)vi.W * vi.H;
    const int64_t pix = (int64_t)py * vi.W + px;
    float* img = a.image + 3 * vi.pix_base;
    img[pix] = c0 + T * a.bg[0];
    img[np + pix] = c1 + T * a.bg[1];
    img[2 * np + pix] = c2 + T * a.bg[2];
    if (a.alpha) a.alpha[vi.pix_base + pix] = 1.f - T;
  }
}

struct BwdArgs {
  const float4* xy;
  const float4* conic;
  const float4* rgb;
  const uint2* rect;
  const uint32_t* pair_off;
  const uint32_t* vals;
  const uint2* ranges;
  uint32_t* counts;
  int64_t n;
  int64_t cap;
  float bg[3];
  const float* dimage;
  const float* dalpha;
  float* partials;  // [K][9]: dmx, dmy, dA, dB, dC, dopacity, dr, dg, db
};

constexpr int kBwdBatch = 128;
constexpr int kWarps = kTilePixels / 32;

// Warp sum of 9 values per lane with 14 shuffles instead of 45: values 0-7
// are reduced by halving exchanges (each step a lane keeps half of what it
// carries and sends the other half to its partner), value 8 by a plain
// butterfly.  On return lane l holds the total of value idx(l) in s8 where
// idx(l) = 4 [l & 16] + 2 [l & 8] + [l & 4] (lanes 0, 4, ..., 28 cover 0-7),
// and every lane holds the total of value 8 in t8.
__device__ __forceinline__ void warp_sum9(const float (&d)[kPartialStride], int lane, float& s8,
                                          int& idx, float& t8) {
  const unsigned full = 0xffffffffu;
  const bool u1 = (lane & 16) != 0, u2 = (lane & 8) != 0, u3 = (lane & 4) != 0;
  float k4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = u1 ? d[i] : d[i + 4];
    const float keep = u1 ? d[i + 4] : d[i];
    k4[i] = keep + __shfl_xor_sync(full, send, 16);
  }
  float k2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = u2 ? k4[i] : k4[i + 2];
    const float keep = u2 ? k4[i + 2] : k4[i];
    k2[i] = keep + __shfl_xor_sync(full, send, 8);
  }
  const float send = u3 ? k2[0] : k2[1];
  float k1 = (u3 ? k2[1] : k2[0]) + __shfl_xor_sync(full, send, 4);
  k1 += __shfl_xor_sync(full, k1, 2);
  k1 += __shfl_xor_sync(full, k1, 1);
  s8 = k1;
  idx = (u1 ? 4 : 0) + (u2 ? 2 : 0) + (u3 ? 1 : 0);
  float v = d[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
  t8 = v;
}

__global__ void __launch_bounds__(kTilePixels) k_render_bwd(const BwdArgs a, const ViewTable vt) {
  __shared__ float4 s_xy[kBwdBatch], s_co[kBwdBatch], s_rgb[kBwdBatch];
  __shared__ uint32_t s_pidx[kBwdBatch];
  __shared__ float s_red[kBwdBatch][kWarps][kPartialStride];
  __shared__ int s_maxlast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gt = blockIdx.x;
  const int v = view_of_tile(vt, gt);
  const ViewInfo& vi = vt.v[v];
  const int lt = gt - vi.tile_base;
  const int tx = lt % vi.TX, ty = lt / vi.TX;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < vi.W && py < vi.H;
  const float pxf = (float)px, pyf = (float)py;
  const uint2 rg = a.ranges[gt];
  const int64_t vbase = (int64_t)v * a.n;
  if (threadIdx.x == 0) s_maxlast = -1;

  // ---- 1. replay the forward: final transmittance and last blended position
  float T = 1.f;
  int last = -1;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += kBwdBatch) {
    if (__syncthreads_count(done) == kTilePixels) break;
    const uint32_t j = start + threadIdx.x;
    if (threadIdx.x < kBwdBatch && j < rg.y) {
      const uint32_t g = a.vals[j];
      if (g < a.n) {
        const int64_t gi = vbase + g;
        s_xy[threadIdx.x] = a.xy[gi];
        s_co[threadIdx.x] = a.conic[gi];
        s_rgb[threadIdx.x] = a.rgb[gi];
      } else {
        null_splat(s_xy[threadIdx.x], s_co[threadIdx.x], s_rgb[threadIdx.x]);
      }
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBwdBatch, rg.y - start);
    for (int k = 0; !done && k < cnt; ++k) {
      Eval e;
      if (!splat_alpha(s_xy[k], s_co[k], s_rgb[k].w, pxf, pyf, e)) continue;
      const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
      if (Tn < kTransMin) { done = true; break; }
      T = Tn;
      last = (int)(start + k);
    }
  }
  __syncthreads();
  if (last >= 0) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int maxlast = s_maxlast;
  const float Tfinal = T;

  float g0 = 0.f, g1 = 0.f, g2 = 0.f, ga = 0.f;
  if (inside) {
    const int64_t np = (int64_t)vi.W * vi.H;
    const int64_t pix = (int64_t)py * vi.W + px;
    const float* gi = a.dimage + 3 * vi.pix_base;
    g0 = gi[pix]; g1 = gi[np + pix]; g2 = gi[2 * np + pix];
    if (a.dalpha) ga = a.dalpha[vi.pix_base + pix];
  }
  float acc0 = Tfinal * a.bg[0], acc1 = Tfinal * a.bg[1], acc2 = Tfinal * a.bg[2];

  // pairs behind every pixel's last blended splat receive zero gradient
  for (uint32_t p = (uint32_t)(maxlast + 1) + threadIdx.x; p < rg.y; p += kTilePixels) {
    const uint32_t g = a.vals[p];
    if (g >= a.n) continue;
    const int64_t gi = vbase + g;
    const uint32_t pidx = a.pair_off[gi] + rect_index(a.rect[gi], tx, ty);
    if ((int64_t)pidx >= a.cap) {
      atomicOr(&a.counts[2], 2u);
      continue;
    }
    float* dst = a.partials + (int64_t)pidx * kPartialStride;
#pragma unroll
    for (int c = 0; c < kPartialStride; ++c) dst[c] = 0.f;
  }

  // ---- 2. back to front over [rg.x, maxlast]
  for (int bend = maxlast + 1; bend > (int)rg.x; bend -= kBwdBatch) {
    const int bstart = max((int)rg.x, bend - kBwdBatch);
    const int cnt = bend - bstart;
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint32_t g = a.vals[bstart + threadIdx.x];
      uint32_t pidx = 0xffffffffu;
      if (g < a.n) {
        const int64_t gi = vbase + g;
        s_xy[threadIdx.x] = a.xy[gi];
        s_co[threadIdx.x] = a.conic[gi];
        s_rgb[threadIdx.x] = a.rgb[gi];
        pidx = a.pair_off[gi] + rect_index(a.rect[gi], tx, ty);
      } else {
        null_splat(s_xy[threadIdx.x], s_co[threadIdx.x], s_rgb[threadIdx.x]);
      }
      s_pidx[threadIdx.x] = pidx;
    }
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      float d[kPartialStride];
#pragma unroll
      for (int c = 0; c < kPartialStride; ++c) d[c] = 0.f;
      bool contrib = false;
      Eval e;
      if (bstart + k <= last) {
        const float4 co = s_co[k];
        const float4 col = s_rgb[k];
        if (splat_alpha(s_xy[k], co, col.w, pxf, pyf, e)) {
          // 1 - alpha >= 0.01: one approximate reciprocal (relative error ~1e-7)
          // serves the transmittance recovery and the suffix terms
          const float rom = __fdividef(1.f, 1.f - e.alpha);
          const float Tb = T * rom;           // transmittance in front of this splat
          const float w = e.alpha * Tb;
          d[6] = g0 * w; d[7] = g1 * w; d[8] = g2 * w;
          float dal = g0 * (col.x * Tb - acc0 * rom) + g1 * (col.y * Tb - acc1 * rom) +
                      g2 * (col.z * Tb - acc2 * rom) + ga * Tfinal * rom;
          acc0 += col.x * w; acc1 += col.y * w; acc2 += col.z * w;
          if (e.raw <= kAlphaMax) {
            d[5] = dal * e.ex;                // d alpha / d opacity = exp(power)
            const float dp = dal * e.alpha;   // d alpha / d power = alpha
            d[2] = -0.5f * e.dx * e.dx * dp;
            d[3] = -e.dx * e.dy * dp;
            d[4] = -0.5f * e.dy * e.dy * dp;
            d[0] = -(co.x * e.dx + co.y * e.dy) * dp;
            d[1] = -(co.z * e.dy + co.y * e.dx) * dp;
          }
          T = Tb;
          contrib = true;
        }
      }
      float s8 = 0.f, t8 = 0.f;
      int idx = ((lane & 16) ? 4 : 0) + ((lane & 8) ? 2 : 0) + ((lane & 4) ? 1 : 0);
      if (__any_sync(0xffffffffu, contrib)) warp_sum9(d, lane, s8, idx, t8);
      if ((lane & 3) == 0) s_red[k][warp][idx] = s8;
      if (lane == 0) s_red[k][warp][8] = t8;
    }
    __syncthreads();
    if (threadIdx.x < cnt && (int64_t)s_pidx[threadIdx.x] >= a.cap) atomicOr(&a.counts[2], 2u);
    if (threadIdx.x < cnt && (int64_t)s_pidx[threadIdx.x] < a.cap) {
      float* dst = a.partials + (int64_t)s_pidx[threadIdx.x] * kPartialStride;
#pragma unroll
      for (int c = 0; c < kPartialStride; ++c) {
        float s = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < kWarps; ++w2) s += s_red[threadIdx.x][w2][c];
        dst[c] = s;
      }
    }
  }
}

}  // namespace

gs_status launch_render_fwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, float* image, float* alpha, cudaStream_t s) {
  FwdArgs a;
  a.xy = reinterpret_cast<const float4*>(sp.xy);
  a.conic = reinterpret_cast<const float4*>(sp.conic);
  a.rgb = reinterpret_cast<const float4*>(sp.rgb);
  a.vals = bins.vals;
  a.ranges = reinterpret_cast<const uint2*>(bins.ranges);
  a.counts = bins.counts;
  a.n = sp.n;
  for (int c = 0; c < 3; ++c) a.bg[c] = cfg.bg[c];
  a.image = image;
  a.alpha = alpha;
  if (vt.total_tiles == 0) return GS_OK;
  k_render_fwd<false><<<vt.total_tiles, kTilePixels, 0, s>>>(a, vt, nullptr);
  return check_launch("k_render_fwd");
}

gs_status launch_render_stats(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                              unsigned long long* stats, cudaStream_t s) {
  FwdArgs a;
  a.xy = reinterpret_cast<const float4*>(sp.xy);
  a.conic = reinterpret_cast<const float4*>(sp.conic);
  a.rgb = reinterpret_cast<const float4*>(sp.rgb);
  a.vals = bins.vals;
  a.ranges = reinterpret_cast<const uint2*>(bins.ranges);
  a.counts = bins.counts;
  a.n = sp.n;
  a.bg[0] = a.bg[1] = a.bg[2] = 0.f;
  a.image = nullptr;
  a.alpha = nullptr;
  if (cudaMemsetAsync(stats, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) return check_launch("stats");
  if (vt.total_tiles == 0) return GS_OK;
  k_render_fwd<true><<<vt.total_tiles, kTilePixels, 0, s>>>(a, vt, stats);
  return check_launch("k_render_fwd<count>");
}

gs_status launch_render_bwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, const float* dimage, const float* dalpha,
                            float* partials, cudaStream_t s) {
  BwdArgs a;
  a.xy = reinterpret_cast<const float4*>(sp.xy);
  a.conic = reinterpret_cast<const float4*>(sp.conic);
  a.rgb = reinterpret_cast<const float4*>(sp.rgb);
  a.rect = reinterpret_cast<const uint2*>(sp.rect);
  a.pair_off = bins.pair_off;
  a.vals = bins.vals;
  a.ranges = reinterpret_cast<const uint2*>(bins.ranges);
  a.counts = bins.counts;
  a.n = sp.n;
  a.cap = bins.capacity;
  for (int c = 0; c < 3; ++c) a.bg[c] = cfg.bg[c];
  a.dimage = dimage;
  a.dalpha = dalpha;
  a.partials = partials;
  if (vt.total_tiles == 0) return GS_OK;
  k_render_bwd<<<vt.total_tiles, kTilePixels, 0, s>>>(a, vt);
  return check_launch("k_render_bwd");
}

}  // namespace gs
