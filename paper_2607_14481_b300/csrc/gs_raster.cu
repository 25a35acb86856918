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
  float dx, dy, power, raw, alpha;
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
  e.raw = __fmul_rn(co.w, __expf(e.power));
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

__global__ void __launch_bounds__(kTilePixels) k_render_fwd(const FwdArgs a, const ViewTable vt) {
  __shared__ float4 s_xy[kFwdBatch], s_co[kFwdBatch], s_rgb[kFwdBatch];
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
      if (!splat_alpha(s_xy[k], s_co[k], col.w, pxf, pyf, e)) continue;
      const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
      if (Tn < kTransMin) { done = true; break; }
      const float w = e.alpha * T;
      c0 += col.x * w; c1 += col.y * w; c2 += col.z * w;
      T = Tn;
    }
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
          const float om = 1.f - e.alpha;
          const float Tb = T / om;            // transmittance in front of this splat
          const float w = e.alpha * Tb;
          d[6] = g0 * w; d[7] = g1 * w; d[8] = g2 * w;
          float dal = g0 * (col.x * Tb - acc0 / om) + g1 * (col.y * Tb - acc1 / om) +
                      g2 * (col.z * Tb - acc2 / om) + ga * Tfinal / om;
          acc0 += col.x * w; acc1 += col.y * w; acc2 += col.z * w;
          if (e.raw <= kAlphaMax) {
            d[5] = dal * (e.alpha / co.w);    // d alpha / d opacity = exp(power)
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
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int c = 0; c < kPartialStride; ++c) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) d[c] += __shfl_xor_sync(0xffffffffu, d[c], o);
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < kPartialStride; ++c) s_red[k][warp][c] = d[c];
      }
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
  k_render_fwd<<<vt.total_tiles, kTilePixels, 0, s>>>(a, vt);
  return check_launch("k_render_fwd");
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
