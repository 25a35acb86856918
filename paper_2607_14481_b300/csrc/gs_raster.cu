// Front-to-back alpha compositing per tile and its backward (the per-pixel
// stages of the splat renderer of §5.2), for tiles of 16x16, 32x8 or 8x32
// pixels.
//
// One CTA of 128 threads per (view, tile); each thread owns two vertically
// adjacent pixels, so a warp covers a strip of 64 pixels (16x4, 32x2 or 8x8)
// and every splat read from shared memory serves two pixels.  Each batch of
// the tile's sorted splat list is staged in shared memory by the CTA's
// threads with coalesced float4 loads, together with a mask of the warps
// whose strip the splat can reach at alpha >= 1/255 (the exponent's maximum
// over the strip, a conservative test, so a warp never skips a splat the
// exact per-pixel test would accept).  Each warp turns its bits of the masks
// into a bit set with one ballot per 32 staged splats and visits only the set
// bits, in list order.  The CTA leaves the list as soon as every pixel has
// saturated (__syncthreads_count).
//
// The backward accumulates per pixel only the moments of dL/dpower (dx dp,
// dy dp, dx^2 dp, dx dy dp, dy^2 dp) for the splat's mean and conic; the conic
// is applied once per (tile, splat) when the pair's reduced gradient is
// stored.  In the single-pass backward the stores of one batch's pairs and
// the staging of the next run side by side on different threads, and the
// staging asks L1 for the next batch's records one batch ahead.
//
// Each staged splat carries its centre relative to the tile origin, its conic
// scaled to base-2 exponent units and the exponent threshold below which its
// alpha would fall under 1/255, so a pixel test is a few FMAs and compares.
// A pixel's step over a visited splat has no branch: the test, the stop and
// the contribution are computed and masked to zero where the pixel does not
// blend.  The test is written once (splat_x with the pixel steps, and
// splat_alpha for the replay form) with explicit round-to-nearest intrinsics,
// so that the forward and every backward form take bit-identical decisions.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kThreads = kTilePixels / 2;   // two pixels per thread
constexpr int kWarps = kThreads / 32;
// Splats staged per batch: a template parameter of the composite (64, 128,
// 256) and of the single-pass backward (64, 128), chosen by the schedule.
//
// Tile shapes (a template parameter TW, the tile width; every shape has 256
// pixels): 16x16, 32x8, 8x32.  Thread t owns column t % TW and rows
// 2 (t / TW), 2 (t / TW) + 1, so warp w covers the strip of rows
// [w R, (w + 1) R) with R = 64 / TW rows: 16 x 4, 32 x 2 or 8 x 8 pixels.
template <int TW>
struct TileShape {
  static_assert(TW == 8 || TW == 16 || TW == 32, "tile width 8, 16 or 32");
  static constexpr int kW = TW;
  static constexpr int kH = kTilePixels / TW;
  static constexpr int kRowsPerWarp = 64 / TW;
};

struct Eval {
  float dx, dy, ex, raw, alpha;  // ex = exp(power), raw = opacity ex, alpha = min(0.99, raw)
};

constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the PTX instruction ex2.approx.ftz.f32 (relative error ~2^-22; the
// arguments here lie in [-8, 0], far from subnormal results).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Terms of the pixel test that depend only on the splat and the pixel
// column, shared by a thread's two pixels.
struct XTerms {
  float dx, a2dx2, b2dx;
};

// geo = (cx, cy, a2, b2): centre relative to the tile origin; a2 = -A/2 log2 e,
// b2 = -B log2 e.  geo2 = (c2, thr, opacity, r): c2 = -C/2 log2 e;
// thr = log2(1 / (255 opacity)).  lx = pixel column within the tile.
__device__ __forceinline__ XTerms splat_x(const float4 g, float lx) {
  XTerms t;
  t.dx = __fsub_rn(g.x, lx);
  t.b2dx = __fmul_rn(g.w, t.dx);
  t.a2dx2 = __fmul_rn(__fmul_rn(g.z, t.dx), t.dx);
  return t;
}

// Alpha of one splat at the pixel (lx, ly) of the tile: false when it is
// skipped (centre outside [m-r, m+r]^2, power > 0 or alpha < 1/255).  With
// p = power log2 e = a2 dx^2 + dy (b2 dx + c2 dy), alpha >= 1/255 is
// p >= thr, tested before the exponential.
__device__ __forceinline__ bool splat_alpha(const XTerms& x, const float4 g, const float4 g2, float ly,
                                            Eval& e) {
  e.dx = x.dx;
  e.dy = __fsub_rn(g.y, ly);
  if (fabsf(e.dx) > g2.w || fabsf(e.dy) > g2.w) return false;
  const float p = __fmaf_rn(e.dy, __fmaf_rn(g2.x, e.dy, x.b2dx), x.a2dx2);
  if (!(p <= 0.f && p >= g2.y)) return false;
  e.ex = ex2_approx(p);
  e.raw = __fmul_rn(g2.z, e.ex);
  e.alpha = fminf(kAlphaMax, e.raw);
  return true;
}

struct TileCoords {
  int v, tx, ty, px, py0;
  bool in0, in1;
  float ox, oy;        // tile origin (pixels)
  float lx, ly0, ly1;  // the thread's pixels within the tile
  float wlo, whi;      // the warp's first and last tile row
};

template <int TW>
__device__ __forceinline__ TileCoords tile_coords(const ViewTable& vt, int gt) {
  using S = TileShape<TW>;
  TileCoords c;
  c.v = view_of_tile(vt, gt);
  const ViewInfo& vi = vt.v[c.v];
  const int lt = gt - vi.tile_base;
  c.tx = lt % vi.TX;
  c.ty = lt / vi.TX;
  c.px = c.tx * S::kW + (threadIdx.x % S::kW);
  c.py0 = c.ty * S::kH + 2 * (threadIdx.x / S::kW);
  c.in0 = c.px < vi.W && c.py0 < vi.H;
  c.in1 = c.px < vi.W && c.py0 + 1 < vi.H;
  c.ox = (float)(c.tx * S::kW);
  c.oy = (float)(c.ty * S::kH);
  c.lx = (float)(threadIdx.x % S::kW);
  c.ly0 = (float)(2 * (threadIdx.x / S::kW));
  c.ly1 = c.ly0 + 1.f;
  c.wlo = (float)((threadIdx.x >> 5) * S::kRowsPerWarp);
  c.whi = c.wlo + (float)(S::kRowsPerWarp - 1);
  return c;
}

struct FwdArgs {
  const uint32_t* order;  // tile of each block (nullptr: block index)
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

// Largest exponent p(dx, dy) = a2 dx^2 + b2 dx dy + c2 dy^2 (a2, c2 < 0) over
// the rectangle [dxl, dxh] x [dyl, dyh]: 0 if it holds the centre, else the
// largest of the four edge maxima (each a concave parabola, its vertex
// clamped to the edge).
__device__ __forceinline__ float rect_pmax(float a2, float b2, float c2, float dxl, float dxh, float dyl,
                                           float dyh) {
  if (dxl <= 0.f && dxh >= 0.f && dyl <= 0.f && dyh >= 0.f) return 0.f;
  const float ia = -0.5f / a2, ic = -0.5f / c2;
  float best = -INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float dx = e ? dxh : dxl;  // vertical edge: maximise over dy
    const float dy = fminf(fmaxf(b2 * dx * ic, dyl), dyh);
    best = fmaxf(best, fmaf(c2 * dy + b2 * dx, dy, a2 * dx * dx));
    const float dy2 = e ? dyh : dyl;  // horizontal edge: maximise over dx
    const float dx2 = fminf(fmaxf(b2 * dy2 * ia, dxl), dxh);
    best = fmaxf(best, fmaf(a2 * dx2 + b2 * dy2, dx2, c2 * dy2 * dy2));
  }
  return best;
}

// Warp culling of a staged splat: bit w is set unless no point of warp w's
// strip of the tile (rows R w .. R (w + 1) - 1 with R = 64 / TW, columns
// 0..TW-1, as a continuous rectangle, cut to the support box |dx|, |dy| <= r)
// reaches the alpha threshold p >= thr (with a margin of 1e-3 (1 + |thr|)).
// Conservative: a warp with its bit clear has no pixel that passes the exact
// per-pixel test, so skipping it changes nothing.
template <int TW>
__device__ __forceinline__ uint8_t warp_mask(float cx, float cy, float a2, float b2, float c2, float thr,
                                             float r) {
  constexpr int R = TileShape<TW>::kRowsPerWarp;
  const float xl = fmaxf(0.f, cx - r), xh = fminf((float)(TW - 1), cx + r);
  if (!(a2 < 0.f && c2 < 0.f) || xl > xh) return 0u;
  const float lim = thr - 1e-3f * (1.f + fabsf(thr));
  uint8_t m = 0u;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const float yl = fmaxf((float)(R * w), cy - r);
    const float yh = fminf((float)(R * w + R - 1), cy + r);
    if (yl > yh) continue;
    if (rect_pmax(a2, b2, c2, cx - xh, cx - xl, cy - yh, cy - yl) >= lim) m |= (uint8_t)(1u << w);
  }
  return m;
}

// Stages splat `j` of the list (or a null splat: radius -1, opacity 0, which
// never passes the test, standing in for an out-of-range id reported through
// counts[2] bit 2) in shared memory slot `t`, relative to the tile origin
// (ox, oy).  rows = the tile rows [cy - r - 1, cy + r + 1] the splat can touch
// (one pixel of margin over the exact test), empty for a null splat.
// s_co (optional) keeps the unscaled conic and opacity for the backward.
template <int TW>
__device__ __forceinline__ void stage_splat(const float4* xy, const float4* conic, const float4* rgb,
                                            const uint32_t* vals, int64_t n, int64_t vbase, uint32_t j,
                                            int t, float ox, float oy, float4* s_geo, float4* s_geo2,
                                            float4* s_rgb, uint8_t* s_mask, float4* s_co, uint32_t* counts) {
  const uint32_t g = vals[j];
  float4 m, co, col;
  if (g < n) {
    const int64_t gi = vbase + g;
    m = xy[gi];
    co = conic[gi];
    col = rgb[gi];
  } else {
    m = make_float4(0.f, 0.f, 0.f, 0.f);
    co = m;
    col = make_float4(0.f, 0.f, 0.f, -1.f);
    if (counts) atomicOr(&counts[2], 2u);
  }
  const float cx = __fadd_rn(__fsub_rn(m.x, ox), __fsub_rn(m.z, 0.5f));
  const float cy = __fadd_rn(__fsub_rn(m.y, oy), __fsub_rn(m.w, 0.5f));
  s_geo[t] = make_float4(cx, cy, __fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y));
  s_geo2[t] = make_float4(__fmul_rn(-0.5f * kLog2e, co.z), -log2f(255.f * co.w), co.w, col.w);
  s_rgb[t] = col;
  if (s_co) s_co[t] = co;
  s_mask[t] = col.w < 0.f ? 0u : warp_mask<TW>(cx, cy, __fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y),
                                             __fmul_rn(-0.5f * kLog2e, co.z), -log2f(255.f * co.w), col.w);
}

// Asks this SM's L1 for the records of list position j one batch before
// they are staged: the staging's two dependent loads (list id, then
// records) then find their lines in L1 instead of waiting on L2 with every
// warp of the CTA at the barrier behind them.  Callers skip it once half of
// the tile's threads have stopped (the next batch may never be staged).
__device__ __forceinline__ void prefetch_splat(const float4* xy, const float4* conic, const float4* rgb,
                                               const uint32_t* vals, int64_t n, int64_t vbase, uint32_t j) {
  const uint32_t g = vals[j];
  if (g >= n) return;
  const int64_t gi = vbase + g;
  prefetch_l1(xy + gi);
  prefetch_l1(conic + gi);
  prefetch_l1(rgb + gi);
}

// Bit set of the staged splats [0, cnt) that warp `warp` can reach (its bit
// of s_mask), 32 per word, written to s_wb[0 .. ceil(cnt/32)): the warp's
// loop visits only these, in ascending order (front to back), instead of
// stepping over every staged splat and testing its bit.  Each warp builds
// and reads its own words (a __syncwarp orders them).
template <int kBatch>
__device__ __forceinline__ void warp_bits(const uint8_t* s_mask, int cnt, int warp, int lane, uint32_t* s_wb) {
#pragma unroll
  for (int q = 0; q < kBatch / 32; ++q) {
    const int k = q * 32 + lane;
    const uint32_t word = __ballot_sync(0xffffffffu, k < cnt && ((s_mask[k] >> warp) & 1u));
    if (lane == 0) s_wb[q] = word;
  }
  __syncwarp();
}

// Counters of the diagnostic instantiation (gs_render_stats).
struct CountState {
  uint32_t n_tested = 0, n_blended = 0;
  uint32_t stop0 = 0xffffffffu, stop1 = 0xffffffffu;  // list position of the splat that stopped the pixel
  int last = -1;                                       // last blended list position
};

// One pixel's composite step without branches: the splat test (as
// splat_alpha), the stop test, and the blend with the weight masked to zero
// when the pixel does not blend the splat (so its colour and transmittance
// keep their exact values).  Returns whether it blended; *stopped is set
// when the splat stops the pixel (and then done).
__device__ __forceinline__ bool pixel_step_fwd(const XTerms& x, const float4 g, const float4 g2, float ly,
                                               const float4 col, float& T, float& c0, float& c1, float& c2,
                                               bool& done, bool& stopped) {
  const float dy = __fsub_rn(g.y, ly);
  const float p = __fmaf_rn(dy, __fmaf_rn(g2.x, dy, x.b2dx), x.a2dx2);
  const bool hit = !done && fabsf(x.dx) <= g2.w && fabsf(dy) <= g2.w && p <= 0.f && p >= g2.y;
  // a power above zero fails the test; its exponential (up to +inf) is masked
  const float alpha = fminf(kAlphaMax, __fmul_rn(g2.z, ex2_approx(p)));
  const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
  stopped = hit && Tn < kTransMin;
  const bool blend = hit && !stopped;
  done = done || stopped;
  const float w = blend ? alpha * T : 0.f;
  c0 += col.x * w;
  c1 += col.y * w;
  c2 += col.z * w;
  T = blend ? Tn : T;
  return blend;
}

// Front-to-back composite of one tile's list for the thread's two pixels:
// on return T0/T1 hold the final transmittance and c0/c1 the colour
// composited (background not added).  Shared arrays: the staging slots of
// kBatch splats and the calling warp's words of the bit sets.  COUNT = true
// also counts per pixel the splats tested (up to and including the one that
// stops it) and blended.
template <bool COUNT, int kBatch, int TW>
__device__ __forceinline__ void composite_tile(const FwdArgs& a, const TileCoords& tc, const uint2 rg,
                                               const int64_t vbase, float4* s_geo, float4* s_geo2, float4* s_rgb,
                                               uint8_t* s_mask, uint32_t* s_wbw, float& T0, float& T1,
                                               float (&c0)[3], float (&c1)[3], CountState& cs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T0 = 1.f;
  T1 = 1.f;
  float c00 = 0.f, c01 = 0.f, c02 = 0.f, c10 = 0.f, c11 = 0.f, c12 = 0.f;
  bool d0 = !tc.in0, d1 = !tc.in1;
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    const int ndone = __syncthreads_count(d0 && d1);
    if (ndone == kThreads) break;
    const int cnt = (int)min((uint32_t)kBatch, rg.y - start);
    if (2 * ndone < kThreads)
      for (int t = threadIdx.x; t < kBatch && start + kBatch + t < rg.y; t += kThreads)
        prefetch_splat(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, start + kBatch + t);
    for (int t = threadIdx.x; t < cnt; t += kThreads)
      stage_splat<TW>(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, start + t, t, tc.ox, tc.oy, s_geo, s_geo2,
                      s_rgb, s_mask, nullptr, COUNT ? nullptr : a.counts);
    __syncthreads();
    warp_bits<kBatch>(s_mask, cnt, warp, lane, s_wbw);
    for (int q = 0; q * 32 < cnt && !(d0 && d1); ++q) {
     for (uint32_t bits = s_wbw[q]; bits && !(d0 && d1); bits &= bits - 1) {
      const int k = q * 32 + __ffs(bits) - 1;
      const float4 g = s_geo[k], g2 = s_geo2[k], col = s_rgb[k];
      const XTerms x = splat_x(g, tc.lx);
      if (COUNT) cs.n_tested += (d0 ? 0u : 1u) + (d1 ? 0u : 1u);
      bool st0, st1;
      const bool b0 = pixel_step_fwd(x, g, g2, tc.ly0, col, T0, c00, c01, c02, d0, st0);
      const bool b1 = pixel_step_fwd(x, g, g2, tc.ly1, col, T1, c10, c11, c12, d1, st1);
      if (COUNT) {
        if (st0) cs.stop0 = start + k;
        if (st1) cs.stop1 = start + k;
        cs.n_blended += (b0 ? 1u : 0u) + (b1 ? 1u : 0u);
        if (b0 || b1) cs.last = max(cs.last, (int)(start + k));
      }
     }
    }
  }
  c0[0] = c00; c0[1] = c01; c0[2] = c02;
  c1[0] = c10; c1[1] = c11; c1[2] = c12;
}

// COUNT = true is the diagnostic instantiation behind gs_render_stats: the
// same loop, also counting per pixel the splats tested (up to and including
// the one that stops it) and blended, and per tile the backward's walk length.
template <bool COUNT, int kBatch, int TW>
__global__ void __launch_bounds__(kThreads) k_render_fwd(const FwdArgs a, const ViewTable vt,
                                                         unsigned long long* stats) {
  __shared__ float4 s_geo[kBatch], s_geo2[kBatch], s_rgb[kBatch];
  __shared__ uint8_t s_mask[kBatch];
  __shared__ uint32_t s_wb[kWarps][kBatch / 32];
  __shared__ int s_last;
  const int warp = threadIdx.x >> 5;
  const int gt = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;  // longest lists first
  const TileCoords tc = tile_coords<TW>(vt, gt);
  const ViewInfo& vi = vt.v[tc.v];
  const uint2 rg = a.ranges[gt];
  const int64_t vbase = (int64_t)tc.v * a.n;
  if (COUNT && threadIdx.x == 0) s_last = -1;
  float T0, T1, cc0[3], cc1[3];
  CountState cs;
  composite_tile<COUNT, kBatch, TW>(a, tc, rg, vbase, s_geo, s_geo2, s_rgb, s_mask, s_wb[warp], T0, T1, cc0, cc1,
                                    cs);
  const uint32_t n_tested = cs.n_tested, n_blended = cs.n_blended, stop0 = cs.stop0, stop1 = cs.stop1;
  const int last = cs.last;
  const float c00 = cc0[0], c01 = cc0[1], c02 = cc0[2], c10 = cc1[0], c11 = cc1[1], c12 = cc1[2];
  if (COUNT) {
    __syncthreads();
    if (last >= 0) atomicMax(&s_last, last);
    unsigned long long t = n_tested, b = n_blended;
    // pairs the plain per-pixel loop evaluates: every list entry up to and
    // including the one that stops the pixel (the whole list otherwise)
    const uint32_t len = rg.y - rg.x;
    unsigned long long ev = (tc.in0 ? (stop0 != 0xffffffffu ? stop0 - rg.x + 1u : len) : 0u) +
                            (tc.in1 ? (stop1 != 0xffffffffu ? stop1 - rg.x + 1u : len) : 0u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], t);
      atomicAdd(&stats[1], b);
      atomicAdd(&stats[4], ev);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_last >= 0) atomicAdd(&stats[2], (unsigned long long)(s_last + 1 - (int)rg.x));
    if (threadIdx.x == 0) atomicAdd(&stats[3], (unsigned long long)(rg.y - rg.x));
    return;
  }
  const int64_t np = (int64_t)vi.W * vi.H;
  float* img = a.image + 3 * vi.pix_base;
  if (tc.in0) {
    const int64_t pix = (int64_t)tc.py0 * vi.W + tc.px;
    img[pix] = c00 + T0 * a.bg[0];
    img[np + pix] = c01 + T0 * a.bg[1];
    img[2 * np + pix] = c02 + T0 * a.bg[2];
    if (a.alpha) a.alpha[vi.pix_base + pix] = 1.f - T0;
  }
  if (tc.in1) {
    const int64_t pix = (int64_t)(tc.py0 + 1) * vi.W + tc.px;
    img[pix] = c10 + T1 * a.bg[0];
    img[np + pix] = c11 + T1 * a.bg[1];
    img[2 * np + pix] = c12 + T1 * a.bg[2];
    if (a.alpha) a.alpha[vi.pix_base + pix] = 1.f - T1;
  }
}

struct BwdArgs {
  const uint32_t* order;  // tile of each block (nullptr: block index)
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
  const float* image;  // the forward's output (single-pass variant)
  float* partials;  // [K][12]: dmx, dmy, dA, dB | dC, dopacity, dr, dg | db, 0, 0, 0
};

// Slot of the (tile, Gaussian) pair of list position j, 0xffffffff for an
// out-of-range id.
__device__ __forceinline__ uint32_t pair_slot(const BwdArgs& a, int64_t vbase, uint32_t j,
                                              const TileCoords& tc) {
  const uint32_t g = a.vals[j];
  return g < a.n ? a.pair_off[vbase + g] + rect_index(a.rect[vbase + g], tc.tx, tc.ty) : 0xffffffffu;
}

// Stores one pair's gradients: the sum over the warps that touched it, in
// warp order (deterministic), or zeros when none did.  Values 0-4 arrive as
// the moments S = (sum dx dp, sum dy dp, sum dx^2 dp, sum dx dy dp,
// sum dy^2 dp) of dp = dL/dpower over the tile's pixels (alpha_grad); with
// power = -(A dx^2 / 2 + B dx dy + C dy^2 / 2) and dx = m_x - p_x they give,
// with the splat's conic co = (A, B, C):
//   dL/dm_x = -(A S_x + B S_y),  dL/dm_y = -(B S_x + C S_y),
//   dL/dA = -S_xx / 2,  dL/dB = -S_xy,  dL/dC = -S_yy / 2.
__device__ __forceinline__ void store_pair(const BwdArgs& a, uint32_t pidx,
                                           const float (&red)[kWarps][kPartialValues],
                                           const uint8_t (&hit)[kWarps], const float4 co) {
  if ((int64_t)pidx >= a.cap) {
    if (pidx != 0xffffffffu) atomicOr(&a.counts[2], 2u);
    return;
  }
  float sum[kPartialValues];
#pragma unroll
  for (int c = 0; c < kPartialValues; ++c) {
    float acc = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
      if (hit[w]) acc += red[w][c];
    sum[c] = acc;
  }
  const float sx = sum[0], sy = sum[1], sxx = sum[2], sxy = sum[3], syy = sum[4];
  sum[0] = -(co.x * sx + co.y * sy);
  sum[1] = -(co.y * sx + co.z * sy);
  sum[2] = -0.5f * sxx;
  sum[3] = -sxy;
  sum[4] = -0.5f * syy;
  float4* dst = reinterpret_cast<float4*>(a.partials + (int64_t)pidx * kPartialStride);
  dst[0] = make_float4(sum[0], sum[1], sum[2], sum[3]);
  dst[1] = make_float4(sum[4], sum[5], sum[6], sum[7]);
  dst[2] = make_float4(sum[8], 0.f, 0.f, 0.f);
}

// Zero gradients for the pair of list position j (a splat no pixel reached).
__device__ __forceinline__ void zero_pair(const BwdArgs& a, int64_t vbase, uint32_t j, const TileCoords& tc) {
  const uint32_t g = a.vals[j];
  if (g >= a.n) return;
  const int64_t gi = vbase + g;
  const uint32_t pidx = a.pair_off[gi] + rect_index(a.rect[gi], tc.tx, tc.ty);
  if ((int64_t)pidx >= a.cap) {
    atomicOr(&a.counts[2], 2u);
    return;
  }
  float4* dst = reinterpret_cast<float4*>(a.partials + (int64_t)pidx * kPartialStride);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  dst[0] = z; dst[1] = z; dst[2] = z;
}

// Warp sum of 9 values per lane with 14 shuffles instead of 45: values 0-7
// are reduced by halving exchanges (each step a lane keeps half of what it
// carries and sends the other half to its partner), value 8 by a plain
// butterfly.  On return lane l holds the total of value idx(l) in s8 where
// idx(l) = 4 [l & 16] + 2 [l & 8] + [l & 4] (lanes 0, 4, ..., 28 cover 0-7),
// and every lane holds the total of value 8 in t8.
__device__ __forceinline__ void warp_sum9(const float (&d)[kPartialValues], int lane, float& s8,
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

// Chain rule from dL/dalpha to the splat's opacity and to dp = dL/dpower
// (none while alpha is clamped at its maximum).  The mean and conic
// gradients are linear in dp with coefficients from the pixel offset and the
// conic, so a pixel adds only the moments dx dp, dy dp, dx^2 dp, dx dy dp,
// dy^2 dp to d[0..4]; store_pair applies the conic once per (tile, splat).
__device__ __forceinline__ void alpha_grad(const Eval& e, float dal, float (&d)[kPartialValues]) {
  if (e.raw <= kAlphaMax) {
    d[5] += dal * e.ex;                  // d alpha / d opacity = exp(power)
    const float dp = dal * e.alpha;      // d alpha / d power = alpha
    const float xp = e.dx * dp, yp = e.dy * dp;
    d[0] += xp;
    d[1] += yp;
    d[2] += e.dx * xp;
    d[3] += e.dy * xp;
    d[4] += e.dy * yp;
  }
}

// Gradient contribution of one blended splat at one pixel, walking back to
// front: T is the transmittance behind the splat on entry and in front of it
// on return; acc is the colour behind it (background included).
__device__ __forceinline__ void splat_grad(const Eval& e, const float4 col, float g0,
                                           float g1, float g2, float ga, float Tfinal, float& T,
                                           float& acc0, float& acc1, float& acc2,
                                           float (&d)[kPartialValues]) {
  // 1 - alpha >= 0.01: one approximate reciprocal (relative error ~1e-7)
  // serves the transmittance recovery and the suffix terms
  const float rom = __fdividef(1.f, 1.f - e.alpha);
  const float Tb = T * rom;
  const float w = e.alpha * Tb;
  d[6] += g0 * w; d[7] += g1 * w; d[8] += g2 * w;
  const float dal = g0 * (col.x * Tb - acc0 * rom) + g1 * (col.y * Tb - acc1 * rom) +
                    g2 * (col.z * Tb - acc2 * rom) + ga * Tfinal * rom;
  acc0 += col.x * w; acc1 += col.y * w; acc2 += col.z * w;
  alpha_grad(e, dal, d);
  T = Tb;
}

// The single-pass form walks front to back with T, the transmittance in
// front of the splat.  rem, the colour still to come behind the splat
// (background included, the forward image minus the colour composited so
// far), enters the gradient only through g . rem, so the pixel carries that
// one number, R = g . rem, and drops each blended splat's share from it.
// dL/dalpha = T (g . c) - (g . rem) / (1 - alpha): the colour behind the
// splat seen through it is T S = rem / (1 - alpha).
//
// One pixel's step of the single-pass backward without branches: the splat
// test (as splat_alpha), the stop test, and the gradient contribution with
// alpha, exp(power) and the weight masked to zero when the pixel does not
// blend the splat, so that a contribution is exactly zero then and the
// transmittance and g . rem stay.  ACC = false writes the contribution into
// d (the first pixel), true adds it (the second), so the partials need no
// zeroing per splat.  Returns whether the pixel blended the splat; *done is
// set when it stops there.
template <bool ACC>
__device__ __forceinline__ bool pixel_step_front(const XTerms& x, const float4 g, const float4 g2, float ly,
                                                 const float4 col, float g0, float g1, float g2c, float& T,
                                                 float& R, bool& done, float (&d)[kPartialValues]) {
  const float dx = x.dx, dy = __fsub_rn(g.y, ly);
  const float p = __fmaf_rn(dy, __fmaf_rn(g2.x, dy, x.b2dx), x.a2dx2);
  const bool hit = !done && fabsf(dx) <= g2.w && fabsf(dy) <= g2.w && p <= 0.f && p >= g2.y;
  // a power above zero fails the test; its exponential (up to +inf) is masked
  const float ex0 = ex2_approx(p);
  const float raw0 = __fmul_rn(g2.z, ex0);
  const float alpha0 = fminf(kAlphaMax, raw0);
  const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha0));
  const bool stop = hit && Tn < kTransMin;
  const bool blend = hit && !stop;
  done = done || stop;
  const float alpha = blend ? alpha0 : 0.f;
  // no opacity / power gradient while alpha is clamped at its maximum;
  // unclamped, d alpha / d power = alpha = opacity * exp(power), the same
  // product as raw0
  const float exg = blend && raw0 <= kAlphaMax ? ex0 : 0.f;
  const float w = alpha * T;
  const float gc = g0 * col.x + g1 * col.y + g2c * col.z;
  R -= gc * w;
  const float rom = __fdividef(1.f, 1.f - alpha);
  const float dal = gc * T - R * rom;
  const float dex = dal * exg;
  const float dp = dal * __fmul_rn(g2.z, exg);
  const float xp = dx * dp, yp = dy * dp;
  if (ACC) {
    d[0] += xp; d[1] += yp; d[2] += dx * xp; d[3] += dy * xp; d[4] += dy * yp;
    d[5] += dex; d[6] += g0 * w; d[7] += g1 * w; d[8] += g2c * w;
  } else {
    d[0] = xp; d[1] = yp; d[2] = dx * xp; d[3] = dy * xp; d[4] = dy * yp;
    d[5] = dex; d[6] = g0 * w; d[7] = g1 * w; d[8] = g2c * w;
  }
  T = blend ? Tn : T;
  return blend;
}

template <int TW>
__global__ void __launch_bounds__(kThreads) k_render_bwd(const BwdArgs a, const ViewTable vt) {
  constexpr int kBatch = kThreads;
  __shared__ float4 s_geo[kBatch], s_geo2[kBatch], s_rgb[kBatch], s_co[kBatch];
  __shared__ uint8_t s_mask[kBatch];
  __shared__ uint32_t s_wb[kWarps][kBatch / 32];
  __shared__ uint32_t s_pidx[kBatch];
  __shared__ float s_red[kBatch][kWarps][kPartialValues];
  __shared__ uint8_t s_hit[kBatch][kWarps];
  __shared__ int s_maxlast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gt = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;  // longest lists first
  const TileCoords tc = tile_coords<TW>(vt, gt);
  const ViewInfo& vi = vt.v[tc.v];
  const uint2 rg = a.ranges[gt];
  const int64_t vbase = (int64_t)tc.v * a.n;
  if (threadIdx.x == 0) s_maxlast = -1;

  // ---- 1. replay the forward: final transmittance and last blended position
  float T0 = 1.f, T1 = 1.f;
  int last0 = -1, last1 = -1;
  bool d0 = !tc.in0, d1 = !tc.in1;
  for (uint32_t start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(d0 && d1) == kThreads) break;
    const uint32_t j = start + threadIdx.x;
    if (j < rg.y)
      stage_splat<TW>(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, j, threadIdx.x, tc.ox, tc.oy, s_geo, s_geo2,
                  s_rgb, s_mask, nullptr, nullptr);
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBatch, rg.y - start);
    warp_bits<kBatch>(s_mask, cnt, warp, lane, s_wb[warp]);
    for (int q = 0; q * 32 < cnt && !(d0 && d1); ++q) {
     for (uint32_t bits = s_wb[warp][q]; bits && !(d0 && d1); bits &= bits - 1) {
      const int k = q * 32 + __ffs(bits) - 1;
      const float4 g = s_geo[k], g2 = s_geo2[k];
      const XTerms x = splat_x(g, tc.lx);
      Eval e;
      if (!d0 && splat_alpha(x, g, g2, tc.ly0, e)) {
        const float Tn = __fmul_rn(T0, __fsub_rn(1.f, e.alpha));
        if (Tn < kTransMin) d0 = true; else { T0 = Tn; last0 = (int)(start + k); }
      }
      if (!d1 && splat_alpha(x, g, g2, tc.ly1, e)) {
        const float Tn = __fmul_rn(T1, __fsub_rn(1.f, e.alpha));
        if (Tn < kTransMin) d1 = true; else { T1 = Tn; last1 = (int)(start + k); }
      }
     }
    }
  }
  __syncthreads();
  if (max(last0, last1) >= 0) atomicMax(&s_maxlast, max(last0, last1));
  __syncthreads();
  const int maxlast = s_maxlast;
  const float Tf0 = T0, Tf1 = T1;

  const int64_t np = (int64_t)vi.W * vi.H;
  const float* gimg = a.dimage + 3 * vi.pix_base;
  float g00 = 0.f, g01 = 0.f, g02 = 0.f, ga0 = 0.f, g10 = 0.f, g11 = 0.f, g12 = 0.f, ga1 = 0.f;
  if (tc.in0) {
    const int64_t pix = (int64_t)tc.py0 * vi.W + tc.px;
    g00 = gimg[pix]; g01 = gimg[np + pix]; g02 = gimg[2 * np + pix];
    if (a.dalpha) ga0 = a.dalpha[vi.pix_base + pix];
  }
  if (tc.in1) {
    const int64_t pix = (int64_t)(tc.py0 + 1) * vi.W + tc.px;
    g10 = gimg[pix]; g11 = gimg[np + pix]; g12 = gimg[2 * np + pix];
    if (a.dalpha) ga1 = a.dalpha[vi.pix_base + pix];
  }
  float a00 = Tf0 * a.bg[0], a01 = Tf0 * a.bg[1], a02 = Tf0 * a.bg[2];
  float a10 = Tf1 * a.bg[0], a11 = Tf1 * a.bg[1], a12 = Tf1 * a.bg[2];

  // pairs behind every pixel's last blended splat receive zero gradient
  for (uint32_t p = (uint32_t)(maxlast + 1) + threadIdx.x; p < rg.y; p += kThreads) zero_pair(a, vbase, p, tc);

  // ---- 2. back to front over [rg.x, maxlast]
  const int mylast = max(last0, last1);
  for (int bend = maxlast + 1; bend > (int)rg.x; bend -= kBatch) {
    const int bstart = max((int)rg.x, bend - kBatch);
    const int cnt = bend - bstart;
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint32_t j = (uint32_t)(bstart + threadIdx.x);
      stage_splat<TW>(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, j, threadIdx.x, tc.ox, tc.oy, s_geo, s_geo2,
                  s_rgb, s_mask, s_co, nullptr);
      s_pidx[threadIdx.x] = pair_slot(a, vbase, j, tc);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s_hit[threadIdx.x][w] = 0;
    }
    __syncthreads();
    warp_bits<kBatch>(s_mask, cnt, warp, lane, s_wb[warp]);
    for (int q = (cnt - 1) >> 5; q >= 0; --q) {
     for (uint32_t bits = s_wb[warp][q]; bits;) {  // highest bit first: back to front
      const int hb = 31 - __clz(bits);
      bits ^= 1u << hb;
      const int k = q * 32 + hb;
      const int pos = bstart + k;
      float d[kPartialValues];
#pragma unroll
      for (int c = 0; c < kPartialValues; ++c) d[c] = 0.f;
      bool contrib = false;
      if (pos <= mylast) {
        const float4 g = s_geo[k], g2 = s_geo2[k], col = s_rgb[k];
        const XTerms x = splat_x(g, tc.lx);
        Eval e;
        if (pos <= last0 && splat_alpha(x, g, g2, tc.ly0, e)) {
          splat_grad(e, col, g00, g01, g02, ga0, Tf0, T0, a00, a01, a02, d);
          contrib = true;
        }
        if (pos <= last1 && splat_alpha(x, g, g2, tc.ly1, e)) {
          splat_grad(e, col, g10, g11, g12, ga1, Tf1, T1, a10, a11, a12, d);
          contrib = true;
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        float s8, t8;
        int idx;
        warp_sum9(d, lane, s8, idx, t8);
        if ((lane & 3) == 0) s_red[k][warp][idx] = s8;
        if (lane == 0) {
          s_red[k][warp][8] = t8;
          s_hit[k][warp] = 1;
        }
      }
     }
    }
    __syncthreads();
    if (threadIdx.x < cnt)
      store_pair(a, s_pidx[threadIdx.x], s_red[threadIdx.x], s_hit[threadIdx.x], s_co[threadIdx.x]);
  }
}

// Shared arrays of the single-pass backward: the staged splats, the bit
// sets, and per staged splat the warps' reduced partials and which warps
// wrote them (cleared by the thread that stores the pair, so every slot is
// zero again when the next batch is staged).
template <int kBatch>
struct BwdSmem {
  float4 geo[kBatch], geo2[kBatch], rgb[kBatch];
  uint8_t mask[kBatch];
  uint32_t wb[kWarps][kBatch / 32];
  float red[kBatch][kWarps][kPartialValues];
  uint8_t hit[kBatch][kWarps];
};

// Zeroes the hit flags once, before a CTA's first tile.
template <int kBatch>
__device__ __forceinline__ void clear_hits(BwdSmem<kBatch>& sm) {
  for (int i = threadIdx.x; i < kBatch * kWarps; i += kThreads) (&sm.hit[0][0])[i] = 0;
}

// Stores the pair of list position j from staged slot k's partials: its
// pair slot and unscaled conic are read again from memory (lines the
// staging brought into L1), so no shared slot carries them from the staging
// to the store, and clears the slot's hit flags.
__device__ __forceinline__ void store_staged(const BwdArgs& a, int64_t vbase, uint32_t j, const TileCoords& tc,
                                             const float (&red)[kWarps][kPartialValues], uint8_t (&hit)[kWarps]) {
  const uint32_t g = a.vals[j];
  if (g < a.n) {
    const int64_t gi = vbase + g;
    const uint32_t pidx = a.pair_off[gi] + rect_index(a.rect[gi], tc.tx, tc.ty);
    store_pair(a, pidx, red, hit, a.conic[gi]);
  }
#pragma unroll
  for (int w = 0; w < kWarps; ++w) hit[w] = 0;
}

// Single front-to-back backward pass over one tile's list for the thread's
// two pixels, with upstream colour gradients g0/g1 and R0/R1 = g . (forward
// image): the colour behind splat i is the forward's output minus what has
// been composited up to and including i, so one traversal in the forward's
// order, with the forward's own decisions (same splat test, same
// transmittance products, same stop), yields every gradient without a replay
// and without recovering T by division.  Stores every pair's partials (zeros
// for pairs no pixel reached).  Two barriers per batch: after the batch's
// pixel steps, the pairs of the batch are stored by the threads from kBatch
// on (modulo the CTA) while threads [0, kBatch) stage the next batch, which
// touch different shared arrays.  The hit flags must be zero on entry.
template <int kBatch, int TW>
__device__ __forceinline__ void bwd_front_tile(const BwdArgs& a, const TileCoords& tc, const uint2 rg,
                                               const int64_t vbase, const float (&gp0)[3], const float (&gp1)[3],
                                               float R0, float R1, BwdSmem<kBatch>& sm) {
  static_assert(kBatch <= kThreads, "one staged splat per thread");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float g00 = gp0[0], g01 = gp0[1], g02 = gp0[2], g10 = gp1[0], g11 = gp1[1], g12 = gp1[2];
  const int ss = (int)((threadIdx.x + kThreads - kBatch) % kThreads);  // the slot this thread stores
  float T0 = 1.f, T1 = 1.f;
  bool d0 = !tc.in0, d1 = !tc.in1;
  uint32_t start = rg.x;
  // the first barrier also ends the previous phase's reads of the staging slots
  int ndone = __syncthreads_count(d0 && d1);
  if (ndone < kThreads && start < rg.y) {
    int cnt = (int)min((uint32_t)kBatch, rg.y - start);
    for (;;) {
      if (threadIdx.x < cnt) {
        const uint32_t j = start + threadIdx.x;
        if (2 * ndone < kThreads && j + kBatch < rg.y)
          prefetch_splat(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, j + kBatch);
        stage_splat<TW>(a.xy, a.conic, a.rgb, a.vals, a.n, vbase, j, threadIdx.x, tc.ox, tc.oy, sm.geo, sm.geo2,
                        sm.rgb, sm.mask, nullptr, nullptr);
        // the pair slot's inputs, read by the store after this batch
        const uint32_t g = a.vals[j];
        if (g < a.n) {
          prefetch_l1(a.pair_off + vbase + g);
          prefetch_l1(a.rect + vbase + g);
        }
      }
      __syncthreads();
      warp_bits<kBatch>(sm.mask, cnt, warp, lane, sm.wb[warp]);
      bool live = true;
      for (int q = 0; q * 32 < cnt && live; ++q) {
       for (uint32_t bits = sm.wb[warp][q]; bits; bits &= bits - 1) {  // warp-uniform
        if (__all_sync(0xffffffffu, d0 && d1)) {  // the warp's pixels are done
          live = false;
          break;
        }
        const int k = q * 32 + __ffs(bits) - 1;
        float d[kPartialValues];
        const float4 g = sm.geo[k], g2 = sm.geo2[k], col = sm.rgb[k];
        const XTerms x = splat_x(g, tc.lx);
        bool contrib = pixel_step_front<false>(x, g, g2, tc.ly0, col, g00, g01, g02, T0, R0, d0, d);
        contrib |= pixel_step_front<true>(x, g, g2, tc.ly1, col, g10, g11, g12, T1, R1, d1, d);
        if (__any_sync(0xffffffffu, contrib)) {
          float s8, t8;
          int idx;
          warp_sum9(d, lane, s8, idx, t8);
          if ((lane & 3) == 0) sm.red[k][warp][idx] = s8;
          if (lane == 0) {
            sm.red[k][warp][8] = t8;
            sm.hit[k][warp] = 1;
          }
        }
       }
      }
      // every warp is past this batch's pixel steps: its partials are
      // complete and the staging slots are free
      ndone = __syncthreads_count(d0 && d1);
      if (ss < cnt) store_staged(a, vbase, start + ss, tc, sm.red[ss], sm.hit[ss]);
      start += kBatch;
      if (ndone == kThreads || start >= rg.y) break;
      cnt = (int)min((uint32_t)kBatch, rg.y - start);
    }
  }
  // pairs past the batch where every pixel of the tile had stopped
  for (uint32_t p = start + threadIdx.x; p < rg.y; p += kThreads) zero_pair(a, vbase, p, tc);
}

// Single front-to-back backward, for losses on the image alone (the forward's
// image and the loss gradient read from memory).
template <int kBatch, int TW>
__global__ void __launch_bounds__(kThreads) k_render_bwd_front(const BwdArgs a, const ViewTable vt) {
  __shared__ BwdSmem<kBatch> sm;
  clear_hits(sm);  // ordered before their first use by the backward's first barrier
  const int gt = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;  // longest lists first
  const TileCoords tc = tile_coords<TW>(vt, gt);
  const ViewInfo& vi = vt.v[tc.v];
  const uint2 rg = a.ranges[gt];
  const int64_t vbase = (int64_t)tc.v * a.n;

  const int64_t np = (int64_t)vi.W * vi.H;
  const float* gimg = a.dimage + 3 * vi.pix_base;
  const float* cimg = a.image + 3 * vi.pix_base;
  float g0[3] = {0.f, 0.f, 0.f}, g1[3] = {0.f, 0.f, 0.f};
  float R0 = 0.f, R1 = 0.f;  // g . (colour still to come), per pixel
  if (tc.in0) {
    const int64_t pix = (int64_t)tc.py0 * vi.W + tc.px;
    g0[0] = gimg[pix]; g0[1] = gimg[np + pix]; g0[2] = gimg[2 * np + pix];
    R0 = g0[0] * cimg[pix] + g0[1] * cimg[np + pix] + g0[2] * cimg[2 * np + pix];
  }
  if (tc.in1) {
    const int64_t pix = (int64_t)(tc.py0 + 1) * vi.W + tc.px;
    g1[0] = gimg[pix]; g1[1] = gimg[np + pix]; g1[2] = gimg[2 * np + pix];
    R1 = g1[0] * cimg[pix] + g1[1] * cimg[np + pix] + g1[2] * cimg[2 * np + pix];
  }
  bwd_front_tile<kBatch, TW>(a, tc, rg, vbase, g0, g1, R0, R1, sm);
}

// ---------------------------------------------------------------------------
// The fused per-tile training pass: one persistent launch over every
// (view, tile) item of all views.  Each CTA takes items from a device counter
// (one atomicAdd per item, in `order`: longest lists first, or view-major)
// and for each runs the composite, the image loss of its pixels (L1 or mean
// squared error against the target, over all views' pixels and channels) and
// the single front-to-back backward, with the composite's colour held in
// registers in between (nothing per pixel goes through memory but the image
// written out).  Items never wait for one another: every tile list is
// complete when the launch starts, so no CTA spins.  Per tile the loss terms
// of its pixels are summed in a fixed order; the last CTA to finish (a ticket
// counter) sums the tiles in tile order, so the loss is deterministic.
// ---------------------------------------------------------------------------
struct FusedArgs {
  FwdArgs f;                // composite: splats, lists, background, image, alpha
  BwdArgs b;                // backward: splats, lists, pair slots, partials
  const uint32_t* order;    // item -> global tile (nullptr: item = tile)
  const float* target;      // [3 * pixels], layout of the image
  float inv_count;          // 1 / (3 * pixels of all views)
  float* tile_loss;         // [tiles] loss terms summed per tile
  uint32_t* queue;          // [0] next item, [1] CTAs finished (zero at launch)
  float* loss;              // mean loss (one float)
  int32_t tiles;
};

template <int kBatch, int TW, int LOSS>
__global__ void __launch_bounds__(kThreads) k_render_fused(const FusedArgs a, const ViewTable vt) {
  __shared__ BwdSmem<kBatch> sm;
  __shared__ int s_item;
  __shared__ float s_red[kWarps];
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  clear_hits(sm);  // ordered before their first use by the barrier below
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.queue[0], 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= a.tiles) break;
    const int gt = a.order ? (int)a.order[item] : item;
    const TileCoords tc = tile_coords<TW>(vt, gt);
    const ViewInfo& vi = vt.v[tc.v];
    const uint2 rg = a.f.ranges[gt];
    const int64_t vbase = (int64_t)tc.v * a.f.n;
    // 1. composite
    float T0, T1, cc0[3], cc1[3];
    CountState cs;
    composite_tile<false, kBatch, TW>(a.f, tc, rg, vbase, sm.geo, sm.geo2, sm.rgb, sm.mask, sm.wb[warp], T0, T1,
                                      cc0, cc1, cs);
    // 2. image, loss terms and dL/dimage per pixel
    const int64_t np = (int64_t)vi.W * vi.H;
    float* img = a.f.image + 3 * vi.pix_base;
    const float* tgt = a.target + 3 * vi.pix_base;
    // (the same expressions as gs_render_fwd, gs_image_loss and the
    // single-pass backward's set-up, so the two paths give the same bits)
    float g0[3] = {0.f, 0.f, 0.f}, g1[3] = {0.f, 0.f, 0.f};
    float R0 = 0.f, R1 = 0.f, lsum = 0.f;
    if (tc.in0) {
      const int64_t pix = (int64_t)tc.py0 * vi.W + tc.px;
      float out[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        out[c] = cc0[c] + T0 * a.f.bg[c];
        img[c * np + pix] = out[c];
        const float d = out[c] - tgt[c * np + pix];
        if (LOSS == 0) {
          lsum += fabsf(d);
          g0[c] = d > 0.f ? a.inv_count : (d < 0.f ? -a.inv_count : 0.f);
        } else {
          lsum += d * d;
          g0[c] = 2.f * d * a.inv_count;
        }
      }
      R0 = g0[0] * out[0] + g0[1] * out[1] + g0[2] * out[2];
      if (a.f.alpha) a.f.alpha[vi.pix_base + pix] = 1.f - T0;
    }
    if (tc.in1) {
      const int64_t pix = (int64_t)(tc.py0 + 1) * vi.W + tc.px;
      float out[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        out[c] = cc1[c] + T1 * a.f.bg[c];
        img[c * np + pix] = out[c];
        const float d = out[c] - tgt[c * np + pix];
        if (LOSS == 0) {
          lsum += fabsf(d);
          g1[c] = d > 0.f ? a.inv_count : (d < 0.f ? -a.inv_count : 0.f);
        } else {
          lsum += d * d;
          g1[c] = 2.f * d * a.inv_count;
        }
      }
      R1 = g1[0] * out[0] + g1[1] * out[1] + g1[2] * out[2];
      if (a.f.alpha) a.f.alpha[vi.pix_base + pix] = 1.f - T1;
    }
    // the tile's loss terms in a fixed order: lanes by a butterfly, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) s_red[warp] = lsum;
    // 3. backward (its first barrier also orders s_red and s_item)
    bwd_front_tile<kBatch, TW>(a.b, tc, rg, vbase, g0, g1, R0, R1, sm);
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t += s_red[w];
      a.tile_loss[gt] = t;
    }
  }
  // ticket: the last CTA to finish sums the tiles' loss terms in tile order
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&a.queue[1], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float t = 0.f;
  for (int i = threadIdx.x; i < a.tiles; i += kThreads) t += __ldcg(&a.tile_loss[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) s_red[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sum += s_red[w];
    *a.loss = sum * a.inv_count;
  }
}

// Calls f(std::integral_constant<int, TW>) for the view table's tile width.
template <class F>
void with_tile_width(const ViewTable& vt, F&& f) {
  switch (vt.tw) {
    case 8: f(std::integral_constant<int, 8>()); break;
    case 32: f(std::integral_constant<int, 32>()); break;
    default: f(std::integral_constant<int, 16>()); break;
  }
}

}  // namespace

gs_status launch_render_fwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, float* image, float* alpha, cudaStream_t s) {
  FwdArgs a;
  a.order = (cfg.schedule & kSchedFwdLongestFirst) ? bins.tile_order : nullptr;
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
  const uint32_t batch = (cfg.schedule >> kSchedFwdBatchShift) & 3u;
  with_tile_width(vt, [&](auto tw) {
    constexpr int TW = decltype(tw)::value;
    switch (batch) {
      case 1: k_render_fwd<false, 64, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt, nullptr); break;
      case 2: k_render_fwd<false, 256, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt, nullptr); break;
      default: k_render_fwd<false, 128, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt, nullptr); break;
    }
  });
  return check_launch("k_render_fwd");
}

gs_status launch_render_stats(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                              unsigned long long* stats, cudaStream_t s) {
  FwdArgs a;
  a.order = nullptr;
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
  if (cudaMemsetAsync(stats, 0, 5 * sizeof(unsigned long long), s) != cudaSuccess) return check_launch("stats");
  if (vt.total_tiles == 0) return GS_OK;
  with_tile_width(vt, [&](auto tw) {
    constexpr int TW = decltype(tw)::value;
    k_render_fwd<true, 128, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt, stats);
  });
  return check_launch("k_render_fwd<count>");
}

static BwdArgs bwd_args(const gs_splats& sp, const gs_bins& bins, const gs_raster_cfg& cfg, const float* dimage,
                        const float* dalpha, const float* image, float* partials, bool longest_first) {
  BwdArgs a;
  a.order = longest_first ? bins.tile_order : nullptr;
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
  a.image = image;
  a.partials = partials;
  return a;
}

gs_status launch_render_bwd(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                            const gs_raster_cfg& cfg, const float* dimage, const float* dalpha,
                            const float* image, float* partials, cudaStream_t s) {
  const BwdArgs a = bwd_args(sp, bins, cfg, dimage, dalpha, image, partials,
                             (cfg.schedule & kSchedBwdLongestFirst) != 0);
  if (vt.total_tiles == 0) return GS_OK;
  if (image && !dalpha) {
    const bool b64 = ((cfg.schedule >> kSchedBwdBatchShift) & 3u) == 1;
    with_tile_width(vt, [&](auto tw) {
      constexpr int TW = decltype(tw)::value;
      if (b64)
        k_render_bwd_front<64, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt);
      else
        k_render_bwd_front<128, TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt);
    });
    return check_launch("k_render_bwd_front");
  }
  with_tile_width(vt, [&](auto tw) {
    constexpr int TW = decltype(tw)::value;
    k_render_bwd<TW><<<vt.total_tiles, kThreads, 0, s>>>(a, vt);
  });
  return check_launch("k_render_bwd");
}

// Resident CTAs of a kernel on the current device (occupancy x SMs), cached
// per device and kernel: the persistent grid size.
template <class K>
int persistent_grid(K kernel, size_t slot) {
  constexpr int kDev = 64, kSlots = 64;
  static int cache[kDev][kSlots] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev || slot >= (size_t)kSlots) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev][slot] == 0) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess)
      return 0;
    cache[dev][slot] = std::max(1, sms * std::max(1, per_sm));
  }
  return cache[dev][slot];
}

gs_status launch_render_fused(const gs_splats& sp, const gs_bins& bins, const ViewTable& vt,
                              const gs_raster_cfg& cfg, const float* target, int loss_kind, float* image,
                              float* alpha, float* loss, float* partials, float* tile_loss, uint32_t* queue,
                              cudaStream_t s) {
  FusedArgs a;
  a.f.order = nullptr;
  a.f.xy = reinterpret_cast<const float4*>(sp.xy);
  a.f.conic = reinterpret_cast<const float4*>(sp.conic);
  a.f.rgb = reinterpret_cast<const float4*>(sp.rgb);
  a.f.vals = bins.vals;
  a.f.ranges = reinterpret_cast<const uint2*>(bins.ranges);
  a.f.counts = bins.counts;
  a.f.n = sp.n;
  for (int c = 0; c < 3; ++c) a.f.bg[c] = cfg.bg[c];
  a.f.image = image;
  a.f.alpha = alpha;
  a.b = bwd_args(sp, bins, cfg, nullptr, nullptr, nullptr, partials, false);
  a.order = (cfg.schedule & GS_SCHED_FUSED_LONGEST_FIRST) ? bins.tile_order : nullptr;
  a.target = target;
  int64_t pixels = 0;
  for (int v = 0; v < vt.views; ++v) pixels += (int64_t)vt.v[v].W * vt.v[v].H;
  a.inv_count = 1.0f / (float)(3 * pixels);
  a.tile_loss = tile_loss;
  a.queue = queue;
  a.loss = loss;
  a.tiles = vt.total_tiles;
  if (cudaMemsetAsync(queue, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return check_launch("fused queue");
  if (vt.total_tiles == 0) {
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return check_launch("fused loss");
    return GS_OK;
  }
  const uint32_t bsel = (cfg.schedule >> kSchedFusedBatchShift) & 3u;  // 0: 128, 1: 64, 2: 32
  bool ok = true;
  with_tile_width(vt, [&](auto tw) {
    constexpr int TW = decltype(tw)::value;
    auto go = [&](auto kernel, size_t slot) {
      const int g = std::min(persistent_grid(kernel, slot), vt.total_tiles);
      if (g <= 0) { ok = false; return; }
      kernel<<<g, kThreads, 0, s>>>(a, vt);
    };
    const size_t base = (TW == 8 ? 0 : TW == 16 ? 6 : 12);
    if (loss_kind == 0) {
      if (bsel == 1) go(k_render_fused<64, TW, 0>, base + 0);
      else if (bsel == 2) go(k_render_fused<32, TW, 0>, base + 1);
      else go(k_render_fused<128, TW, 0>, base + 2);
    } else {
      if (bsel == 1) go(k_render_fused<64, TW, 1>, base + 3);
      else if (bsel == 2) go(k_render_fused<32, TW, 1>, base + 4);
      else go(k_render_fused<128, TW, 1>, base + 5);
    }
  });
  if (!ok) return fail(GS_ERR_CUDA, "k_render_fused: occupancy query failed");
  return check_launch("k_render_fused");
}

}  // namespace gs
