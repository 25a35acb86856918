// Per-Gaussian backward: sums each (view, Gaussian)'s per-tile partial
// gradients in a fixed order, then applies the chain rule of the projection
// to the parameters (means, log-scales, quaternion, opacity logit, SH) and to
// each view's pose for the left perturbation T <- Exp(xi) T, xi = (v, omega).
//
// k_pair_sum, one thread per (view, Gaussian), sums its per-tile partials in
// list order (pairs of one (view, Gaussian) are contiguous) into three
// planes; then two kernels, one thread per Gaussian, all views in one
// fixed-order loop:
//   k_project_bwd  pixel-space mean, conic, opacity -> means, log-scales,
//                  quaternion, opacity logit, pose (t and rotation terms);
//   k_sh_bwd       colour -> SH coefficients and, through the view
//                  direction, the means and the pose translation;
//   k_sh_bwd_adam  the same, with the Adam step of every parameter of the
//                  Gaussian applied once its gradients are complete (the
//                  training step's form).
// A thread first loads every view's pair count and offset (a bit set of the
// views that see its Gaussian), so a view loop waits on memory only in those
// views.  Pose gradients are reduced per warp (shuffles, fixed tree), then
// over fixed chunks of warps and the chunks in a fixed order: deterministic,
// no atomics.  The pair sum is its own kernel so that its scattered loads run
// at full occupancy: the chain-rule kernels hold ~120 registers per thread.
// The kernels of a backward are chained as programmatic dependent launches.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

struct GradArgs {
  const float4* means4;
  const float4* scale_opa;
  const float4* quat;
  const float* sh;
  int64_t n;
  int64_t sh_stride;
  const float* poses;
  int clamp_j;
  const uint32_t* touched;
  const uint32_t* aux;
  const uint32_t* pair_off;
  const uint32_t* counts;  // [3] = pairs in the lists (min(K, capacity))
  const float* partials;
  float4* g_means4;
  float4* g_scale_opa;
  float4* g_quat;
  float* g_sh;
  int64_t g_sh_stride;
  float* pose_a;         // [V][warps][6] from k_project_bwd
  float* pose_b;         // [V][warps][3] from k_sh_bwd (translation part)
  float4* gsum;          // [2][V][n]: (dmx, dmy, dA, dB), (dC, dopacity, -, -) per visible (view, Gaussian)
  float4* drgb;          // [V][n] summed colour gradient of each visible (view, Gaussian)
};

// Warp sum of K values; lane 0 writes them to out[0..K).
template <int K>
__device__ __forceinline__ void warp_store_sum(float (&x)[K], float* out) {
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x[c] += __shfl_xor_sync(0xffffffffu, x[c], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int c = 0; c < K; ++c) out[c] = x[c];
  }
}

__device__ __forceinline__ bool pair_range_ok(const GradArgs& a, int64_t o, uint32_t kpairs, uint32_t& tch) {
  tch = a.touched[o];
  // pairs cut off by a capacity overflow were never rendered: skip them
  if (tch > 0 && (uint64_t)a.pair_off[o] + tch > kpairs) tch = 0;
  return tch > 0;
}

// The views (bit v) in which Gaussian i has rendered pairs (as
// pair_range_ok), with every view's count and offset loaded before any
// view's work: a per-view loop then waits for memory only in the views that
// see the Gaussian (a few of a batch's views), not twice per view.
__device__ __forceinline__ uint64_t visible_views(const GradArgs& a, int64_t i, bool valid, int views,
                                                  uint32_t kpairs) {
  uint64_t m = 0;
  if (!valid) return m;
#pragma unroll 8
  for (int v = 0; v < views; ++v) {
    const int64_t o = (int64_t)v * a.n + i;
    const uint32_t tch = a.touched[o], off = a.pair_off[o];
    if (tch > 0 && (uint64_t)off + tch <= kpairs) m |= 1ull << v;
  }
  return m;
}

// Sum of each visible (view, Gaussian)'s per-tile partials, in a fixed
// order.  A (view, Gaussian) with at most kWideSegment pairs is summed by its
// own thread in list order, four pairs per step so that their twelve loads
// are in flight together.  Wider ones (a splat near the camera can cover
// thousands of tiles) are summed by the whole warp, one at a time: lane l
// takes pairs l, l + 32, ... in order, then a fixed butterfly combines the
// lanes, so the warp's time is not set by one thread walking a long segment.
constexpr uint32_t kWideSegment = 16;

__global__ void __launch_bounds__(256, 6) k_pair_sum(const GradArgs a, int64_t m) {
  chain_enter();
  const int64_t o = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t tch = 0;
  const bool live = o < m && pair_range_ok(a, o, a.counts[3], tch);
  const uint32_t off = live ? a.pair_off[o] : 0u;
  const bool wide = live && tch > kWideSegment;
  if (live && !wide) {
    const float4* pp = reinterpret_cast<const float4*>(a.partials + (int64_t)off * kPartialStride);
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
    float s2 = 0.f;
    uint32_t k = 0;
    for (; k + 4 <= tch; k += 4) {
      float4 p[12];
#pragma unroll
      for (int j = 0; j < 12; ++j) p[j] = pp[3 * k + j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        s0.x += p[3 * j].x; s0.y += p[3 * j].y; s0.z += p[3 * j].z; s0.w += p[3 * j].w;
        s1.x += p[3 * j + 1].x; s1.y += p[3 * j + 1].y; s1.z += p[3 * j + 1].z; s1.w += p[3 * j + 1].w;
        s2 += p[3 * j + 2].x;
      }
    }
    for (; k < tch; ++k) {
      const float4 p0 = pp[3 * k], p1 = pp[3 * k + 1], p2 = pp[3 * k + 2];
      s0.x += p0.x; s0.y += p0.y; s0.z += p0.z; s0.w += p0.w;
      s1.x += p1.x; s1.y += p1.y; s1.z += p1.z; s1.w += p1.w;
      s2 += p2.x;
    }
    a.gsum[o] = s0;
    a.gsum[m + o] = make_float4(s1.x, s1.y, 0.f, 0.f);
    a.drgb[o] = make_float4(s1.z, s1.w, s2, 0.f);
  }
  unsigned pending = __ballot_sync(0xffffffffu, wide);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const uint32_t cnt = __shfl_sync(0xffffffffu, tch, src);
    const uint32_t base = __shfl_sync(0xffffffffu, off, src);
    const float4* pp = reinterpret_cast<const float4*>(a.partials + (int64_t)base * kPartialStride);
    float acc[kPartialValues];
#pragma unroll
    for (int c = 0; c < kPartialValues; ++c) acc[c] = 0.f;
    uint32_t k = lane;
    for (; k + 96 < cnt; k += 128) {
      float4 p[12];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        p[3 * j] = pp[3 * (k + 32 * j)];
        p[3 * j + 1] = pp[3 * (k + 32 * j) + 1];
        p[3 * j + 2] = pp[3 * (k + 32 * j) + 2];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[0] += p[3 * j].x; acc[1] += p[3 * j].y; acc[2] += p[3 * j].z; acc[3] += p[3 * j].w;
        acc[4] += p[3 * j + 1].x; acc[5] += p[3 * j + 1].y; acc[6] += p[3 * j + 1].z; acc[7] += p[3 * j + 1].w;
        acc[8] += p[3 * j + 2].x;
      }
    }
    for (; k < cnt; k += 32) {
      const float4 p0 = pp[3 * k], p1 = pp[3 * k + 1], p2 = pp[3 * k + 2];
      acc[0] += p0.x; acc[1] += p0.y; acc[2] += p0.z; acc[3] += p0.w;
      acc[4] += p1.x; acc[5] += p1.y; acc[6] += p1.z; acc[7] += p1.w;
      acc[8] += p2.x;
    }
#pragma unroll
    for (int c = 0; c < kPartialValues; ++c) {
#pragma unroll
      for (int x = 16; x > 0; x >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], x);
    }
    if (lane == src) {
      a.gsum[o] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      a.gsum[m + o] = make_float4(acc[4], acc[5], 0.f, 0.f);
      a.drgb[o] = make_float4(acc[6], acc[7], acc[8], 0.f);
    }
  }
}

// ONE (a single view): the same code bounded to 3 CTAs per SM (85
// registers) instead of 2 (its per-view loop runs once).
template <int DEG, bool ONE>
__global__ void __launch_bounds__(kGradBlock, ONE ? 3 : 2) k_project_bwd(const GradArgs a, const ViewTable vt) {
  chain_enter();
  const int64_t i = (int64_t)blockIdx.x * kGradBlock + threadIdx.x;
  const bool valid = i < a.n;
  const int64_t warp_id = i >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kGradBlock / 32);

  float4 mu = make_float4(0.f, 0.f, 0.f, 0.f), so = mu, q4 = mu;
  if (valid) { mu = a.means4[i]; so = a.scale_opa[i]; q4 = a.quat[i]; }
  // quaternion, rotation, scales (view independent)
  const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
  const float qi = valid ? 1.0f / qn : 0.f;
  const float qw = q4.x * qi, qx = q4.y * qi, qy = q4.z * qi, qz = q4.w * qi;
  float Rq[9];
  quat_rot(qw, qx, qy, qz, Rq);
  const float s[3] = {expf(so.x), expf(so.y), expf(so.z)};
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
  const float opa = 1.0f / (1.0f + expf(-so.w));

  float gmu[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  float gol = 0.f;
  float gRq[9];  // gradient w.r.t. the rotation matrix entries, over views
#pragma unroll
  for (int k = 0; k < 9; ++k) gRq[k] = 0.f;
  float gsc[3] = {0.f, 0.f, 0.f};

  if (vt.views == 1 && valid) {
    // one view: its summed gradients requested with the pair count, not
    // after it
    prefetch_l1(a.gsum + i);
    prefetch_l1(a.gsum + a.n + i);
    prefetch_l1(a.aux + i);
  }
  const uint64_t vmask = visible_views(a, i, valid, vt.views, a.counts[3]);
  // the summed gradients of the views that see the Gaussian, fetched into L1
  // while the first views are worked on
  if (vt.views > 1) {
    for (uint64_t mm = vmask; mm; mm &= mm - 1) {
      const int64_t o = (int64_t)(__ffsll((long long)mm) - 1) * a.n + i;
      prefetch_l1(a.gsum + o);
      prefetch_l1(a.gsum + (int64_t)vt.views * a.n + o);
      prefetch_l1(a.aux + o);
    }
  }
  for (int v = 0; v < vt.views; ++v) {
    float pv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t o = (int64_t)v * a.n + i;
    if ((vmask >> v) & 1ull) {
      const ViewInfo vi = vt.v[v];
      const uint32_t auxb = a.aux[o];
      // ---- this (view, Gaussian)'s summed pixel-space gradients
      const float4 ga4 = a.gsum[o], gb4 = a.gsum[(int64_t)vt.views * a.n + o];
      const float G[6] = {ga4.x, ga4.y, ga4.z, ga4.w, gb4.x, gb4.y};
      const float* P = a.poses + 12 * v;
      const float R[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]};
      const float tc[3] = {P[3], P[7], P[11]};
      float t[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) t[r] = R[3 * r] * mu.x + R[3 * r + 1] * mu.y + R[3 * r + 2] * mu.z + tc[r];
      const float iz = 1.0f / t[2], iz2 = iz * iz;
      float dt[3] = {0.f, 0.f, 0.f};

      // ---- opacity
      gol += G[5] * opa * (1.f - opa);

      // ---- pixel-space mean m = f t_xy / t_z + c
      dt[0] += G[0] * vi.fx * iz;
      dt[1] += G[1] * vi.fy * iz;
      dt[2] -= (G[0] * vi.fx * t[0] + G[1] * vi.fy * t[1]) * iz2;

      // ---- conic -> 2D covariance -> (J, R, Rq, s)
      float u = t[0] * iz, w = t[1] * iz;
      const bool cx = (auxb & 8u) != 0, cy = (auxb & 16u) != 0;
      if (a.clamp_j) {
        const float limx = kGuard * 0.5f * (float)vi.W / vi.fx;
        const float limy = kGuard * 0.5f * (float)vi.H / vi.fy;
        if (cx) u = u > 0.f ? limx : -limx;
        if (cy) w = w > 0.f ? limy : -limy;
      }
      const float J00 = vi.fx * iz, J02 = -vi.fx * u * iz;
      const float J11 = vi.fy * iz, J12 = -vi.fy * w * iz;
      const float T0[3] = {J00 * R[0] + J02 * R[6], J00 * R[1] + J02 * R[7], J00 * R[2] + J02 * R[8]};
      const float T1[3] = {J11 * R[3] + J12 * R[6], J11 * R[4] + J12 * R[7], J11 * R[5] + J12 * R[8]};
      float P0[3], P1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        P0[c] = T0[0] * M[c] + T0[1] * M[3 + c] + T0[2] * M[6 + c];
        P1[c] = T1[0] * M[c] + T1[1] * M[3 + c] + T1[2] * M[6 + c];
      }
      const float ca = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2] + kDilation;
      const float cb = P0[0] * P1[0] + P0[1] * P1[1] + P0[2] * P1[2];
      const float cc = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2] + kDilation;
      const float det = ca * cc - cb * cb;
      const float id = 1.0f / det, id2 = id * id;
      const float gA = G[2], gB = G[3], gC = G[4];
      const float ga = (-cc * cc * gA + cb * cc * gB - cb * cb * gC) * id2;
      const float gb = (2.f * cb * cc * gA - (ca * cc + cb * cb) * gB + 2.f * ca * cb * gC) * id2;
      const float gc = (-cb * cb * gA + ca * cb * gB - ca * ca * gC) * id2;
      float dP0[3], dP1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dP0[c] = 2.f * ga * P0[c] + gb * P1[c];
        dP1[c] = gb * P0[c] + 2.f * gc * P1[c];
      }
      // P = T M:  dT = dP M^T,  dM = T^T dP
      float dT0[3], dT1[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        dT0[r] = dP0[0] * M[3 * r] + dP0[1] * M[3 * r + 1] + dP0[2] * M[3 * r + 2];
        dT1[r] = dP1[0] * M[3 * r] + dP1[1] * M[3 * r + 1] + dP1[2] * M[3 * r + 2];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float dm = T0[r] * dP0[c] + T1[r] * dP1[c];
          gsc[c] += dm * Rq[3 * r + c];
          gRq[3 * r + c] += dm * s[c];
        }
      // T = J R (rows): dJ and the rotation-matrix gradient of the pose
      const float dJ00 = dT0[0] * R[0] + dT0[1] * R[1] + dT0[2] * R[2];
      const float dJ02 = dT0[0] * R[6] + dT0[1] * R[7] + dT0[2] * R[8];
      const float dJ11 = dT1[0] * R[3] + dT1[1] * R[4] + dT1[2] * R[5];
      const float dJ12 = dT1[0] * R[6] + dT1[1] * R[7] + dT1[2] * R[8];
      float dR[9];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dR[c] = J00 * dT0[c];
        dR[3 + c] = J11 * dT1[c];
        dR[6 + c] = J02 * dT0[c] + J12 * dT1[c];
      }
      // J as a function of t
      dt[2] -= (dJ00 * vi.fx + dJ11 * vi.fy) * iz2;
      if (cx) {
        dt[2] += dJ02 * vi.fx * u * iz2;
      } else {
        dt[0] -= dJ02 * vi.fx * iz2;
        dt[2] += dJ02 * 2.f * vi.fx * t[0] * iz2 * iz;
      }
      if (cy) {
        dt[2] += dJ12 * vi.fy * w * iz2;
      } else {
        dt[1] -= dJ12 * vi.fy * iz2;
        dt[2] += dJ12 * 2.f * vi.fy * t[1] * iz2 * iz;
      }
      // t = R mu + t_cam
      gmu[0] += R[0] * dt[0] + R[3] * dt[1] + R[6] * dt[2];
      gmu[1] += R[1] * dt[0] + R[4] * dt[1] + R[7] * dt[2];
      gmu[2] += R[2] * dt[0] + R[5] * dt[1] + R[8] * dt[2];
      // pose: t -> t + omega x t + v ; R -> R + [omega]x R
      pv[0] = dt[0]; pv[1] = dt[1]; pv[2] = dt[2];
      pv[3] = t[1] * dt[2] - t[2] * dt[1];
      pv[4] = t[2] * dt[0] - t[0] * dt[2];
      pv[5] = t[0] * dt[1] - t[1] * dt[0];
      // N = R dR^T; d omega += (N12 - N21, N20 - N02, N01 - N10)
      float N[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          N[3 * r + c] = R[3 * r] * dR[3 * c] + R[3 * r + 1] * dR[3 * c + 1] + R[3 * r + 2] * dR[3 * c + 2];
      pv[3] += N[5] - N[7];
      pv[4] += N[6] - N[2];
      pv[5] += N[1] - N[3];
    }
    warp_store_sum<6>(pv, a.pose_a + ((int64_t)v * warps + warp_id) * 6);
  }

  if (!valid) return;
  // rotation entries -> unit quaternion -> quaternion
  const float dqw = gRq[1] * (-2.f * qz) + gRq[2] * (2.f * qy) + gRq[3] * (2.f * qz) +
                    gRq[5] * (-2.f * qx) + gRq[6] * (-2.f * qy) + gRq[7] * (2.f * qx);
  const float dqx = gRq[1] * (2.f * qy) + gRq[2] * (2.f * qz) + gRq[3] * (2.f * qy) +
                    gRq[4] * (-4.f * qx) + gRq[5] * (-2.f * qw) + gRq[6] * (2.f * qz) +
                    gRq[7] * (2.f * qw) + gRq[8] * (-4.f * qx);
  const float dqy = gRq[0] * (-4.f * qy) + gRq[1] * (2.f * qx) + gRq[2] * (2.f * qw) +
                    gRq[3] * (2.f * qx) + gRq[5] * (2.f * qz) + gRq[6] * (-2.f * qw) +
                    gRq[7] * (2.f * qz) + gRq[8] * (-4.f * qy);
  const float dqz = gRq[0] * (-4.f * qz) + gRq[1] * (-2.f * qw) + gRq[2] * (2.f * qx) +
                    gRq[3] * (2.f * qw) + gRq[4] * (-4.f * qz) + gRq[5] * (2.f * qy) +
                    gRq[6] * (2.f * qx) + gRq[7] * (2.f * qy);
  const float pr = qw * dqw + qx * dqx + qy * dqy + qz * dqz;
  gq[0] = (dqw - qw * pr) * qi;
  gq[1] = (dqx - qx * pr) * qi;
  gq[2] = (dqy - qy * pr) * qi;
  gq[3] = (dqz - qz * pr) * qi;
  a.g_means4[i] = make_float4(gmu[0], gmu[1], gmu[2], 0.f);
  a.g_scale_opa[i] = make_float4(gsc[0] * s[0], gsc[1] * s[1], gsc[2] * s[2], gol);
  a.g_quat[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
}

// SH coefficients and the view direction: for every visible view (fixed
// order), g_c Y_k(dir) for each unclamped channel c, and through dir =
// normalise(mu - centre) the means (added to k_project_bwd's) and the pose
// translation (mu - centre moves by R^T v).
template <int DEG>
__global__ void __launch_bounds__(kGradBlock) k_sh_bwd(const GradArgs a, const ViewTable vt) {
  chain_enter();
  constexpr int NC = (DEG + 1) * (DEG + 1);
  const int64_t i = (int64_t)blockIdx.x * kGradBlock + threadIdx.x;
  const bool valid = i < a.n;
  const int64_t warp_id = i >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kGradBlock / 32);
  const float4 mu = valid ? a.means4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  float gsh[3][NC];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch)
#pragma unroll
    for (int k = 0; k < NC; ++k) gsh[ch][k] = 0.f;
  float gmu[3] = {0.f, 0.f, 0.f};
  const uint64_t vmask = visible_views(a, i, valid, vt.views, a.counts[3]);
  for (int v = 0; v < vt.views; ++v) {
    float pv[3] = {0.f, 0.f, 0.f};
    const int64_t o = (int64_t)v * a.n + i;
    if ((vmask >> v) & 1ull) {
      const float4 g = a.drgb[o];
      const uint32_t auxb = a.aux[o];
      const float* P = a.poses + 12 * v;
      const float oc0 = -(P[0] * P[3] + P[4] * P[7] + P[8] * P[11]);
      const float oc1 = -(P[1] * P[3] + P[5] * P[7] + P[9] * P[11]);
      const float oc2 = -(P[2] * P[3] + P[6] * P[7] + P[10] * P[11]);
      const float wx = mu.x - oc0, wy = mu.y - oc1, wz = mu.z - oc2;
      const float inv = 1.0f / sqrtf(wx * wx + wy * wy + wz * wz);
      const float dx = wx * inv, dy = wy * inv, dz = wz * inv;
      float Y[NC];
      sh_basis<DEG>(dx, dy, dz, Y);
      const float gc[3] = {(auxb & 1u) ? 0.f : g.x, (auxb & 2u) ? 0.f : g.y, (auxb & 4u) ? 0.f : g.z};
      float dY[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) dY[k] = 0.f;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          gsh[ch][k] += gc[ch] * Y[k];
          if (k > 0) dY[k] += gc[ch] * a.sh[(int64_t)(ch * NC + k) * a.sh_stride + i];
        }
      }
      if (DEG > 0) {
        float ddx, ddy, ddz;
        sh_basis_grad<DEG>(dx, dy, dz, dY, ddx, ddy, ddz);
        const float pr = dx * ddx + dy * ddy + dz * ddz;
        const float dwx = (ddx - dx * pr) * inv, dwy = (ddy - dy * pr) * inv, dwz = (ddz - dz * pr) * inv;
        gmu[0] += dwx; gmu[1] += dwy; gmu[2] += dwz;
        pv[0] = P[0] * dwx + P[1] * dwy + P[2] * dwz;
        pv[1] = P[4] * dwx + P[5] * dwy + P[6] * dwz;
        pv[2] = P[8] * dwx + P[9] * dwy + P[10] * dwz;
      }
    }
    warp_store_sum<3>(pv, a.pose_b + ((int64_t)v * warps + warp_id) * 3);
  }
  if (!valid) return;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch)
#pragma unroll
    for (int k = 0; k < NC; ++k) a.g_sh[(int64_t)(ch * NC + k) * a.g_sh_stride + i] = gsh[ch][k];
  if (DEG > 0) {
    float4 gm = a.g_means4[i];
    gm.x += gmu[0]; gm.y += gmu[1]; gm.z += gmu[2];
    a.g_means4[i] = gm;
  }
}

// Per-parameter Adam settings of the fused form: one learning rate per lane
// of the float4 parameters and per SH plane (ch * nc + k); a parameter whose
// rate entry is marked off keeps its value and moments.
struct AdamFamilies {
  float lr4[3][4];      // means4, scale_opa, quat
  float lr_sh[48];
  uint32_t on4;         // bit f: float4 family f updated
  uint32_t on_sh;       // 1: the SH planes updated
  float b1, b2, eps, bc1, bc2;
  const int32_t* step_dev;
  const uint32_t* skip_dev;
  uint32_t* status;
  float4* p_means4;     // parameters (read and written); the chain-rule reads go through GradArgs
  float4* p_scale_opa;
  float4* p_quat;
  float* p_sh;
  int64_t p_sh_stride;
  float4 *m_means4, *m_scale_opa, *m_quat, *v_means4, *v_scale_opa, *v_quat;
  float *m_sh, *v_sh;
  int64_t mv_sh_stride;
};

__device__ __forceinline__ bool adam4(float4& p, const float4 g, float4& m, float4& v, const float (&lr)[4],
                                      float ss, const AdamFamilies& f, float rs_bc2) {
  bool ok = adam_elem(p.x, g.x, m.x, v.x, lr[0] * ss, f.b1, f.b2, f.eps, rs_bc2);
  ok &= adam_elem(p.y, g.y, m.y, v.y, lr[1] * ss, f.b1, f.b2, f.eps, rs_bc2);
  ok &= adam_elem(p.z, g.z, m.z, v.z, lr[2] * ss, f.b1, f.b2, f.eps, rs_bc2);
  ok &= adam_elem(p.w, g.w, m.w, v.w, lr[3] * ss, f.b1, f.b2, f.eps, rs_bc2);
  return ok;
}

// k_sh_bwd with the Adam update of the Gaussian fused in: once its SH
// gradients (in registers) and its means gradient (k_project_bwd's plus the
// view-direction term) are complete, every parameter of Gaussian i takes the
// Adam step of gs_adam_step (same element update, same constants), so the SH
// gradients never reach memory and the update needs no pass of its own.
// ONE (a single view): the SH gradient g_c Y_k is formed in the update from
// the view's colour gradient and basis instead of 48 accumulators (0 + g_c Y_k,
// the accumulated value's bits), which frees registers for occupancy.
template <int DEG, bool ONE>
__global__ void __launch_bounds__(kGradBlock, ONE ? 4 : 3) k_sh_bwd_adam(const GradArgs a, const ViewTable vt,
                                                            const AdamFamilies f) {
  chain_enter();
  constexpr int NC = (DEG + 1) * (DEG + 1);
  const int64_t i = (int64_t)blockIdx.x * kGradBlock + threadIdx.x;
  const bool valid = i < a.n;
  const int64_t warp_id = i >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kGradBlock / 32);
  const float4 mu = valid ? a.means4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  // several views: the 3 NC SH gradient sums live in shared memory (plane
  // pl of thread t at s_gsh[pl][t], conflict-free), not in registers
  __shared__ float s_gsh[ONE ? 1 : 3 * NC][ONE ? 1 : kGradBlock];
  float Ys[ONE ? NC : 1], gcs[3] = {0.f, 0.f, 0.f};
  if constexpr (ONE) {
#pragma unroll
    for (int k = 0; k < NC; ++k) Ys[k] = 0.f;
  } else {
#pragma unroll
    for (int pl = 0; pl < 3 * NC; ++pl) s_gsh[pl][threadIdx.x] = 0.f;
  }
  float gmu[3] = {0.f, 0.f, 0.f};
  if constexpr (ONE) {
    // one view: the chain rule reads 45 SH planes once the view is known to
    // see the Gaussian, and the update reads all 48 of every Gaussian: ask
    // for their lines in L2 at once
    if (valid) {
#pragma unroll
      for (int pl = 0; pl < 3 * NC; ++pl)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a.sh + (int64_t)pl * a.sh_stride + i)));
    }
  }
  const uint64_t vmask = visible_views(a, i, valid, vt.views, a.counts[3]);
  if constexpr (!ONE) {
    // the colour gradients of the views that see the Gaussian and its SH
    // planes, fetched into L1 ahead of the view loop
    for (uint64_t mm = vmask; mm; mm &= mm - 1) {
      const int64_t o = (int64_t)(__ffsll((long long)mm) - 1) * a.n + i;
      prefetch_l1(a.drgb + o);
      prefetch_l1(a.aux + o);
    }
    if (vmask) {
#pragma unroll
      for (int pl = 1; pl < 3 * NC; ++pl)
        if (pl % NC) prefetch_l1(a.sh + (int64_t)pl * a.sh_stride + i);
    }
  }
  for (int v = 0; v < vt.views; ++v) {
    float pv[3] = {0.f, 0.f, 0.f};
    const int64_t o = (int64_t)v * a.n + i;
    if ((vmask >> v) & 1ull) {
      const float4 g = a.drgb[o];
      const uint32_t auxb = a.aux[o];
      const float* P = a.poses + 12 * v;
      const float oc0 = -(P[0] * P[3] + P[4] * P[7] + P[8] * P[11]);
      const float oc1 = -(P[1] * P[3] + P[5] * P[7] + P[9] * P[11]);
      const float oc2 = -(P[2] * P[3] + P[6] * P[7] + P[10] * P[11]);
      const float wx = mu.x - oc0, wy = mu.y - oc1, wz = mu.z - oc2;
      const float inv = 1.0f / sqrtf(wx * wx + wy * wy + wz * wz);
      const float dx = wx * inv, dy = wy * inv, dz = wz * inv;
      float Y[NC];
      sh_basis<DEG>(dx, dy, dz, Y);
      const float gc[3] = {(auxb & 1u) ? 0.f : g.x, (auxb & 2u) ? 0.f : g.y, (auxb & 4u) ? 0.f : g.z};
      float dY[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) dY[k] = 0.f;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          if constexpr (!ONE) s_gsh[ch * NC + k][threadIdx.x] += gc[ch] * Y[k];
          if (k > 0) dY[k] += gc[ch] * a.sh[(int64_t)(ch * NC + k) * a.sh_stride + i];
        }
      }
      if constexpr (ONE) {
#pragma unroll
        for (int k = 0; k < NC; ++k) Ys[k] = Y[k];
        gcs[0] = gc[0]; gcs[1] = gc[1]; gcs[2] = gc[2];
      }
      if (DEG > 0) {
        float ddx, ddy, ddz;
        sh_basis_grad<DEG>(dx, dy, dz, dY, ddx, ddy, ddz);
        const float pr = dx * ddx + dy * ddy + dz * ddz;
        const float dwx = (ddx - dx * pr) * inv, dwy = (ddy - dy * pr) * inv, dwz = (ddz - dz * pr) * inv;
        gmu[0] += dwx; gmu[1] += dwy; gmu[2] += dwz;
        pv[0] = P[0] * dwx + P[1] * dwy + P[2] * dwz;
        pv[1] = P[4] * dwx + P[5] * dwy + P[6] * dwz;
        pv[2] = P[8] * dwx + P[9] * dwy + P[10] * dwz;
      }
    }
    warp_store_sum<3>(pv, a.pose_b + ((int64_t)v * warps + warp_id) * 3);
  }
  if (!valid || (f.skip_dev && *f.skip_dev)) return;
  float bc1 = f.bc1, bc2 = f.bc2;
  if (f.step_dev) {
    const int st = *f.step_dev + 1;
    bc1 = bias_corr(f.b1, st);
    bc2 = bias_corr(f.b2, st);
  }
  const float rs_bc2 = rsqrtf(bc2), ss = 1.f / bc1;
  bool ok = true;
  // every load of a group of parameters is issued before its updates, so the
  // memory round trips overlap (this kernel runs at a low occupancy)
  {
    float4 gm = a.g_means4[i];
    if (DEG > 0) {
      gm.x += gmu[0]; gm.y += gmu[1]; gm.z += gmu[2];
    }
    const float4 gso = a.g_scale_opa[i], gq = a.g_quat[i];
    float4 p0 = f.p_means4[i], m0 = f.m_means4[i], v0 = f.v_means4[i];
    float4 p1 = f.p_scale_opa[i], m1 = f.m_scale_opa[i], v1 = f.v_scale_opa[i];
    float4 p2 = f.p_quat[i], m2 = f.m_quat[i], v2 = f.v_quat[i];
    if (f.on4 & 1u) {
      ok &= adam4(p0, gm, m0, v0, f.lr4[0], ss, f, rs_bc2);
      f.p_means4[i] = p0; f.m_means4[i] = m0; f.v_means4[i] = v0;
    }
    if (f.on4 & 2u) {
      ok &= adam4(p1, gso, m1, v1, f.lr4[1], ss, f, rs_bc2);
      f.p_scale_opa[i] = p1; f.m_scale_opa[i] = m1; f.v_scale_opa[i] = v1;
    }
    if (f.on4 & 4u) {
      ok &= adam4(p2, gq, m2, v2, f.lr4[2], ss, f, rs_bc2);
      f.p_quat[i] = p2; f.m_quat[i] = m2; f.v_quat[i] = v2;
    }
  }
  if (f.on_sh) {
    constexpr int NP = 3 * NC, B = 8;
#pragma unroll
    for (int p0 = 0; p0 < NP; p0 += B) {
      float P[B], M[B], V[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (p0 + b >= NP) break;
        const int64_t ip = (int64_t)(p0 + b) * f.p_sh_stride + i, im = (int64_t)(p0 + b) * f.mv_sh_stride + i;
        P[b] = f.p_sh[ip];
        M[b] = f.m_sh[im];
        V[b] = f.v_sh[im];
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (p0 + b >= NP) break;
        const int pl = p0 + b;
        float gp;
        if constexpr (ONE) gp = __fadd_rn(0.f, __fmul_rn(gcs[pl / NC], Ys[pl % NC]));
        else gp = s_gsh[pl][threadIdx.x];
        ok &= adam_elem(P[b], gp, M[b], V[b], f.lr_sh[pl] * ss, f.b1, f.b2, f.eps, rs_bc2);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (p0 + b >= NP) break;
        const int64_t ip = (int64_t)(p0 + b) * f.p_sh_stride + i, im = (int64_t)(p0 + b) * f.mv_sh_stride + i;
        f.p_sh[ip] = P[b];
        f.m_sh[im] = M[b];
        f.v_sh[im] = V[b];
      }
    }
  }
  if (!ok && f.status) atomicOr(f.status, 1u);
}

constexpr int kPoseChunks = 64;

// Stage 1 of the pose sum: block (chunk j, view v) sums the per-warp partials
// of warps [j c, (j+1) c) in a fixed order and stores the 6 values in place
// of the chunk's first warp (no other block reads that chunk).
__global__ void __launch_bounds__(256) k_pose_chunks(float* __restrict__ pa, const float* __restrict__ pb,
                                                     int64_t warps, int64_t chunk) {
  chain_enter();
  __shared__ float s[256][6];
  const int v = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(warps, b0 + chunk);
  if (b0 >= warps) return;  // block-uniform
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t b = b0 + threadIdx.x; b < b1; b += 256) {
    const float* p = pa + ((int64_t)v * warps + b) * 6;
    const float* q = pb + ((int64_t)v * warps + b) * 3;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += p[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += q[c];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) s[threadIdx.x][c] = acc[c];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int c = 0; c < 6; ++c) s[threadIdx.x][c] += s[threadIdx.x + h][c];
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) pa[((int64_t)v * warps + b0) * 6 + threadIdx.x] = s[0][threadIdx.x];
}

// Stage 2: the chunks of each view in order (staged through shared memory so
// that the loads are issued together).
__global__ void __launch_bounds__(kPoseChunks) k_pose_finalize(const float* __restrict__ pa, int64_t warps,
                                                             int64_t chunk, float* __restrict__ dpose) {
  chain_enter();
  __shared__ float s[kPoseChunks][6];
  const int v = blockIdx.x, t = threadIdx.x;
  const int64_t b0 = (int64_t)t * chunk;
#pragma unroll
  for (int c = 0; c < 6; ++c) s[t][c] = b0 < warps ? pa[((int64_t)v * warps + b0) * 6 + c] : 0.f;
  __syncthreads();
  if (t < 6) {
    float acc = 0.f;
    for (int j = 0; j < kPoseChunks; ++j) acc += s[j][t];
    dpose[v * 6 + t] = acc;
  }
}

}  // namespace

int64_t pose_partial_warps(int64_t n) {
  return std::max<int64_t>(1, (n + kGradBlock - 1) / kGradBlock) * (kGradBlock / 32);
}

gs_status launch_project_bwd(const gs_params& p, const float* poses, const ViewTable& vt,
                             const gs_raster_cfg& cfg, const gs_splats& sp, const gs_bins& bins,
                             const float* partials, const gs_grads& g, float* pose_partials, float* dpose,
                             float* drgb, cudaStream_t s) {
  GradArgs a;
  a.means4 = reinterpret_cast<const float4*>(p.means4);
  a.scale_opa = reinterpret_cast<const float4*>(p.scale_opa);
  a.quat = reinterpret_cast<const float4*>(p.quat);
  a.sh = p.sh;
  a.n = p.n;
  a.sh_stride = p.sh_stride > 0 ? p.sh_stride : p.n;
  a.poses = poses;
  a.clamp_j = cfg.clamp_jacobian;
  a.touched = sp.touched;
  a.aux = sp.aux;
  a.pair_off = bins.pair_off;
  a.counts = bins.counts;
  a.partials = partials;
  a.g_means4 = reinterpret_cast<float4*>(g.means4);
  a.g_scale_opa = reinterpret_cast<float4*>(g.scale_opa);
  a.g_quat = reinterpret_cast<float4*>(g.quat);
  a.g_sh = g.sh;
  a.g_sh_stride = g.sh_stride > 0 ? g.sh_stride : g.n;
  const int64_t warps = pose_partial_warps(p.n);
  a.pose_a = pose_partials;
  a.pose_b = pose_partials + 6 * warps * vt.views;
  // drgb: three planes [V][n] float4, the colour gradients last
  a.gsum = reinterpret_cast<float4*>(drgb);
  a.drgb = a.gsum + 2 * p.n * vt.views;
  if (p.n == 0) {
    if (dpose) cudaMemsetAsync(dpose, 0, sizeof(float) * 6 * vt.views, s);
    return check_launch("project_bwd");
  }
  const unsigned grid = (unsigned)((p.n + kGradBlock - 1) / kGradBlock);
  const int64_t m = p.n * vt.views;
  launch_dependent(k_pair_sum, (unsigned)((m + 255) / 256), 256, s, a, m);
  switch (p.sh_degree) {
    case 0:
      if (vt.views == 1) launch_dependent(k_project_bwd<0, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<0, false>, grid, kGradBlock, s, a, vt);
      launch_dependent(k_sh_bwd<0>, grid, kGradBlock, s, a, vt);
      break;
    case 1:
      if (vt.views == 1) launch_dependent(k_project_bwd<1, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<1, false>, grid, kGradBlock, s, a, vt);
      launch_dependent(k_sh_bwd<1>, grid, kGradBlock, s, a, vt);
      break;
    case 2:
      if (vt.views == 1) launch_dependent(k_project_bwd<2, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<2, false>, grid, kGradBlock, s, a, vt);
      launch_dependent(k_sh_bwd<2>, grid, kGradBlock, s, a, vt);
      break;
    default:
      if (vt.views == 1) launch_dependent(k_project_bwd<3, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<3, false>, grid, kGradBlock, s, a, vt);
      launch_dependent(k_sh_bwd<3>, grid, kGradBlock, s, a, vt);
      break;
  }
  if (dpose) {
    const int64_t chunk = (warps + kPoseChunks - 1) / kPoseChunks;
    launch_dependent(k_pose_chunks, dim3(kPoseChunks, vt.views), 256, s, a.pose_a, a.pose_b, warps, chunk);
    launch_dependent(k_pose_finalize, vt.views, kPoseChunks, s, a.pose_a, warps, chunk, dpose);
  }
  return check_launch("project_bwd");
}

gs_status launch_project_bwd_adam(const gs_params& p, const float* poses, const ViewTable& vt,
                                  const gs_raster_cfg& cfg, const gs_splats& sp, const gs_bins& bins,
                                  const float* partials, const gs_grads& g, float* pose_partials, float* dpose,
                                  float* drgb, const gs_grads& prw, const gs_grads& m, const gs_grads& v,
                                  const gs_adam_params_cfg& acfg, cudaStream_t s) {
  GradArgs a;
  a.means4 = reinterpret_cast<const float4*>(p.means4);
  a.scale_opa = reinterpret_cast<const float4*>(p.scale_opa);
  a.quat = reinterpret_cast<const float4*>(p.quat);
  a.sh = p.sh;
  a.n = p.n;
  a.sh_stride = p.sh_stride > 0 ? p.sh_stride : p.n;
  a.poses = poses;
  a.clamp_j = cfg.clamp_jacobian;
  a.touched = sp.touched;
  a.aux = sp.aux;
  a.pair_off = bins.pair_off;
  a.counts = bins.counts;
  a.partials = partials;
  a.g_means4 = reinterpret_cast<float4*>(g.means4);
  a.g_scale_opa = reinterpret_cast<float4*>(g.scale_opa);
  a.g_quat = reinterpret_cast<float4*>(g.quat);
  a.g_sh = g.sh;
  a.g_sh_stride = g.sh_stride > 0 ? g.sh_stride : g.n;
  const int64_t warps = pose_partial_warps(p.n);
  a.pose_a = pose_partials;
  a.pose_b = pose_partials + 6 * warps * vt.views;
  a.gsum = reinterpret_cast<float4*>(drgb);
  a.drgb = a.gsum + 2 * p.n * vt.views;
  AdamFamilies f;
  const int nc = (p.sh_degree + 1) * (p.sh_degree + 1);
  for (int q = 0; q < 4; ++q) {
    f.lr4[0][q] = acfg.lr_means4[q];
    f.lr4[1][q] = acfg.lr_scale_opa[q];
    f.lr4[2][q] = acfg.lr_quat[q];
  }
  f.on4 = acfg.update_mask & 7u;
  f.on_sh = (acfg.update_mask & 8u) ? 1u : 0u;
  for (int pl = 0; pl < 48; ++pl) f.lr_sh[pl] = pl < 3 * nc ? acfg.lr_sh[pl] : 0.f;
  f.b1 = acfg.beta1; f.b2 = acfg.beta2; f.eps = acfg.eps;
  f.bc1 = bias_corr(acfg.beta1, acfg.step);
  f.bc2 = bias_corr(acfg.beta2, acfg.step);
  f.step_dev = acfg.step_dev;
  f.skip_dev = acfg.skip_dev;
  f.status = acfg.status;
  f.p_means4 = reinterpret_cast<float4*>(prw.means4);
  f.p_scale_opa = reinterpret_cast<float4*>(prw.scale_opa);
  f.p_quat = reinterpret_cast<float4*>(prw.quat);
  f.p_sh = prw.sh;
  f.p_sh_stride = prw.sh_stride > 0 ? prw.sh_stride : prw.n;
  f.m_means4 = reinterpret_cast<float4*>(m.means4);
  f.m_scale_opa = reinterpret_cast<float4*>(m.scale_opa);
  f.m_quat = reinterpret_cast<float4*>(m.quat);
  f.v_means4 = reinterpret_cast<float4*>(v.means4);
  f.v_scale_opa = reinterpret_cast<float4*>(v.scale_opa);
  f.v_quat = reinterpret_cast<float4*>(v.quat);
  f.m_sh = m.sh;
  f.v_sh = v.sh;
  f.mv_sh_stride = m.sh_stride > 0 ? m.sh_stride : m.n;
  if (p.n == 0) {
    if (dpose) cudaMemsetAsync(dpose, 0, sizeof(float) * 6 * vt.views, s);
    return check_launch("project_bwd_adam");
  }
  const unsigned grid = (unsigned)((p.n + kGradBlock - 1) / kGradBlock);
  const int64_t mm = p.n * vt.views;
  launch_dependent(k_pair_sum, (unsigned)((mm + 255) / 256), 256, s, a, mm);
  switch (p.sh_degree) {
    case 0:
      if (vt.views == 1) launch_dependent(k_project_bwd<0, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<0, false>, grid, kGradBlock, s, a, vt);
      if (vt.views == 1) launch_dependent(k_sh_bwd_adam<0, true>, grid, kGradBlock, s, a, vt, f);
      else launch_dependent(k_sh_bwd_adam<0, false>, grid, kGradBlock, s, a, vt, f);
      break;
    case 1:
      if (vt.views == 1) launch_dependent(k_project_bwd<1, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<1, false>, grid, kGradBlock, s, a, vt);
      if (vt.views == 1) launch_dependent(k_sh_bwd_adam<1, true>, grid, kGradBlock, s, a, vt, f);
      else launch_dependent(k_sh_bwd_adam<1, false>, grid, kGradBlock, s, a, vt, f);
      break;
    case 2:
      if (vt.views == 1) launch_dependent(k_project_bwd<2, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<2, false>, grid, kGradBlock, s, a, vt);
      if (vt.views == 1) launch_dependent(k_sh_bwd_adam<2, true>, grid, kGradBlock, s, a, vt, f);
      else launch_dependent(k_sh_bwd_adam<2, false>, grid, kGradBlock, s, a, vt, f);
      break;
    default:
      if (vt.views == 1) launch_dependent(k_project_bwd<3, true>, grid, kGradBlock, s, a, vt);
      else launch_dependent(k_project_bwd<3, false>, grid, kGradBlock, s, a, vt);
      if (vt.views == 1) launch_dependent(k_sh_bwd_adam<3, true>, grid, kGradBlock, s, a, vt, f);
      else launch_dependent(k_sh_bwd_adam<3, false>, grid, kGradBlock, s, a, vt, f);
      break;
  }
  if (dpose) {
    const int64_t chunk = (warps + kPoseChunks - 1) / kPoseChunks;
    launch_dependent(k_pose_chunks, dim3(kPoseChunks, vt.views), 256, s, a.pose_a, a.pose_b, warps, chunk);
    launch_dependent(k_pose_finalize, vt.views, kPoseChunks, s, a.pose_a, warps, chunk, dpose);
  }
  return check_launch("project_bwd_adam");
}

}  // namespace gs
