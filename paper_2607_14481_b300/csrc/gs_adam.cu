// Fused Adam over the flat parameter arena (one launch for every parameter
// group) and the optional pose step (Adam on the twist, then T <- Exp(xi) T).
// HBM-bound: 16 B read + 12 B written per element.
#include <cmath>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kAdamThreads = 256;
constexpr int64_t kAdamChunk = kAdamThreads * 4 * 4;  // elements per block (4 float4 per thread, 2 at a time)

struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t n;
  float b1, b2, eps;
  float bc1, bc2;           // 1 - beta^step
  int num_groups;
  gs_adam_group groups[GS_MAX_ADAM_GROUPS];
  int32_t block_start[GS_MAX_ADAM_GROUPS + 1];  // first block of each group
  uint32_t* status;
  const int32_t* step_dev;   // optional: step = *step_dev + 1
  const uint32_t* skip_dev;  // optional: nonzero = skip the update
};

__device__ __forceinline__ bool adam_elem(float& p, float g, float& m, float& v, float step_size,
                                          const AdamArgs& a, float rs_bc2) {
  return ::gs::adam_elem(p, g, m, v, step_size, a.b1, a.b2, a.eps, rs_bc2);
}

// Block b updates one chunk of one group: the group is found once per block
// (no per-element search); the chunk's 16-byte aligned body is processed as
// float4 (two chunks per thread, loads issued before the stores), its ragged
// head and tail element by element.
__global__ void __launch_bounds__(kAdamThreads) k_adam(const AdamArgs a) {
  if (a.skip_dev && *a.skip_dev) return;
  float bc1 = a.bc1, bc2 = a.bc2;
  if (a.step_dev) {
    const int st = *a.step_dev + 1;
    bc1 = bias_corr(a.b1, st);
    bc2 = bias_corr(a.b2, st);
  }
  const float rs_bc2 = rsqrtf(bc2);
  const int b = blockIdx.x;
  int gi = 0;
  while (gi + 1 < a.num_groups && a.block_start[gi + 1] <= b) ++gi;
  const gs_adam_group G = a.groups[gi];
  const int64_t r0 = G.begin + (int64_t)(b - a.block_start[gi]) * kAdamChunk;
  const int64_t r1 = min(G.end, r0 + kAdamChunk);
  if (r0 >= r1) return;
  const int64_t a0 = min(r1, (r0 + 3) & ~(int64_t)3);  // first 16-byte aligned element
  const int64_t a1 = max(a0, r1 & ~(int64_t)3);        // end of the float4 body
  const float ss = 1.f / bc1;
  bool bad = false;
  for (int64_t e = r0 + threadIdx.x; e < a0; e += kAdamThreads)
    bad |= !adam_elem(a.p[e], a.g[e], a.m[e], a.v[e], G.lr[(e - G.begin) & 3] * ss, a, rs_bc2);
  const int rot = (int)((a0 - G.begin) & 3);
  const float s0 = G.lr[rot & 3] * ss, s1 = G.lr[(rot + 1) & 3] * ss;
  const float s2 = G.lr[(rot + 2) & 3] * ss, s3 = G.lr[(rot + 3) & 3] * ss;
  float4* __restrict__ P4 = reinterpret_cast<float4*>(a.p);
  const float4* __restrict__ G4 = reinterpret_cast<const float4*>(a.g);
  float4* __restrict__ M4 = reinterpret_cast<float4*>(a.m);
  float4* __restrict__ V4 = reinterpret_cast<float4*>(a.v);
  const int64_t c1 = a1 / 4;
  for (int64_t c0 = a0 / 4 + threadIdx.x; c0 < c1; c0 += 2 * kAdamThreads) {
    const int64_t cb = c0 + kAdamThreads;
    const bool two = cb < c1;
    float4 p0 = P4[c0], g0 = G4[c0], m0 = M4[c0], v0 = V4[c0];
    float4 p1, g1, m1, v1;
    if (two) { p1 = P4[cb]; g1 = G4[cb]; m1 = M4[cb]; v1 = V4[cb]; }
    bad |= !adam_elem(p0.x, g0.x, m0.x, v0.x, s0, a, rs_bc2);
    bad |= !adam_elem(p0.y, g0.y, m0.y, v0.y, s1, a, rs_bc2);
    bad |= !adam_elem(p0.z, g0.z, m0.z, v0.z, s2, a, rs_bc2);
    bad |= !adam_elem(p0.w, g0.w, m0.w, v0.w, s3, a, rs_bc2);
    P4[c0] = p0; M4[c0] = m0; V4[c0] = v0;
    if (two) {
      bad |= !adam_elem(p1.x, g1.x, m1.x, v1.x, s0, a, rs_bc2);
      bad |= !adam_elem(p1.y, g1.y, m1.y, v1.y, s1, a, rs_bc2);
      bad |= !adam_elem(p1.z, g1.z, m1.z, v1.z, s2, a, rs_bc2);
      bad |= !adam_elem(p1.w, g1.w, m1.w, v1.w, s3, a, rs_bc2);
      P4[cb] = p1; M4[cb] = m1; V4[cb] = v1;
    }
  }
  for (int64_t e = a1 + threadIdx.x; e < r1; e += kAdamThreads)
    bad |= !adam_elem(a.p[e], a.g[e], a.m[e], a.v[e], G.lr[(e - G.begin) & 3] * ss, a, rs_bc2);
  if (bad && a.status) atomicOr(a.status, 1u);
}

struct PoseArgs {
  float* pose;
  const float* dpose;
  float* m;
  float* v;
  int views;
  float lr, b1, b2, eps, bc1, bc2;
  uint32_t* status;
  const int32_t* step_dev;  // optional shared step (*step_dev + 1)
  int32_t* pose_steps;      // optional per-view steps, incremented here
  const uint32_t* skip_dev;
};

// Pose step per view: Adam on xi (zero-based tangent), then the SE(3)
// exponential (Rodrigues rotation, V-matrix translation) applied on the left.
__global__ void k_pose_adam(const PoseArgs a) {
  chain_enter();
  const int vw = blockIdx.x * blockDim.x + threadIdx.x;
  if (vw >= a.views || (a.skip_dev && *a.skip_dev)) return;
  float bc1 = a.bc1, bc2 = a.bc2;
  if (a.pose_steps) {
    const int st = a.pose_steps[vw] + 1;
    a.pose_steps[vw] = st;
    bc1 = bias_corr(a.b1, st);
    bc2 = bias_corr(a.b2, st);
  } else if (a.step_dev) {
    const int st = *a.step_dev + 1;
    bc1 = bias_corr(a.b1, st);
    bc2 = bias_corr(a.b2, st);
  }
  float xi[6];
  bool bad = false;
  for (int k = 0; k < 6; ++k) {
    const int j = 6 * vw + k;
    const float g = a.dpose[j];
    const float m = a.b1 * a.m[j] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[j] + (1.f - a.b2) * g * g;
    a.m[j] = m; a.v[j] = v;
    xi[k] = -a.lr * (m / bc1) / (sqrtf(v / bc2) + a.eps);
    bad |= !isfinite(g);
  }
  const float wx = xi[3], wy = xi[4], wz = xi[5];
  const float th2 = wx * wx + wy * wy + wz * wz;
  const float th = sqrtf(th2);
  float A, B, C;
  if (th < 1e-2f) {  // Taylor series, accurate to float rounding below 1e-2
    A = 1.f - th2 / 6.f * (1.f - th2 / 20.f);
    B = 0.5f - th2 / 24.f * (1.f - th2 / 30.f);
    C = 1.f / 6.f - th2 / 120.f * (1.f - th2 / 42.f);
  } else {
    A = sinf(th) / th;
    B = (1.f - cosf(th)) / th2;
    C = (th - sinf(th)) / (th2 * th);
  }
  const float K[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
  float K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  float Re[9], Vm[9];
  for (int k = 0; k < 9; ++k) {
    const float I = (k % 4 == 0) ? 1.f : 0.f;
    Re[k] = I + A * K[k] + B * K2[k];
    Vm[k] = I + B * K[k] + C * K2[k];
  }
  float te[3];
  for (int r = 0; r < 3; ++r) te[r] = Vm[3 * r] * xi[0] + Vm[3 * r + 1] * xi[1] + Vm[3 * r + 2] * xi[2];
  float* P = a.pose + 12 * vw;
  float R0[9], t0[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R0[3 * r + c] = P[4 * r + c];
    t0[r] = P[4 * r + 3];
  }
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      P[4 * r + c] = Re[3 * r] * R0[c] + Re[3 * r + 1] * R0[3 + c] + Re[3 * r + 2] * R0[6 + c];
    P[4 * r + 3] = Re[3 * r] * t0[0] + Re[3 * r + 1] * t0[1] + Re[3 * r + 2] * t0[2] + te[r];
  }
  if (bad && a.status) atomicOr(a.status, 1u);
}

__global__ void k_step_increment(int32_t* step, const uint32_t* skip) {
  chain_enter();
  if (!(skip && *skip)) *step += 1;
}

}  // namespace

gs_status launch_adam(float* p, const float* g, float* m, float* v, int64_t n,
                      const gs_adam_cfg& cfg, int step, cudaStream_t s) {
  AdamArgs a;
  a.p = p; a.g = g; a.m = m; a.v = v; a.n = n;
  a.b1 = cfg.beta1; a.b2 = cfg.beta2; a.eps = cfg.eps;
  a.bc1 = bias_corr(cfg.beta1, step);
  a.bc2 = bias_corr(cfg.beta2, step);
  a.num_groups = cfg.num_groups;
  int64_t blocks = 0;
  for (int k = 0; k < cfg.num_groups; ++k) {
    a.groups[k] = cfg.groups[k];
    a.block_start[k] = (int32_t)blocks;
    blocks += (cfg.groups[k].end - cfg.groups[k].begin + kAdamChunk - 1) / kAdamChunk;
  }
  a.block_start[cfg.num_groups] = (int32_t)blocks;
  a.status = cfg.status;
  a.step_dev = cfg.step_dev;
  a.skip_dev = cfg.skip_dev;
  if (n > 0 && blocks > 0) k_adam<<<(unsigned)blocks, kAdamThreads, 0, s>>>(a);
  if (cfg.pose && cfg.views > 0) {
    PoseArgs pa;
    pa.pose = cfg.pose; pa.dpose = cfg.dpose; pa.m = cfg.pose_m; pa.v = cfg.pose_v;
    pa.views = cfg.views; pa.lr = cfg.pose_lr; pa.b1 = cfg.beta1; pa.b2 = cfg.beta2; pa.eps = cfg.eps;
    const int ps = cfg.pose_step > 0 ? cfg.pose_step : step;
    pa.bc1 = bias_corr(cfg.beta1, ps);
    pa.bc2 = bias_corr(cfg.beta2, ps);
    pa.status = cfg.status;
    pa.step_dev = cfg.step_dev;
    pa.pose_steps = cfg.pose_steps_dev;
    pa.skip_dev = cfg.skip_dev;
    launch_dependent(k_pose_adam, (cfg.views + 63) / 64, 64, s, pa);
  }
  if (cfg.step_dev) launch_dependent(k_step_increment, 1, 1, s, cfg.step_dev, cfg.skip_dev);
  return check_launch("adam");
}

}  // namespace gs
