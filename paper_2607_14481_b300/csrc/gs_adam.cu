// Fused Adam over the flat parameter arena (one launch for every parameter
// group) and the optional pose step (Adam on the twist, then T <- Exp(xi) T).
// HBM-bound: 16 B read + 12 B written per element.
#include <cmath>

#include "gs_internal.h"

namespace gs {

namespace {

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
  uint32_t* status;
};

__device__ __forceinline__ bool adam_elem(float& p, float g, float& m, float& v, float lr,
                                          const AdamArgs& a) {
  m = a.b1 * m + (1.f - a.b1) * g;
  v = a.b2 * v + (1.f - a.b2) * g * g;
  const float mh = m / a.bc1, vh = v / a.bc2;
  p -= lr * mh / (sqrtf(vh) + a.eps);
  return isfinite(g) && isfinite(v);
}

__device__ __forceinline__ float lr_of(const AdamArgs& a, int64_t e, bool& in_group) {
  for (int k = 0; k < a.num_groups; ++k) {
    const gs_adam_group& G = a.groups[k];
    if (e >= G.begin && e < G.end) { in_group = true; return G.lr[(e - G.begin) & 3]; }
  }
  in_group = false;
  return 0.f;
}

// Grid-stride over float4 chunks (the arena is 16-byte aligned); the scalar
// tail is handled by the first threads.
__global__ void __launch_bounds__(256) k_adam(const AdamArgs a) {
  const int64_t n4 = a.n / 4;
  bool bad = false;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n4;
       c += (int64_t)gridDim.x * blockDim.x) {
    float4 p = reinterpret_cast<float4*>(a.p)[c];
    const float4 g = reinterpret_cast<const float4*>(a.g)[c];
    float4 m = reinterpret_cast<float4*>(a.m)[c];
    float4 v = reinterpret_cast<float4*>(a.v)[c];
    float* pp = &p.x; const float* gg = &g.x; float* mm = &m.x; float* vv = &v.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool in;
      const float lr = lr_of(a, 4 * c + k, in);
      if (in) bad |= !adam_elem(pp[k], gg[k], mm[k], vv[k], lr, a);
    }
    reinterpret_cast<float4*>(a.p)[c] = p;
    reinterpret_cast<float4*>(a.m)[c] = m;
    reinterpret_cast<float4*>(a.v)[c] = v;
  }
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t e = 4 * n4 + t;
  if (t < 4 && e < a.n) {
    bool in;
    const float lr = lr_of(a, e, in);
    if (in) bad |= !adam_elem(a.p[e], a.g[e], a.m[e], a.v[e], lr, a);
  }
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
};

// Pose step per view: Adam on xi (zero-based tangent), then the SE(3)
// exponential (Rodrigues rotation, V-matrix translation) applied on the left.
__global__ void k_pose_adam(const PoseArgs a) {
  const int vw = blockIdx.x * blockDim.x + threadIdx.x;
  if (vw >= a.views) return;
  float xi[6];
  bool bad = false;
  for (int k = 0; k < 6; ++k) {
    const int j = 6 * vw + k;
    const float g = a.dpose[j];
    const float m = a.b1 * a.m[j] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[j] + (1.f - a.b2) * g * g;
    a.m[j] = m; a.v[j] = v;
    xi[k] = -a.lr * (m / a.bc1) / (sqrtf(v / a.bc2) + a.eps);
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

}  // namespace

gs_status launch_adam(float* p, const float* g, float* m, float* v, int64_t n,
                      const gs_adam_cfg& cfg, int step, cudaStream_t s) {
  AdamArgs a;
  a.p = p; a.g = g; a.m = m; a.v = v; a.n = n;
  a.b1 = cfg.beta1; a.b2 = cfg.beta2; a.eps = cfg.eps;
  a.bc1 = (float)(1.0 - std::pow((double)cfg.beta1, step));
  a.bc2 = (float)(1.0 - std::pow((double)cfg.beta2, step));
  a.num_groups = cfg.num_groups;
  for (int k = 0; k < cfg.num_groups; ++k) a.groups[k] = cfg.groups[k];
  a.status = cfg.status;
  if (n > 0) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n4 = std::max<int64_t>(1, n / 4);
    const int64_t want = (n4 + 255) / 256;
    const int64_t grid = std::min<int64_t>(want, (int64_t)sms * 8);  // 8 resident CTAs per SM
    k_adam<<<(unsigned)grid, 256, 0, s>>>(a);
  }
  if (cfg.pose && cfg.views > 0) {
    PoseArgs pa;
    pa.pose = cfg.pose; pa.dpose = cfg.dpose; pa.m = cfg.pose_m; pa.v = cfg.pose_v;
    pa.views = cfg.views; pa.lr = cfg.pose_lr; pa.b1 = cfg.beta1; pa.b2 = cfg.beta2; pa.eps = cfg.eps;
    const int ps = cfg.pose_step > 0 ? cfg.pose_step : step;
    pa.bc1 = (float)(1.0 - std::pow((double)cfg.beta1, ps));
    pa.bc2 = (float)(1.0 - std::pow((double)cfg.beta2, ps));
    pa.status = cfg.status;
    k_pose_adam<<<(cfg.views + 63) / 64, 64, 0, s>>>(pa);
  }
  return check_launch("adam");
}

}  // namespace gs
