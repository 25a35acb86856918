// Loop-closure update of the Gaussians (Sec. 5.5: each Gaussian keeps the
// keyframe that added it and receives that keyframe's Sim(3) correction, with
// scale and rotation updated accordingly).  One thread per Gaussian; the
// corrections of all keyframes are small and stay in L1/L2.  HBM-bound: 4 B
// keyframe id + 48 B read and 48 B written per Gaussian.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

__global__ void __launch_bounds__(256) k_sim3_update(float4* __restrict__ means4, float4* __restrict__ scale_opa,
                                                     float4* __restrict__ quat, const int32_t* __restrict__ kf,
                                                     const float* __restrict__ sim3, int32_t num_kf, int64_t n,
                                                     uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t k = kf[i];
  if (k < 0) return;  // not moved
  if (k >= num_kf) {
    atomicOr(status, 1u);  // a keyframe id without a correction: skipped
    return;
  }
  const float* S = sim3 + 8 * (int64_t)k;
  const float qn = rsqrtf(S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + S[3] * S[3]);
  const float w = S[0] * qn, x = S[1] * qn, y = S[2] * qn, z = S[3] * qn;
  float R[9];
  quat_rot(w, x, y, z, R);
  const float s = S[7];
  const float4 m = means4[i];
  means4[i] = make_float4(s * (R[0] * m.x + R[1] * m.y + R[2] * m.z) + S[4],
                          s * (R[3] * m.x + R[4] * m.y + R[5] * m.z) + S[5],
                          s * (R[6] * m.x + R[7] * m.y + R[8] * m.z) + S[6], m.w);
  const float ls = logf(s);
  const float4 so = scale_opa[i];
  scale_opa[i] = make_float4(so.x + ls, so.y + ls, so.z + ls, so.w);
  const float4 q = quat[i];  // (w, x, y, z): q' = q_S q
  quat[i] = make_float4(w * q.x - x * q.y - y * q.z - z * q.w, w * q.y + x * q.x + y * q.w - z * q.z,
                        w * q.z - x * q.w + y * q.x + z * q.y, w * q.w + x * q.z - y * q.y + z * q.x);
}

// Leaf Gaussians per keyframe (integer counts: the order of the atomics does
// not show); ids outside [0, num_kf) are not counted.
__global__ void __launch_bounds__(256) k_keyframe_counts(const int32_t* __restrict__ kf, int64_t n, int32_t num_kf,
                                                         uint32_t* __restrict__ counts,
                                                         const uint8_t* __restrict__ active) {
  extern __shared__ uint32_t s_c[];
  const bool local = num_kf <= 8192;  // histogram in shared memory
  if (local)
    for (int k = threadIdx.x; k < num_kf; k += blockDim.x) s_c[k] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = kf[i];
    if (k < 0 || k >= num_kf || (active && !active[i])) continue;
    atomicAdd(local ? &s_c[k] : &counts[k], 1u);
  }
  __syncthreads();
  if (local)
    for (int k = threadIdx.x; k < num_kf; k += blockDim.x)
      if (s_c[k]) atomicAdd(&counts[k], s_c[k]);
}

__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

gs_status launch_keyframe_counts(const int32_t* kf, int64_t n, int32_t num_kf, uint32_t* counts, cudaStream_t s,
                                 const uint8_t* active) {
  if (num_kf <= 0) return GS_OK;
  if (cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)num_kf, s) != cudaSuccess)
    return check_launch("keyframe counts");
  if (n <= 0) return GS_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(592, (n + 255) / 256);
  const size_t smem = num_kf <= 8192 ? sizeof(uint32_t) * (size_t)num_kf : 0;
  k_keyframe_counts<<<grid, 256, smem, s>>>(kf, n, num_kf, counts, active);
  return check_launch("k_keyframe_counts");
}

gs_status launch_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s) {
  if (n <= 0) return GS_OK;
  k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, n);
  return check_launch("k_fill_i32");
}

gs_status launch_sim3_update(const gs_grads& p, const int32_t* kf, const float* sim3, int32_t num_kf,
                             uint32_t* status, cudaStream_t s) {
  if (p.n == 0) return GS_OK;
  k_sim3_update<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<float4*>(p.means4), reinterpret_cast<float4*>(p.scale_opa), reinterpret_cast<float4*>(p.quat),
      kf, sim3, num_kf, p.n, status);
  return check_launch("k_sim3_update");
}

}  // namespace gs
