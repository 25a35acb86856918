// Image loss of a training step (L1 or mean squared error against a target)
// and its gradient dL/dimage, which the renderer's backward consumes.  The
// paper only names its rendering loss; these two are the readings used here.
// Fixed grid and fixed-order reductions: the loss value is deterministic.
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kLossThreads = 256;
constexpr int kLossBlocks = 592;  // 4 per SM on a 148-SM part; fixed for determinism

__global__ void __launch_bounds__(kLossThreads) k_loss(const float* __restrict__ img,
                                                       const float* __restrict__ tgt, int64_t count,
                                                       int kind, float* __restrict__ grad,
                                                       float* __restrict__ partial) {
  __shared__ float s[kLossThreads];
  const float inv = 1.0f / (float)count;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * kLossThreads + threadIdx.x; i < count;
       i += (int64_t)kLossBlocks * kLossThreads) {
    const float d = img[i] - tgt[i];
    if (kind == 0) {
      acc += fabsf(d);
      if (grad) grad[i] = (d > 0.f ? inv : (d < 0.f ? -inv : 0.f));
    } else {
      acc += d * d;
      if (grad) grad[i] = 2.f * d * inv;
    }
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kLossThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(1024) k_loss_final(const float* __restrict__ partial, int64_t count,
                                                     float* __restrict__ loss) {
  __shared__ float s[1024];
  s[threadIdx.x] = threadIdx.x < kLossBlocks ? partial[threadIdx.x] : 0.f;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = s[0] / (float)count;
}

}  // namespace

size_t loss_workspace_bytes() { return align_up(sizeof(float) * kLossBlocks, 256); }

gs_status launch_loss(const float* img, const float* tgt, int64_t count, int kind, float* grad,
                      float* loss, void* ws, cudaStream_t s) {
  float* partial = static_cast<float*>(ws);
  k_loss<<<kLossBlocks, kLossThreads, 0, s>>>(img, tgt, count, kind, grad, partial);
  k_loss_final<<<1, 1024, 0, s>>>(partial, count, loss);
  return check_launch("loss");
}

}  // namespace gs
