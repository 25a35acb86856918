// Level-of-detail hierarchy over the Gaussians (Sec. 6: coarse nodes hold
// the parameters of a merged group of children; rendering descends from the
// roots until a node's screen size falls below tau or a leaf is reached).
//
// Three levels: the leaves, level 1 (one node per 8 leaves) and level 2 (one
// node per 8 level-1 nodes).  Grouping is spatial and data parallel: leaves
// are sorted by the Morton code of their mean (10 bits per axis over the
// leaves' bounding box, stable, so equal codes keep index order) and every run
// of 8 consecutive leaves shares a parent; runs of 8 consecutive level-1 nodes
// share a level-2 parent.  A parent is the moment-matching merge of its
// children with weights w = opacity: mean and covariance of the mixture,
// opacity-weighted SH, opacity min(0.99, sum w o / sum w); its rotation and
// scales come from a Jacobi eigen-decomposition of the covariance.
//
// Coarse nodes are written into the same parameter arrays after the leaves:
// leaves [0, n), level 1 [n, n + n1), level 2 [n + n1, n + n1 + n2).
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kLodThreads = 256;

__global__ void k_lod_init(uint32_t* bbox, uint32_t* n_word, uint32_t n) {
  if (threadIdx.x < 3) {
    bbox[threadIdx.x] = 0xffffffffu;  // min (ordered)
    bbox[3 + threadIdx.x] = 0u;       // max (ordered)
  }
  if (threadIdx.x == 0) *n_word = n;
}

// Bounding box of the leaf means (order-independent min / max).
__global__ void __launch_bounds__(kLodThreads) k_lod_bbox(const float4* __restrict__ means4, int64_t n,
                                                          uint32_t* bbox) {
  __shared__ uint32_t s[6];
  if (threadIdx.x < 3) {
    s[threadIdx.x] = 0xffffffffu;
    s[3 + threadIdx.x] = 0u;
  }
  __syncthreads();
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 m = means4[i];
    const uint32_t o[3] = {float_order(m.x), float_order(m.y), float_order(m.z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = min(lo[a], o[a]);
      hi[a] = max(hi[a], o[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    atomicMin(&s[a], lo[a]);
    atomicMax(&s[3 + a], hi[a]);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    atomicMin(&bbox[threadIdx.x], s[threadIdx.x]);
    atomicMax(&bbox[3 + threadIdx.x], s[3 + threadIdx.x]);
  }
}

// Morton code of every leaf (quantised in single precision) and its index.
__global__ void __launch_bounds__(kLodThreads) k_lod_morton(const float4* __restrict__ means4, int64_t n,
                                                            const uint32_t* bbox, uint32_t* code, uint32_t* idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float lo[3], scale[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = float_unorder(bbox[a]);
    const float ext = __fsub_rn(float_unorder(bbox[3 + a]), lo[a]);
    scale[a] = ext > 0.f ? __fdiv_rn(1024.0f, ext) : 0.f;
  }
  const float4 m = means4[i];
  code[i] = spread10(quantise10(m.x, lo[0], scale[0])) | (spread10(quantise10(m.y, lo[1], scale[1])) << 1) |
            (spread10(quantise10(m.z, lo[2], scale[2])) << 2);
  idx[i] = (uint32_t)i;
}

struct MergeArgs {
  float4* means4;
  float4* scale_opa;
  float4* quat;
  float* sh;
  int64_t sh_stride;
  int32_t* parent;
  const uint32_t* order;  // level 1: leaves in Morton order
  float* wts;             // [n1 + n2][8] children's merge weights (opacities), level 1 then level 2
  float* iws;             // [n1 + n2] 1 / sum of the weights
  int64_t n_leaf, n1, n2;
};

// One thread per coarse node of the level: the moment-matching merge of its
// (up to 8) children's geometry and opacity; the weights go to a.wts for the
// SH pass.
template <int NC, bool LEVEL2>
__global__ void __launch_bounds__(kLodThreads) k_lod_merge(const MergeArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t groups = LEVEL2 ? a.n2 : a.n1;
  if (g >= groups) return;
  const int64_t members = LEVEL2 ? a.n1 : a.n_leaf;
  const int k = (int)min((int64_t)8, members - 8 * g);
  const int64_t node = LEVEL2 ? a.n_leaf + a.n1 + g : a.n_leaf + g;
  int64_t child[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    child[j] = j < k ? (LEVEL2 ? a.n_leaf + 8 * g + j : (int64_t)a.order[8 * g + j]) : 0;
  // weights and the mean
  float w[8], W = 0.f, o2 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    w[j] = 0.f;
    if (j < k) {
      const float4 so = a.scale_opa[child[j]];
      const float4 mu = a.means4[child[j]];
      w[j] = 1.0f / (1.0f + expf(-so.w));
      W += w[j];
      o2 += w[j] * w[j];
      mx += w[j] * mu.x; my += w[j] * mu.y; mz += w[j] * mu.z;
    }
  }
  const float iW = 1.0f / W;
  mx *= iW; my *= iW; mz *= iW;
  // covariance of the mixture
  float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx xy xz yy yz zz
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j < k) {
      const float4 mu = a.means4[child[j]], so = a.scale_opa[child[j]], q4 = a.quat[child[j]];
      const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
      float R[9];
      quat_rot(q4.x * qn, q4.y * qn, q4.z * qn, q4.w * qn, R);
      const float v[3] = {expf(2.f * so.x), expf(2.f * so.y), expf(2.f * so.z)};
      const float d[3] = {mu.x - mx, mu.y - my, mu.z - mz};
      const int rr[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int r = rr[e], c = cc[e];
        const float s = R[3 * r] * v[0] * R[3 * c] + R[3 * r + 1] * v[1] * R[3 * c + 1] +
                        R[3 * r + 2] * v[2] * R[3 * c + 2];
        C[e] += w[j] * (s + d[r] * d[c]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) C[e] *= iW;
  {  // the SH pass (k_lod_merge_sh) averages the coefficients with these weights
    const int64_t wi = LEVEL2 ? a.n1 + g : g;
    float4* w4 = reinterpret_cast<float4*>(a.wts + 8 * wi);
    w4[0] = make_float4(w[0], w[1], w[2], w[3]);
    w4[1] = make_float4(w[4], w[5], w[6], w[7]);
    a.iws[wi] = iW;
  }
  // rotation and scales from the eigen-decomposition
  float A[9] = {C[0], C[1], C[2], C[1], C[3], C[4], C[2], C[4], C[5]};
  float lam[3], V[9];
  jacobi3(A, lam, V);
  const float det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                    V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (det < 0.f) {
    V[2] = -V[2]; V[5] = -V[5]; V[8] = -V[8];
  }
  const float op = fminf(0.99f, o2 * iW);
  a.means4[node] = make_float4(mx, my, mz, 0.f);
  a.scale_opa[node] = make_float4(0.5f * logf(fmaxf(lam[0], 1e-30f)), 0.5f * logf(fmaxf(lam[1], 1e-30f)),
                                  0.5f * logf(fmaxf(lam[2], 1e-30f)), logf(op / (1.f - op)));
  a.quat[node] = rot_to_quat(V);
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (j < k) a.parent[child[j]] = (int32_t)node;
  if (LEVEL2) a.parent[node] = -1;
}

// SH of the level's coarse nodes: the opacity-weighted mean of every
// coefficient of the (up to 8) children.  Block (x, y) covers 256 nodes and
// kShPlanes coefficient planes; the blocks of one group of planes run before
// the next group's, so the planes being gathered (n floats each) stay in L2
// while the children, scattered in memory in level 1, are read one value at a
// time.
constexpr int kShPlanes = 4;
template <int NC, bool LEVEL2>
__global__ void __launch_bounds__(kLodThreads) k_lod_merge_sh(const MergeArgs a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t groups = LEVEL2 ? a.n2 : a.n1;
  if (g >= groups) return;
  const int64_t members = LEVEL2 ? a.n1 : a.n_leaf;
  const int k = (int)min((int64_t)8, members - 8 * g);
  const int64_t node = LEVEL2 ? a.n_leaf + a.n1 + g : a.n_leaf + g;
  const int64_t wi = LEVEL2 ? a.n1 + g : g;
  const float4* w4 = reinterpret_cast<const float4*>(a.wts + 8 * wi);
  const float4 wa = w4[0], wb = w4[1];
  const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
  const float iW = a.iws[wi];
  int64_t child[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    child[j] = j < k ? (LEVEL2 ? a.n_leaf + 8 * g + j : (int64_t)a.order[8 * g + j]) : 0;
  const int p0 = blockIdx.y * kShPlanes;
#pragma unroll
  for (int q = 0; q < kShPlanes; ++q) {
    const int p = p0 + q;
    if (p >= 3 * NC) break;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < k) acc += w[j] * a.sh[(int64_t)p * a.sh_stride + child[j]];
    a.sh[(int64_t)p * a.sh_stride + node] = acc * iW;
  }
}

struct LodWs {
  uint32_t *bbox, *n_word;
  uint32_t *keys_a, *vals_a, *keys_b, *vals_b, *keys_out, *vals_out;
  float *wts, *iws;
  void* radix;
  size_t bytes;
};

LodWs lod_layout(char* base, int64_t n) {
  LodWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1), 256);
    return p;
  };
  const size_t m = sizeof(uint32_t) * (size_t)std::max<int64_t>(1, n);
  w.bbox = (uint32_t*)take(8 * sizeof(uint32_t));
  w.n_word = w.bbox + 6;
  w.keys_a = (uint32_t*)take(m); w.vals_a = (uint32_t*)take(m);
  w.keys_b = (uint32_t*)take(m); w.vals_b = (uint32_t*)take(m);
  w.keys_out = (uint32_t*)take(m); w.vals_out = (uint32_t*)take(m);
  const int64_t coarse = lod_level1(std::max<int64_t>(1, n)) + lod_level2(std::max<int64_t>(1, n));
  w.wts = (float*)take(sizeof(float) * 8 * (size_t)coarse);
  w.iws = (float*)take(sizeof(float) * (size_t)coarse);
  w.radix = take(radix_workspace(std::max<int64_t>(1, n)));
  w.bytes = off;
  return w;
}

template <int NC>
void launch_merges(const MergeArgs& a, cudaStream_t s) {
  const unsigned planes = (unsigned)((3 * NC + kShPlanes - 1) / kShPlanes);
  if (a.n1 > 0) {
    const unsigned gx = (unsigned)((a.n1 + kLodThreads - 1) / kLodThreads);
    k_lod_merge<NC, false><<<gx, kLodThreads, 0, s>>>(a);
    k_lod_merge_sh<NC, false><<<dim3(gx, planes), kLodThreads, 0, s>>>(a);
  }
  if (a.n2 > 0) {
    const unsigned gx = (unsigned)((a.n2 + kLodThreads - 1) / kLodThreads);
    k_lod_merge<NC, true><<<gx, kLodThreads, 0, s>>>(a);
    k_lod_merge_sh<NC, true><<<dim3(gx, planes), kLodThreads, 0, s>>>(a);
  }
}

}  // namespace

int64_t lod_level1(int64_t n) { return (n + 7) / 8; }
int64_t lod_level2(int64_t n) { return (lod_level1(n) + 7) / 8; }

size_t lod_build_workspace_bytes(int64_t n) { return lod_layout(nullptr, n).bytes; }

gs_status launch_lod_build(const gs_grads& nodes, int64_t n_leaf, int32_t* parent, void* ws, cudaStream_t s) {
  if (n_leaf == 0) return GS_OK;
  LodWs w = lod_layout(static_cast<char*>(ws), n_leaf);
  const unsigned grid = (unsigned)((n_leaf + kLodThreads - 1) / kLodThreads);
  k_lod_init<<<1, 32, 0, s>>>(w.bbox, w.n_word, (uint32_t)n_leaf);
  const float4* m4 = reinterpret_cast<const float4*>(nodes.means4);
  k_lod_bbox<<<std::min(grid, 148u * 8u), kLodThreads, 0, s>>>(m4, n_leaf, w.bbox);
  k_lod_morton<<<grid, kLodThreads, 0, s>>>(m4, n_leaf, w.bbox, w.keys_a, w.vals_a);
  gs_status st = launch_radix_sort(w.keys_a, w.vals_a, w.keys_b, w.vals_b, w.keys_out, w.vals_out, w.n_word,
                                   n_leaf, 30, w.radix, s);
  if (st != GS_OK) return st;
  MergeArgs a;
  a.means4 = reinterpret_cast<float4*>(nodes.means4);
  a.scale_opa = reinterpret_cast<float4*>(nodes.scale_opa);
  a.quat = reinterpret_cast<float4*>(nodes.quat);
  a.sh = nodes.sh;
  a.sh_stride = nodes.sh_stride > 0 ? nodes.sh_stride : nodes.n;
  a.parent = parent;
  a.order = w.vals_out;
  a.wts = w.wts;
  a.iws = w.iws;
  a.n_leaf = n_leaf;
  a.n1 = lod_level1(n_leaf);
  a.n2 = lod_level2(n_leaf);
  switch (nodes.sh_degree) {
    case 0: launch_merges<1>(a, s); break;
    case 1: launch_merges<4>(a, s); break;
    case 2: launch_merges<9>(a, s); break;
    default: launch_merges<16>(a, s); break;
  }
  return check_launch("lod_build");
}

}  // namespace gs
