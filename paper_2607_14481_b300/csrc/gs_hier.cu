// Progressive level-of-detail hierarchy (Sec. 6.1 "Adaptive Gaussian Merging
// and Retrieval", Sec. 6.2): an active set of nodes, leaves and merged
// intermediate nodes, that is a cut of the forest (every leaf has exactly one
// active node on its path to its root).  Nodes live in the parameter arena;
// parent (-1: root), up to 4 children (-1: none) and the active flags are
// device arrays of the caller.
//
// Analysis from a keyframe's camera (gs_hier_analyze), in the paper's order:
//   1. screen size S = f_x 3 max scale / t_z of every active node (+inf at or
//      behind the near plane); candidates: S < tau_l (0.5 px);
//   2. only when more than 20% of the active nodes are candidates (5 C > A):
//   3. an inactive parent whose children are all candidates is pulled: it
//      becomes active, its children inactive (no new node);
//   4. the other candidates without a parent are grouped with their 3 nearest
//      candidates: candidates in Morton order of their means (10 bits per
//      axis over their bounding box, stable), chunks of 64 consecutive ones,
//      exact 3 nearest within a chunk by squared single-precision distance
//      (ties by Morton position), then, in Morton order, a candidate not yet
//      grouped takes those of its 3 nearest not yet grouped (one warp per
//      chunk; the greedy pass runs on one lane);
//   5. each group of 2-4 becomes a new active parent node, the moment-matching
//      merge of its children (as the static hierarchy), numbered after the
//      existing nodes in Morton order of its first child.
// Reload (gs_hier_refine, tau_h = 1 px): an active node with children that
// lies in view and has S > tau_h is replaced by its children, pass after pass.
// A render's view cut (gs_project_hier) is that refinement applied virtually.
//
// Every count stays on the device (kernels read it), so an analysis needs no
// host synchronisation and can run on a side stream while renders use the
// other buffer of a double-buffered active set.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kHT = 256;
constexpr int kChunk = 64;
constexpr int kMaxGroups = kChunk / 2;  // groups have at least 2 members

// words of the analysis workspace
enum : int {
  kWActive = 0, kWCand, kWTrig, kWGroups, kWPulled, kWGrouped, kWG, kWChunks, kWN, kWChanged, kWStatus,
  kWBox = 16,  // 6 ordered bounds
  kWords = 32
};

struct HierView {
  float R[9], t[3], fx, fy, cx, cy, znear;
  int W, H;
};

__device__ __forceinline__ HierView load_view(const float* pose, const gs_camera cam, float znear) {
  HierView v;
  v.R[0] = pose[0]; v.R[1] = pose[1]; v.R[2] = pose[2]; v.t[0] = pose[3];
  v.R[3] = pose[4]; v.R[4] = pose[5]; v.R[5] = pose[6]; v.t[1] = pose[7];
  v.R[6] = pose[8]; v.R[7] = pose[9]; v.R[8] = pose[10]; v.t[2] = pose[11];
  v.fx = cam.fx; v.fy = cam.fy; v.cx = cam.cx; v.cy = cam.cy;
  v.W = cam.width; v.H = cam.height;
  v.znear = znear;
  return v;
}

__device__ __forceinline__ float node_screen(const HierView& v, const float4 m, const float4 so, bool& inview) {
  return hier_node_screen(v.R, v.t, v.fx, v.fy, v.cx, v.cy, v.W, v.H, v.znear, m, so, inview);
}

struct HierArgs {
  float4* means4;
  float4* scale_opa;
  float4* quat;
  float* sh;
  int64_t sh_stride;
  int32_t* parent;
  int32_t* child;
  uint8_t* active;
  uint32_t* n_nodes;
  uint32_t* info;
  int64_t cap;
  // optional: Adam moments of the arena, zeroed for nodes whose flag changes
  float4* m_rows[2][3];
  float* m_sh[2];
  int64_t m_sh_stride;
  int nc;
  // workspace
  uint32_t* word;
  uint8_t* cand;
  uint8_t* mark;
  uint32_t* gpos;
  uint32_t *keys_a, *vals_a, *keys_b, *vals_b, *keys_out, *vals_out;
  uint32_t* ngroups;   // [chunks] groups per chunk
  uint32_t* gbase;     // [chunks] exclusive scan of ngroups
  int32_t* groups;     // [chunks][kMaxGroups][4] node ids, -1 padded
};

// Zeroes the Adam moments of node i (when the caller keeps them in the arena
// layout): a node entering or leaving the active set starts afresh.
__device__ __forceinline__ void zero_moments(const HierArgs& a, int64_t i) {
  for (int k = 0; k < 2; ++k) {
    if (!a.m_rows[k][0]) continue;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    a.m_rows[k][0][i] = z;
    a.m_rows[k][1][i] = z;
    a.m_rows[k][2][i] = z;
    for (int p = 0; p < 3 * a.nc; ++p) a.m_sh[k][(int64_t)p * a.m_sh_stride + i] = 0.f;
  }
}

__device__ __forceinline__ bool triggered(const uint32_t* word) {
  return 5ull * word[kWCand] > (unsigned long long)word[kWActive];
}

__global__ void k_hier_begin(HierArgs a) {
  if (threadIdx.x < kWords) a.word[threadIdx.x] = 0u;
  __syncthreads();
  if (threadIdx.x < 3) {
    a.word[kWBox + threadIdx.x] = 0xffffffffu;  // min (ordered)
    a.word[kWBox + 3 + threadIdx.x] = 0u;       // max (ordered)
  }
  if (threadIdx.x == 0) a.word[kWN] = min((uint32_t)a.cap, *a.n_nodes);
}

// 1. screen sizes and candidates, active and candidate counts
__global__ void __launch_bounds__(kHT) k_hier_screen(HierArgs a, const float* pose, gs_camera cam, float znear,
                                                     float tau_l) {
  const uint32_t n = a.word[kWN];
  const int64_t i = (int64_t)blockIdx.x * kHT + threadIdx.x;
  bool act = false, c = false;
  if (i < n) {
    act = a.active[i] != 0;
    if (act) {
      const HierView v = load_view(pose, cam, znear);
      bool in;
      c = node_screen(v, a.means4[i], a.scale_opa[i], in) < tau_l;
    }
    a.cand[i] = c ? 1 : 0;
  }
  const int na = __syncthreads_count(act), nc = __syncthreads_count(c);
  if (threadIdx.x == 0) {
    if (na) atomicAdd(&a.word[kWActive], (uint32_t)na);
    if (nc) atomicAdd(&a.word[kWCand], (uint32_t)nc);
  }
}

// 3a. parents to pull: inactive, every child a candidate (state before any pull)
__global__ void __launch_bounds__(kHT) k_hier_pull_mark(HierArgs a) {
  const uint32_t n = a.word[kWN];
  const int64_t p = (int64_t)blockIdx.x * kHT + threadIdx.x;
  if (p >= n) return;
  bool pull = false;
  if (triggered(a.word) && !a.active[p] && a.child[4 * p] >= 0) {
    pull = true;
    for (int k = 0; k < 4; ++k) {
      const int32_t c = a.child[4 * p + k];
      if (c >= 0 && (c >= (int64_t)n || !a.cand[c])) pull = false;
    }
  }
  a.mark[p] = pull ? 1 : 0;
}

// 3b. apply the pulls
__global__ void __launch_bounds__(kHT) k_hier_pull_apply(HierArgs a) {
  const uint32_t n = a.word[kWN];
  const int64_t p = (int64_t)blockIdx.x * kHT + threadIdx.x;
  const bool pull = p < n && a.mark[p];
  if (pull) {
    a.active[p] = 1;
    zero_moments(a, p);
    for (int k = 0; k < 4; ++k) {
      const int32_t c = a.child[4 * p + k];
      if (c >= 0) {
        a.active[c] = 0;
        a.cand[c] = 0;
        zero_moments(a, c);
      }
    }
  }
  const int np = __syncthreads_count(pull);
  if (threadIdx.x == 0 && np) atomicAdd(&a.word[kWPulled], (uint32_t)np);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.word[kWTrig] = triggered(a.word) ? 1u : 0u;
}

// 4a. the parentless candidates (in index order after the scan)
__global__ void __launch_bounds__(kHT) k_hier_gflag(HierArgs a) {
  const uint32_t n = a.word[kWN];
  const int64_t i = (int64_t)blockIdx.x * kHT + threadIdx.x;
  if (i >= n) return;
  a.gpos[i] = (triggered(a.word) && a.cand[i] && a.parent[i] < 0) ? 1u : 0u;
}

// 4b. compaction (gpos holds the exclusive scan) and the bounding box of the
// candidates' means
__global__ void __launch_bounds__(kHT) k_hier_compact(HierArgs a) {
  __shared__ uint32_t s[6];
  if (threadIdx.x < 3) {
    s[threadIdx.x] = 0xffffffffu;
    s[3 + threadIdx.x] = 0u;
  }
  __syncthreads();
  const uint32_t n = a.word[kWN];
  const int64_t i = (int64_t)blockIdx.x * kHT + threadIdx.x;
  if (i < n && a.cand[i] && a.parent[i] < 0 && triggered(a.word)) {
    a.vals_a[a.gpos[i]] = (uint32_t)i;
    const float4 m = a.means4[i];
    const uint32_t o[3] = {float_order(m.x), float_order(m.y), float_order(m.z)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(&s[k], o[k]);
      atomicMax(&s[3 + k], o[k]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    atomicMin(&a.word[kWBox + threadIdx.x], s[threadIdx.x]);
    atomicMax(&a.word[kWBox + 3 + threadIdx.x], s[3 + threadIdx.x]);
  }
}

// 4c. Morton codes of the candidates (keys), node ids (values, index order)
__global__ void __launch_bounds__(kHT) k_hier_morton(HierArgs a) {
  const uint32_t G = a.word[kWG];
  const int64_t q = (int64_t)blockIdx.x * kHT + threadIdx.x;
  if (q == 0) a.word[kWChunks] = (G + kChunk - 1) / kChunk;
  if (q >= G) return;
  float lo[3], scale[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = float_unorder(a.word[kWBox + k]);
    const float ext = __fsub_rn(float_unorder(a.word[kWBox + 3 + k]), lo[k]);
    scale[k] = ext > 0.f ? __fdiv_rn(1024.0f, ext) : 0.f;
  }
  const float4 m = a.means4[a.vals_a[q]];
  a.keys_a[q] = spread10(quantise10(m.x, lo[0], scale[0])) | (spread10(quantise10(m.y, lo[1], scale[1])) << 1) |
                (spread10(quantise10(m.z, lo[2], scale[2])) << 2);
}

// 4d. one warp per chunk of 64 Morton-consecutive candidates: 3 nearest by
// squared distance (ties by position), then the greedy grouping on lane 0
__global__ void __launch_bounds__(128) k_hier_group(HierArgs a) {
  __shared__ float s_m[4][kChunk][3];
  __shared__ uint8_t s_knn[4][kChunk][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * 4 + warp;
  const uint32_t G = a.word[kWG];
  if (c * kChunk >= G) return;  // warp-uniform
  const int len = (int)min((int64_t)kChunk, (int64_t)G - c * kChunk);
  for (int q = lane; q < len; q += 32) {
    const float4 m = a.means4[a.vals_out[c * kChunk + q]];
    s_m[warp][q][0] = m.x;
    s_m[warp][q][1] = m.y;
    s_m[warp][q][2] = m.z;
  }
  __syncwarp();
  for (int q = lane; q < len; q += 32) {
    float best[3] = {INFINITY, INFINITY, INFINITY};
    int idx[3] = {-1, -1, -1};
    int nb = 0;
    for (int b = 0; b < len; ++b) {
      if (b == q) continue;
      const float dx = __fsub_rn(s_m[warp][b][0], s_m[warp][q][0]);
      const float dy = __fsub_rn(s_m[warp][b][1], s_m[warp][q][1]);
      const float dz = __fsub_rn(s_m[warp][b][2], s_m[warp][q][2]);
      float d = __fmul_rn(dx, dx);
      d = __fadd_rn(d, __fmul_rn(dy, dy));
      d = __fadd_rn(d, __fmul_rn(dz, dz));
      // sorted insertion into the 3 best (strict <: earlier positions win ties)
      int pos = nb;
      while (pos > 0 && d < best[pos - 1]) --pos;
      if (pos >= 3) continue;
      for (int k = min(nb, 2); k > pos; --k) {
        best[k] = best[k - 1];
        idx[k] = idx[k - 1];
      }
      best[pos] = d;
      idx[pos] = b;
      nb = min(nb + 1, 3);
    }
    for (int k = 0; k < 3; ++k) s_knn[warp][q][k] = (uint8_t)(idx[k] < 0 ? 0xff : idx[k]);
  }
  __syncwarp();
  if (lane == 0) {
    uint64_t taken = 0;
    int ng = 0;
    int32_t* out = a.groups + c * (int64_t)kMaxGroups * 4;
    for (int q = 0; q < len; ++q) {
      if ((taken >> q) & 1ull) continue;
      int members[4] = {q, -1, -1, -1};
      int k = 1;
      taken |= 1ull << q;
      for (int j = 0; j < 3; ++j) {
        const int b = s_knn[warp][q][j];
        if (b != 0xff && !((taken >> b) & 1ull)) {
          taken |= 1ull << b;
          members[k++] = b;
        }
      }
      if (k >= 2) {
        for (int j = 0; j < 4; ++j)
          out[4 * ng + j] = j < k ? (int32_t)a.vals_out[c * kChunk + members[j]] : -1;
        ++ng;
      } else {
        taken &= ~(1ull << q);  // alone: stays available to later candidates
      }
    }
    a.ngroups[c] = (uint32_t)ng;
  }
}

// 5. one thread per group: the merged parent (geometry, opacity, SH) and the links
template <int NC>
__global__ void __launch_bounds__(kHT) k_hier_merge(HierArgs a) {
  const uint32_t chunks = a.word[kWChunks];
  const int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x;
  const int64_t c = t / kMaxGroups, g = t % kMaxGroups;
  if (c >= chunks || g >= a.ngroups[c]) return;
  const uint32_t n = a.word[kWN];
  const uint32_t total = a.word[kWGroups];
  if ((int64_t)n + total > a.cap) {  // no room: no merge at all (the set stays a cut)
    if (t == 0) atomicOr(&a.word[kWStatus], 1u);
    return;
  }
  const int64_t node = (int64_t)n + a.gbase[c] + g;
  const int32_t* mem = a.groups + (c * kMaxGroups + g) * 4;
  int64_t ch[4];
  int k = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ch[j] = mem[j];
    if (mem[j] >= 0) ++k;
  }
  float w[4], W = 0.f, o2 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w[j] = 0.f;
    if (j < k) {
      const float4 so = a.scale_opa[ch[j]];
      const float4 mu = a.means4[ch[j]];
      w[j] = 1.0f / (1.0f + expf(-so.w));
      W += w[j];
      o2 += w[j] * w[j];
      mx += w[j] * mu.x; my += w[j] * mu.y; mz += w[j] * mu.z;
    }
  }
  const float iW = 1.0f / W;
  mx *= iW; my *= iW; mz *= iW;
  float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx xy xz yy yz zz
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < k) {
      const float4 mu = a.means4[ch[j]], so = a.scale_opa[ch[j]], q4 = a.quat[ch[j]];
      const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
      float R[9];
      quat_rot(q4.x * qn, q4.y * qn, q4.z * qn, q4.w * qn, R);
      const float v[3] = {expf(2.f * so.x), expf(2.f * so.y), expf(2.f * so.z)};
      const float d[3] = {mu.x - mx, mu.y - my, mu.z - mz};
      const int rr[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int r = rr[e], cl = cc[e];
        const float s = R[3 * r] * v[0] * R[3 * cl] + R[3 * r + 1] * v[1] * R[3 * cl + 1] +
                        R[3 * r + 2] * v[2] * R[3 * cl + 2];
        C[e] += w[j] * (s + d[r] * d[cl]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) C[e] *= iW;
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
  for (int p = 0; p < 3 * NC; ++p) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < k) acc += w[j] * a.sh[(int64_t)p * a.sh_stride + ch[j]];
    a.sh[(int64_t)p * a.sh_stride + node] = acc * iW;
  }
  a.parent[node] = -1;
  a.active[node] = 1;
  zero_moments(a, node);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a.child[4 * node + j] = (int32_t)ch[j];
    if (j < k) {
      a.parent[ch[j]] = (int32_t)node;
      a.active[ch[j]] = 0;
      zero_moments(a, ch[j]);
    }
  }
  atomicAdd(&a.word[kWGrouped], (uint32_t)k);
}

// end of the analysis: the node count and the summary words
__global__ void k_hier_end(HierArgs a) {
  if (threadIdx.x != 0) return;
  const uint32_t n = a.word[kWN];
  const bool ok = !(a.word[kWStatus] & 1u) && (int64_t)n + a.word[kWGroups] <= a.cap;
  const uint32_t groups = triggered(a.word) && ok ? a.word[kWGroups] : 0u;
  *a.n_nodes = n + groups;
  if (a.info) {
    a.info[0] = n + groups;
    a.info[1] = a.word[kWTrig];
    a.info[2] = a.word[kWCand];
    a.info[3] = a.word[kWActive];
    a.info[4] = a.word[kWPulled];
    a.info[5] = groups;
    a.info[6] = a.word[kWGrouped];
    a.info[7] = a.word[kWStatus];
  }
}

// Reload pass: mark the active nodes with children that are in view with S >
// tau_h (state before the pass), then replace them by their children.
__global__ void __launch_bounds__(kHT) k_hier_refine_mark(HierArgs a, const float* pose, gs_camera cam, float znear,
                                                          float tau_h, int pass) {
  const uint32_t n = min((uint32_t)a.cap, *a.n_nodes);
  if (pass > 0 && a.word[kWChanged] == 0u) return;  // the previous pass changed nothing: a fixpoint
  const int64_t i = (int64_t)blockIdx.x * kHT + threadIdx.x;
  if (i >= n) return;
  bool e = false;
  if (a.active[i] && a.child[4 * i] >= 0) {
    const HierView v = load_view(pose, cam, znear);
    bool in;
    const float S = node_screen(v, a.means4[i], a.scale_opa[i], in);
    e = in && S > tau_h;
  }
  a.mark[i] = e ? 1 : 0;
}

__global__ void k_hier_refine_reset(HierArgs a, int pass) {
  if (threadIdx.x == 0 && (pass == 0 || a.word[kWChanged] != 0u)) a.word[kWChanged + 1] = 0u;
}

__global__ void __launch_bounds__(kHT) k_hier_refine_apply(HierArgs a, int pass) {
  if (pass > 0 && a.word[kWChanged] == 0u) return;
  const uint32_t n = min((uint32_t)a.cap, *a.n_nodes);
  const int64_t i = (int64_t)blockIdx.x * kHT + threadIdx.x;
  const bool e = i < n && a.mark[i];
  if (e) {
    a.active[i] = 0;
    zero_moments(a, i);
    for (int k = 0; k < 4; ++k) {
      const int32_t c = a.child[4 * i + k];
      if (c >= 0) {
        a.active[c] = 1;
        zero_moments(a, c);
      }
    }
  }
  const int cnt = __syncthreads_count(e);
  if (threadIdx.x == 0 && cnt) atomicAdd(&a.word[kWChanged + 1], (uint32_t)cnt);
}

// the changes of this pass become the previous pass's count; the total goes to info[0]
__global__ void k_hier_refine_step(HierArgs a, int pass) {
  if (threadIdx.x != 0) return;
  if (pass > 0 && a.word[kWChanged] == 0u) return;
  a.word[kWChanged] = a.word[kWChanged + 1];
  if (a.info) a.info[0] += a.word[kWChanged + 1];
}

__global__ void k_hier_refine_begin(HierArgs a) {
  if (threadIdx.x == 0) {
    a.word[kWChanged] = 0u;
    a.word[kWChanged + 1] = 0u;
    if (a.info) a.info[0] = 0u;
  }
}

struct HierWs {
  uint32_t* word;
  uint8_t *cand, *mark;
  uint32_t *gpos, *keys_a, *vals_a, *keys_b, *vals_b, *keys_out, *vals_out, *ngroups, *gbase;
  int32_t* groups;
  void *scan, *radix;
  size_t bytes;
};

HierWs hier_layout(char* base, int64_t cap) {
  HierWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1), 256);
    return p;
  };
  const size_t c = (size_t)std::max<int64_t>(1, cap);
  const size_t chunks = (c + kChunk - 1) / kChunk;
  w.word = (uint32_t*)take(kWords * sizeof(uint32_t));
  w.cand = (uint8_t*)take(c);
  w.mark = (uint8_t*)take(c);
  w.gpos = (uint32_t*)take(4 * c);
  w.keys_a = (uint32_t*)take(4 * c); w.vals_a = (uint32_t*)take(4 * c);
  w.keys_b = (uint32_t*)take(4 * c); w.vals_b = (uint32_t*)take(4 * c);
  w.keys_out = (uint32_t*)take(4 * c); w.vals_out = (uint32_t*)take(4 * c);
  w.ngroups = (uint32_t*)take(4 * chunks);
  w.gbase = (uint32_t*)take(4 * chunks);
  w.groups = (int32_t*)take(sizeof(int32_t) * 4 * kMaxGroups * chunks);
  w.scan = take(scan_workspace((int64_t)c));
  w.radix = take(radix_workspace((int64_t)c));
  w.bytes = off;
  return w;
}

HierArgs hier_args(const gs_grads& nodes, const gs_hier& h, const gs_grads* m, const gs_grads* v, void* ws) {
  HierArgs a{};
  a.means4 = reinterpret_cast<float4*>(nodes.means4);
  a.scale_opa = reinterpret_cast<float4*>(nodes.scale_opa);
  a.quat = reinterpret_cast<float4*>(nodes.quat);
  a.sh = nodes.sh;
  a.sh_stride = nodes.sh_stride > 0 ? nodes.sh_stride : nodes.n;
  a.parent = h.parent;
  a.child = h.child;
  a.active = h.active;
  a.n_nodes = h.n_nodes;
  a.info = h.info;
  a.cap = h.capacity;
  a.nc = (nodes.sh_degree + 1) * (nodes.sh_degree + 1);
  const gs_grads* mv[2] = {m, v};
  for (int k = 0; k < 2; ++k) {
    if (!mv[k]) continue;
    a.m_rows[k][0] = reinterpret_cast<float4*>(mv[k]->means4);
    a.m_rows[k][1] = reinterpret_cast<float4*>(mv[k]->scale_opa);
    a.m_rows[k][2] = reinterpret_cast<float4*>(mv[k]->quat);
    a.m_sh[k] = mv[k]->sh;
    a.m_sh_stride = mv[k]->sh_stride > 0 ? mv[k]->sh_stride : mv[k]->n;
  }
  if (ws) {
    HierWs w = hier_layout(static_cast<char*>(ws), h.capacity);
    a.word = w.word;
    a.cand = w.cand;
    a.mark = w.mark;
    a.gpos = w.gpos;
    a.keys_a = w.keys_a; a.vals_a = w.vals_a; a.keys_b = w.keys_b; a.vals_b = w.vals_b;
    a.keys_out = w.keys_out; a.vals_out = w.vals_out;
    a.ngroups = w.ngroups;
    a.gbase = w.gbase;
    a.groups = w.groups;
  }
  return a;
}

}  // namespace

size_t hier_workspace_bytes(int64_t cap) { return hier_layout(nullptr, cap).bytes; }

gs_status launch_hier_analyze(const gs_grads& nodes, const gs_hier& h, const gs_grads* m, const gs_grads* v,
                              const float* pose, const gs_camera& cam, float znear, float tau_l, void* ws,
                              cudaStream_t s) {
  HierWs w = hier_layout(static_cast<char*>(ws), h.capacity);
  HierArgs a = hier_args(nodes, h, m, v, ws);
  const unsigned grid = (unsigned)std::max<int64_t>(1, (h.capacity + kHT - 1) / kHT);
  const int64_t chunks_cap = (h.capacity + kChunk - 1) / kChunk;
  k_hier_begin<<<1, 64, 0, s>>>(a);
  k_hier_screen<<<grid, kHT, 0, s>>>(a, pose, cam, znear, tau_l);
  k_hier_pull_mark<<<grid, kHT, 0, s>>>(a);
  k_hier_pull_apply<<<grid, kHT, 0, s>>>(a);
  k_hier_gflag<<<grid, kHT, 0, s>>>(a);
  gs_status st = launch_scan(w.gpos, 1, w.gpos, 1, w.word + kWN, h.capacity, w.word + kWG, w.scan, s);
  if (st != GS_OK) return st;
  k_hier_compact<<<grid, kHT, 0, s>>>(a);
  k_hier_morton<<<grid, kHT, 0, s>>>(a);
  st = launch_radix_sort(w.keys_a, w.vals_a, w.keys_b, w.vals_b, w.keys_out, w.vals_out, w.word + kWG, h.capacity,
                         30, w.radix, s);
  if (st != GS_OK) return st;
  k_hier_group<<<(unsigned)std::max<int64_t>(1, (chunks_cap + 3) / 4), 128, 0, s>>>(a);
  st = launch_scan(w.ngroups, 1, w.gbase, 1, w.word + kWChunks, chunks_cap, w.word + kWGroups, w.scan, s);
  if (st != GS_OK) return st;
  const unsigned mgrid = (unsigned)std::max<int64_t>(1, (chunks_cap * kMaxGroups + kHT - 1) / kHT);
  switch (nodes.sh_degree) {
    case 0: k_hier_merge<1><<<mgrid, kHT, 0, s>>>(a); break;
    case 1: k_hier_merge<4><<<mgrid, kHT, 0, s>>>(a); break;
    case 2: k_hier_merge<9><<<mgrid, kHT, 0, s>>>(a); break;
    default: k_hier_merge<16><<<mgrid, kHT, 0, s>>>(a); break;
  }
  k_hier_end<<<1, 32, 0, s>>>(a);
  return check_launch("hier_analyze");
}

gs_status launch_hier_refine(const gs_grads& nodes, const gs_hier& h, const gs_grads* m, const gs_grads* v,
                             const float* pose, const gs_camera& cam, float znear, float tau_h, int passes, void* ws,
                             cudaStream_t s) {
  HierArgs a = hier_args(nodes, h, m, v, ws);
  const unsigned grid = (unsigned)std::max<int64_t>(1, (h.capacity + kHT - 1) / kHT);
  k_hier_refine_begin<<<1, 32, 0, s>>>(a);
  for (int p = 0; p < passes; ++p) {
    k_hier_refine_mark<<<grid, kHT, 0, s>>>(a, pose, cam, znear, tau_h, p);
    k_hier_refine_reset<<<1, 32, 0, s>>>(a, p);
    k_hier_refine_apply<<<grid, kHT, 0, s>>>(a, p);
    k_hier_refine_step<<<1, 32, 0, s>>>(a, p);
  }
  return check_launch("hier_refine");
}

}  // namespace gs
