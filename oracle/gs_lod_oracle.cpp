// FP64 CPU oracle of the level-of-detail hierarchy over the Gaussians.
//
// TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Parity reference for the CUDA
// hierarchy kernels; only the test suite may load it.  It shares no code,
// header, table or constant generator with the CUDA sources.
//
// What it computes (Sec. 6, the progressive Gaussian hierarchy: coarse nodes
// hold the parameters of a merged group of children, and rendering descends
// from the roots until a node's screen size falls below tau = 1 px or a leaf
// is reached).  The paper merges groups of 4 nearest neighbours with a
// KL-divergence criterion; the hierarchy built here has three levels (leaves,
// level 1, level 2) whose coarse nodes each merge up to 8 children by moment
// matching.  Readings (each listed in the design notes):
//   grouping    leaves in Morton order of their means (10 bits per axis over
//               the leaves' bounding box, quantised in single precision, ties
//               by index); consecutive runs of 8 share a level-1 parent; runs
//               of 8 consecutive level-1 nodes share a level-2 parent
//   weights     w_i = opacity_i = sigmoid(logit_i)
//   merge       mean = sum w mu / W; covariance = sum w (Sigma_i + d d^T) / W
//               with d = mu_i - mean (the mixture's first two moments);
//               SH = sum w c / W; opacity = min(0.99, sum w o / W)
//   factors     Sigma = V diag(lambda) V^T, scales = sqrt(lambda), V a rotation
//   screen size S = f_x * 3 * max_k scale_k / t_z; S = +inf when t_z <= znear
//   cut         a node is rendered iff (it is a leaf or S < tau) and every
//               ancestor has S >= tau
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <numeric>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Morton codes in single precision (the quantisation decides an integer, so
// it is taken in the kernel's precision).
// ---------------------------------------------------------------------------
uint32_t spread10(uint32_t v) {
  // bit i of v goes to bit 3i
  uint32_t r = 0;
  for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1u) << (3 * i);
  return r;
}

uint32_t quantise10(float x, float lo, float scale) {
  const float t = (x - lo) * scale;
  float f = std::floor(t);
  if (!(f >= 0.f)) f = 0.f;
  if (f > 1023.f) f = 1023.f;
  return (uint32_t)f;
}

void morton_codes(int64_t n, const float* means, std::vector<uint32_t>& code) {
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = std::numeric_limits<float>::infinity();
    hi[a] = -std::numeric_limits<float>::infinity();
  }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], means[3 * i + a]);
      hi[a] = std::max(hi[a], means[3 * i + a]);
    }
  float scale[3];
  for (int a = 0; a < 3; ++a) {
    const float ext = hi[a] - lo[a];
    scale[a] = ext > 0.f ? 1024.0f / ext : 0.f;
  }
  code.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t qx = quantise10(means[3 * i], lo[0], scale[0]);
    const uint32_t qy = quantise10(means[3 * i + 1], lo[1], scale[1]);
    const uint32_t qz = quantise10(means[3 * i + 2], lo[2], scale[2]);
    code[i] = spread10(qx) | (spread10(qy) << 1) | (spread10(qz) << 2);
  }
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
void quat_to_rot(const double* q, double* R) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Sigma = R diag(exp(2 s)) R^T, as a full 3x3 (row-major).
void covariance(const double* lsc, const double* q, double* S) {
  double R[9];
  quat_to_rot(q, R);
  const double v[3] = {std::exp(2 * lsc[0]), std::exp(2 * lsc[1]), std::exp(2 * lsc[2])};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * v[k] * R[3 * c + k];
      S[3 * r + c] = acc;
    }
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3: A = V diag(lam) V^T,
// columns of V are the eigenvectors.
void jacobi3(const double* A_in, double* lam, double* V) {
  double A[9];
  std::memcpy(A, A_in, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    const double scale = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-34 * scale || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double apq = A[3 * p + q];
        if (apq == 0.0) continue;
        const double theta = (A[3 * q + q] - A[3 * p + p]) / (2 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        const double c = 1 / std::sqrt(t * t + 1), s = t * c;
        // A <- J^T A J with the rotation in the (p, q) plane
        for (int k = 0; k < 3; ++k) {
          const double akp = A[3 * k + p], akq = A[3 * k + q];
          A[3 * k + p] = c * akp - s * akq;
          A[3 * k + q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[3 * p + k], aqk = A[3 * q + k];
          A[3 * p + k] = c * apk - s * aqk;
          A[3 * q + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[3 * k + p], vkq = V[3 * k + q];
          V[3 * k + p] = c * vkp - s * vkq;
          V[3 * k + q] = s * vkp + c * vkq;
        }
      }
  }
  lam[0] = A[0];
  lam[1] = A[4];
  lam[2] = A[8];
}

// Unit quaternion (w,x,y,z) of a rotation matrix (row-major), w >= 0.
void rot_to_quat(const double* R, double* q) {
  const double tr = R[0] + R[4] + R[8];
  double w, x, y, z;
  if (tr > 0) {
    const double s = std::sqrt(tr + 1.0) * 2;
    w = 0.25 * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const double s = std::sqrt(1.0 + R[0] - R[4] - R[8]) * 2;
    w = (R[7] - R[5]) / s; x = 0.25 * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const double s = std::sqrt(1.0 + R[4] - R[0] - R[8]) * 2;
    w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25 * s; z = (R[5] + R[7]) / s;
  } else {
    const double s = std::sqrt(1.0 + R[8] - R[0] - R[4]) * 2;
    w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25 * s;
  }
  if (w < 0) { w = -w; x = -x; y = -y; z = -z; }
  const double n = std::sqrt(w * w + x * x + y * y + z * z);
  q[0] = w / n; q[1] = x / n; q[2] = y / n; q[3] = z / n;
}

double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }

// Moment-matching merge of k children.
void merge(int k, const double* mu, const double* lsc, const double* quat, const double* opl, const double* sh,
           int nsh, double* mean, double* cov6, double* lsc_out, double* quat_out, double* opl_out,
           double* sh_out) {
  double W = 0, m[3] = {0, 0, 0}, o = 0;
  for (int i = 0; i < k; ++i) {
    const double w = sigmoid(opl[i]);
    W += w;
    for (int a = 0; a < 3; ++a) m[a] += w * mu[3 * i + a];
    o += w * w;
  }
  for (int a = 0; a < 3; ++a) m[a] /= W;
  double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < k; ++i) {
    const double w = sigmoid(opl[i]);
    double S[9];
    covariance(lsc + 3 * i, quat + 4 * i, S);
    const double d[3] = {mu[3 * i] - m[0], mu[3 * i + 1] - m[1], mu[3 * i + 2] - m[2]};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) C[3 * r + c] += w * (S[3 * r + c] + d[r] * d[c]);
  }
  for (int t = 0; t < 9; ++t) C[t] /= W;
  for (int a = 0; a < 3; ++a) mean[a] = m[a];
  cov6[0] = C[0]; cov6[1] = C[1]; cov6[2] = C[2]; cov6[3] = C[4]; cov6[4] = C[5]; cov6[5] = C[8];
  for (int j = 0; j < nsh; ++j) {
    double acc = 0;
    for (int i = 0; i < k; ++i) acc += sigmoid(opl[i]) * sh[(int64_t)i * nsh + j];
    sh_out[j] = acc / W;
  }
  const double op = std::min(0.99, o / W);
  *opl_out = std::log(op / (1 - op));
  double lam[3], V[9];
  jacobi3(C, lam, V);
  const double det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                     V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (det < 0)
    for (int r = 0; r < 3; ++r) V[3 * r + 2] = -V[3 * r + 2];
  for (int a = 0; a < 3; ++a) lsc_out[a] = 0.5 * std::log(std::max(lam[a], 1e-300));
  rot_to_quat(V, quat_out);
}

}  // namespace

extern "C" {

// Morton grouping of n points (float32 means [n][3]): order[i] = index of the
// i-th point in (code, index) order; code[i] = the point's Morton code.
void orc_lod_morton(int64_t n, const float* means, uint32_t* code_out, int64_t* order) {
  std::vector<uint32_t> code;
  morton_codes(n, means, code);
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
  for (int64_t i = 0; i < n; ++i) {
    code_out[i] = code[i];
    order[i] = idx[i];
  }
}

// Moment-matching merge of k children (double inputs, natural layouts:
// means [k][3], log-scales [k][3], quats [k][4] (w,x,y,z), logits [k],
// SH [k][nsh]); outputs the parent's mean, covariance (xx, xy, xz, yy, yz,
// zz), log-scales, quaternion, opacity logit and SH.
void orc_lod_merge(int k, const double* mu, const double* lsc, const double* quat, const double* opl,
                   const double* sh, int nsh, double* mean, double* cov6, double* lsc_out, double* quat_out,
                   double* opl_out, double* sh_out) {
  merge(k, mu, lsc, quat, opl, sh, nsh, mean, cov6, lsc_out, quat_out, opl_out, sh_out);
}

// The three-level hierarchy over n leaves.  Node numbering: leaves [0, n),
// level 1 [n, n + n1), level 2 [n + n1, n + n1 + n2).  means32: the leaves'
// float32 means (grouping); the other inputs in double, natural layouts.
// parent[node] = parent node or -1 (level 2).  Parent parameters are written
// for the n1 + n2 coarse nodes in node order: p_means [.][3], p_cov [.][6],
// p_lsc [.][3], p_quat [.][4], p_opl [.], p_sh [.][nsh].  Returns n1 + n2;
// *n1_out = n1.
int64_t orc_lod_build(int64_t n, int nsh, const float* means32, const double* mu, const double* lsc,
                      const double* quat, const double* opl, const double* sh, int64_t* parent, int64_t* n1_out,
                      double* p_means, double* p_cov, double* p_lsc, double* p_quat, double* p_opl,
                      double* p_sh) {
  std::vector<uint32_t> code;
  morton_codes(n, means32, code);
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
  const int64_t n1 = (n + 7) / 8, n2 = (n1 + 7) / 8;
  *n1_out = n1;
  // gather helpers
  auto merge_group = [&](const std::vector<int64_t>& members, const double* gmu, const double* glsc,
                         const double* gquat, const double* gopl, const double* gsh, int64_t out) {
    const int k = (int)members.size();
    std::vector<double> m(3 * k), l(3 * k), q(4 * k), o(k), s((size_t)k * nsh);
    for (int i = 0; i < k; ++i) {
      const int64_t c = members[i];
      for (int a = 0; a < 3; ++a) { m[3 * i + a] = gmu[3 * c + a]; l[3 * i + a] = glsc[3 * c + a]; }
      for (int a = 0; a < 4; ++a) q[4 * i + a] = gquat[4 * c + a];
      o[i] = gopl[c];
      for (int j = 0; j < nsh; ++j) s[(size_t)i * nsh + j] = gsh[c * nsh + j];
    }
    merge(k, m.data(), l.data(), q.data(), o.data(), s.data(), nsh, p_means + 3 * out, p_cov + 6 * out,
          p_lsc + 3 * out, p_quat + 4 * out, p_opl + out, p_sh + out * nsh);
  };
  for (int64_t g = 0; g < n1; ++g) {
    std::vector<int64_t> members;
    for (int64_t i = 8 * g; i < std::min(n, 8 * g + 8); ++i) {
      members.push_back(order[i]);
      parent[order[i]] = n + g;
    }
    merge_group(members, mu, lsc, quat, opl, sh, g);
  }
  for (int64_t g = 0; g < n2; ++g) {
    std::vector<int64_t> members;
    for (int64_t i = 8 * g; i < std::min(n1, 8 * g + 8); ++i) {
      members.push_back(i);  // index into the level-1 parameter arrays
      parent[n + i] = n + n1 + g;
    }
    merge_group(members, p_means, p_lsc, p_quat, p_opl, p_sh, n1 + g);
  }
  for (int64_t g = 0; g < n2; ++g) parent[n + n1 + g] = -1;
  return n1 + n2;
}

// Screen size of every node and the LoD cut for one camera.  nodes: means
// [N][3], log-scales [N][3]; parent[N] (-1 for roots); nodes with index <
// n_leaf are leaves.  pose12 = [R | t] row-major.  selected[i] = 1 if node i
// is rendered; amb[i] = 1 if S of the node or of an ancestor lies within
// 1e-5 tau of tau (a decision single precision may take either way).
void orc_lod_cut(int64_t N, int64_t n_leaf, const double* mu, const double* lsc, const int64_t* parent,
                 const double* pose12, double fx, double znear, double tau, double* screen, uint8_t* selected,
                 uint8_t* amb) {
  for (int64_t i = 0; i < N; ++i) {
    const double* P = pose12;
    const double tz = P[8] * mu[3 * i] + P[9] * mu[3 * i + 1] + P[10] * mu[3 * i + 2] + P[11];
    const double smax = std::exp(std::max(lsc[3 * i], std::max(lsc[3 * i + 1], lsc[3 * i + 2])));
    screen[i] = tz <= znear ? std::numeric_limits<double>::infinity() : fx * 3.0 * smax / tz;
  }
  for (int64_t i = 0; i < N; ++i) {
    bool ok = i < n_leaf || screen[i] < tau;
    bool a = std::fabs(screen[i] - tau) <= 1e-5 * tau;
    for (int64_t p = parent[i]; p >= 0; p = parent[p]) {
      ok = ok && screen[p] >= tau;
      a = a || std::fabs(screen[p] - tau) <= 1e-5 * tau;
    }
    selected[i] = ok ? 1 : 0;
    amb[i] = a ? 1 : 0;
  }
}

}  // extern "C"

// ===========================================================================
// Progressive hierarchy (Sec. 6.1 "Adaptive Gaussian Merging and Retrieval",
// Sec. 6.2): an active set of nodes (leaves and merged intermediate nodes)
// that is a cut of the forest (every leaf has exactly one active node on its
// path to its root), coarsened when a keyframe is analysed and refined where
// a view needs it.  Nodes hold Gaussian parameters, a parent id (-1: root)
// and up to 4 child ids (-1: none).
//
// Steps of one analysis from a keyframe's camera, in the paper's order:
//   1. screen size S_i = f_x * 3 * max_k scale_k / t_z of every active node
//      (+inf at or behind the near plane); candidates: active, S_i < tau_l
//      (tau_l = 0.5 px);
//   2. merging runs only when more than 20% of the active nodes are
//      candidates (5 |C| > |A|);
//   3. pull: an inactive parent all of whose children are candidates becomes
//      active again and its children inactive (no new node);
//   4. the remaining candidates without a parent are grouped with their 3
//      nearest candidates (groups of up to 4): candidates in Morton order of
//      their means (10 bits per axis over the candidates' bounding box,
//      single precision, ties by index), cut into chunks of 64 consecutive
//      candidates; within a chunk the 3 nearest by squared distance of the
//      single-precision means (summed x, y, z in that order; ties by Morton
//      position); then, in Morton order, a candidate not yet grouped takes
//      those of its 3 nearest that are not yet grouped (a candidate left
//      alone stays ungrouped and available to later ones);
//   5. each group of 2-4 becomes a new parent node (moment-matching merge,
//      as the static hierarchy), active, with the children inactive; new
//      nodes are numbered after the existing ones in Morton order of their
//      first child.
// Readings: the paper's "4 closest" are the candidate and its 3 nearest; its
// KL-divergence merge is read as the moment-matching merge; its fast KNN is
// exact within chunks of 64 Morton-consecutive candidates.
// Reload (Sec. 6.1, tau_h = 1): an active node with children that lies in
// view (t_z > znear and its projected centre within the image widened by S)
// and has S > tau_h is replaced in the active set by its children, repeated
// until no node changes.  The view cut of a render is that refinement
// applied to a copy of the active set.
// ===========================================================================
namespace {

constexpr int kHierChunk = 64;

struct HierView {
  double R[9], t[3], fx, fy, cx, cy, znear;
  int W, H;
};

HierView hier_view(const double* pose12, const double* intr, const int32_t* wh, double znear) {
  HierView v;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) v.R[3 * r + c] = pose12[4 * r + c];
    v.t[r] = pose12[4 * r + 3];
  }
  v.fx = intr[0]; v.fy = intr[1]; v.cx = intr[2]; v.cy = intr[3];
  v.W = wh[0]; v.H = wh[1];
  v.znear = znear;
  return v;
}

// Screen size and the in-view test of node i; *edge (optional) is set when
// the in-view decision lies within 1e-4 px of an image edge (single
// precision may take it either way).
void hier_screen(const HierView& v, const double* mu, const double* lsc, int64_t i, double* S, bool* inview,
                 bool* edge = nullptr) {
  const double* m = mu + 3 * i;
  double tc[3];
  for (int r = 0; r < 3; ++r) tc[r] = v.R[3 * r] * m[0] + v.R[3 * r + 1] * m[1] + v.R[3 * r + 2] * m[2] + v.t[r];
  if (edge) *edge = std::fabs(tc[2] - v.znear) <= 1e-6 * v.znear;
  if (!(tc[2] > v.znear)) {
    *S = std::numeric_limits<double>::infinity();
    *inview = false;
    return;
  }
  const double smax = std::exp(std::max(lsc[3 * i], std::max(lsc[3 * i + 1], lsc[3 * i + 2])));
  *S = v.fx * 3.0 * smax / tc[2];
  const double u = v.fx * tc[0] / tc[2] + v.cx, w = v.fy * tc[1] / tc[2] + v.cy;
  *inview = u >= -*S && u <= v.W + *S && w >= -*S && w <= v.H + *S;
  if (edge) {
    const double e = 1e-4 * (1.0 + *S);
    *edge = *edge || std::fabs(u + *S) <= e || std::fabs(u - v.W - *S) <= e || std::fabs(w + *S) <= e ||
            std::fabs(w - v.H - *S) <= e;
  }
}

bool near_rel(double a, double b, double rel) { return std::fabs(a - b) <= rel * std::fabs(b); }

// Refinement passes (each pass: every expandable active node with children,
// found on the state before the pass, is replaced by its children).
int64_t hier_refine_passes(int64_t n_nodes, const double* mu, const double* lsc, const int32_t* child,
                           uint8_t* active, const HierView& v, double tau_h, uint8_t* amb) {
  int64_t changed = 0;
  for (int pass = 0; pass < 64; ++pass) {
    std::vector<int64_t> expand;
    for (int64_t i = 0; i < n_nodes; ++i) {
      if (!active[i] || child[4 * i] < 0) continue;
      double S;
      bool in, edge;
      hier_screen(v, mu, lsc, i, &S, &in, &edge);
      if (amb && ((std::isfinite(S) && near_rel(S, tau_h, 1e-5)) || edge)) amb[i] = 1;
      if (in && S > tau_h) expand.push_back(i);
    }
    if (expand.empty()) break;
    for (int64_t i : expand) {
      active[i] = 0;
      for (int k = 0; k < 4; ++k)
        if (child[4 * i + k] >= 0) active[child[4 * i + k]] = 1;
    }
    changed += (int64_t)expand.size();
  }
  return changed;
}

}  // namespace

extern "C" {

// One analysis of the progressive hierarchy from a camera (steps 1-5 above).
// Node state of capacity `cap` rows, n_nodes in use: means32 [cap][3]
// (float; rewritten for new nodes), mu, lsc [cap][3], quat [cap][4], opl
// [cap], sh [cap][nsh] (double, natural layouts; new nodes appended),
// parent [cap], child [cap][4], active [cap] (updated).  pose12 [R | t],
// intr (fx, fy, cx, cy), wh (W, H).  S_out [cap]: screen sizes of the nodes
// active before the step (NaN elsewhere); amb [cap]: 1 where S lies within
// 1e-5 of tau_l (a decision single precision may take either way).
// info [8]: new n_nodes, triggered, candidates, active before, pulled parents,
// groups, grouped candidates, 0.  Returns 0, or 1 if the capacity is too small.
int orc_hier_analyze(int64_t n_nodes, int64_t cap, int nsh, float* means32, double* mu, double* lsc, double* quat,
                     double* opl, double* sh, int32_t* parent, int32_t* child, uint8_t* active,
                     const double* pose12, const double* intr, const int32_t* wh, double znear, double tau_l,
                     double* S_out, uint8_t* amb, int64_t* info) {
  const HierView v = hier_view(pose12, intr, wh, znear);
  std::memset(info, 0, 8 * sizeof(int64_t));
  info[0] = n_nodes;
  // 1. screen sizes and candidates
  std::vector<uint8_t> cand((size_t)n_nodes, 0);
  int64_t nA = 0, nC = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    S_out[i] = std::numeric_limits<double>::quiet_NaN();
    amb[i] = 0;
    if (!active[i]) continue;
    ++nA;
    bool in;
    hier_screen(v, mu, lsc, i, &S_out[i], &in);
    if (std::isfinite(S_out[i]) && near_rel(S_out[i], tau_l, 1e-5)) amb[i] = 1;
    if (S_out[i] < tau_l) {
      cand[i] = 1;
      ++nC;
    }
  }
  info[2] = nC;
  info[3] = nA;
  // 2. the trigger: more than 20% of the active nodes
  if (!(5 * nC > nA)) return 0;
  info[1] = 1;
  // 3. pull: inactive parents whose children are all candidates
  std::vector<int64_t> pulled;
  for (int64_t p = 0; p < n_nodes; ++p) {
    if (active[p] || child[4 * p] < 0) continue;
    bool all = true;
    for (int k = 0; k < 4; ++k) {
      const int32_t c = child[4 * p + k];
      if (c >= 0 && !cand[c]) all = false;
    }
    if (all) pulled.push_back(p);
  }
  for (int64_t p : pulled) {
    active[p] = 1;
    for (int k = 0; k < 4; ++k) {
      const int32_t c = child[4 * p + k];
      if (c >= 0) {
        active[c] = 0;
        cand[c] = 0;
      }
    }
  }
  info[4] = (int64_t)pulled.size();
  // 4. grouping of the remaining parentless candidates
  std::vector<int64_t> G;
  for (int64_t i = 0; i < n_nodes; ++i)
    if (cand[i] && parent[i] < 0) G.push_back(i);
  std::vector<float> gm(3 * G.size());
  for (size_t j = 0; j < G.size(); ++j)
    for (int a = 0; a < 3; ++a) gm[3 * j + a] = means32[3 * G[j] + a];
  std::vector<uint32_t> code;
  morton_codes((int64_t)G.size(), gm.data(), code);
  std::vector<int64_t> ord(G.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
  std::vector<std::vector<int64_t>> groups;  // node ids, leader first
  for (size_t c0 = 0; c0 < ord.size(); c0 += kHierChunk) {
    const size_t len = std::min((size_t)kHierChunk, ord.size() - c0);
    std::vector<int> knn(3 * len, -1);
    for (size_t a = 0; a < len; ++a) {
      const float* pa = &gm[3 * ord[c0 + a]];
      float best[3] = {0, 0, 0};
      int nb = 0;
      for (size_t b = 0; b < len; ++b) {
        if (b == a) continue;
        const float* pb = &gm[3 * ord[c0 + b]];
        const float dx = pb[0] - pa[0], dy = pb[1] - pa[1], dz = pb[2] - pa[2];
        float d = dx * dx;
        d = d + dy * dy;
        d = d + dz * dz;
        // insert (d, b) into the sorted top-3 (ties: smaller position first,
        // as b increases)
        int pos = nb;
        while (pos > 0 && d < best[pos - 1]) --pos;
        if (pos >= 3) continue;
        for (int q = std::min(nb, 2); q > pos; --q) {
          best[q] = best[q - 1];
          knn[3 * a + q] = knn[3 * a + q - 1];
        }
        best[pos] = d;
        knn[3 * a + pos] = (int)b;
        nb = std::min(nb + 1, 3);
      }
    }
    std::vector<uint8_t> taken(len, 0);
    for (size_t a = 0; a < len; ++a) {
      if (taken[a]) continue;
      std::vector<int64_t> g = {G[ord[c0 + a]]};
      taken[a] = 1;
      for (int q = 0; q < 3; ++q) {
        const int b = knn[3 * a + q];
        if (b >= 0 && !taken[b]) {
          taken[b] = 1;
          g.push_back(G[ord[c0 + b]]);
        }
      }
      if (g.size() >= 2) {
        groups.push_back(g);
      } else {
        taken[a] = 0;  // alone: stays available to later candidates
      }
    }
  }
  // 5. merge each group into a new active parent
  if (n_nodes + (int64_t)groups.size() > cap) return 1;
  int64_t grouped = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int64_t>& g = groups[gi];
    const int k = (int)g.size();
    const int64_t out = n_nodes + (int64_t)gi;
    std::vector<double> m(3 * k), l(3 * k), q(4 * k), o(k), s((size_t)k * nsh);
    for (int i = 0; i < k; ++i) {
      const int64_t c = g[i];
      for (int a = 0; a < 3; ++a) { m[3 * i + a] = mu[3 * c + a]; l[3 * i + a] = lsc[3 * c + a]; }
      for (int a = 0; a < 4; ++a) q[4 * i + a] = quat[4 * c + a];
      o[i] = opl[c];
      for (int j = 0; j < nsh; ++j) s[(size_t)i * nsh + j] = sh[c * nsh + j];
    }
    double cov6[6];
    merge(k, m.data(), l.data(), q.data(), o.data(), s.data(), nsh, mu + 3 * out, cov6, lsc + 3 * out,
          quat + 4 * out, opl + out, sh + out * nsh);
    for (int a = 0; a < 3; ++a) means32[3 * out + a] = (float)mu[3 * out + a];
    parent[out] = -1;
    active[out] = 1;
    for (int i = 0; i < 4; ++i) child[4 * out + i] = i < k ? (int32_t)g[i] : -1;
    for (int64_t c : g) {
      parent[c] = (int32_t)out;
      active[c] = 0;
    }
    grouped += k;
  }
  info[0] = n_nodes + (int64_t)groups.size();
  info[5] = (int64_t)groups.size();
  info[6] = grouped;
  return 0;
}

// Render cut (Sec. 6.2, rendering a stored hierarchy): start at the roots
// (nodes without a parent) and descend while a node is coarser than tau
// (S > tau, +inf at or behind the near plane) and has children; the nodes
// where the descent stops are rendered.  selected[i] = 1 iff node i does not
// descend and every ancestor does (independent of the active set).  amb[i] =
// 1 when S of the node or of an ancestor lies within 1e-5 of tau.  Returns
// the number of selected nodes.
int64_t orc_hier_render_cut(int64_t n_nodes, const double* mu, const double* lsc, const int32_t* parent,
                            const int32_t* child, const double* pose12, const double* intr, const int32_t* wh,
                            double znear, double tau, uint8_t* selected, uint8_t* amb) {
  const HierView v = hier_view(pose12, intr, wh, znear);
  std::vector<double> S((size_t)n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) {
    bool in;
    hier_screen(v, mu, lsc, i, &S[(size_t)i], &in);
  }
  auto descends = [&](int64_t k) { return child[4 * k] >= 0 && S[(size_t)k] > tau; };
  int64_t cnt = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    bool ok = !descends(i);
    bool a = near_rel(S[(size_t)i], tau, 1e-5);
    for (int32_t p = parent[i]; p >= 0; p = parent[p]) {
      ok = ok && descends(p);
      a = a || near_rel(S[(size_t)p], tau, 1e-5);
    }
    selected[i] = ok ? 1 : 0;
    amb[i] = a ? 1 : 0;
    cnt += ok ? 1 : 0;
  }
  return cnt;
}

// Reload (Sec. 6.1): refinement passes of the active set for one view.
// Returns the number of nodes replaced by their children; amb [n_nodes]
// marks nodes whose S lies within 1e-5 of tau_h.
int64_t orc_hier_refine(int64_t n_nodes, const double* mu, const double* lsc, const int32_t* child,
                        uint8_t* active, const double* pose12, const double* intr, const int32_t* wh, double znear,
                        double tau_h, uint8_t* amb) {
  const HierView v = hier_view(pose12, intr, wh, znear);
  for (int64_t i = 0; i < n_nodes; ++i) amb[i] = 0;
  return hier_refine_passes(n_nodes, mu, lsc, child, active, v, tau_h, amb);
}

}  // extern "C"
