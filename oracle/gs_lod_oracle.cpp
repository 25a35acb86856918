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
