// FP64 CPU oracle of the differentiable 3D Gaussian-splat rasterizer.
//
// TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This file is the parity reference for
// the CUDA path and the timed CPU baseline.  Only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
// table or constant generator with the CUDA sources, and it never reads anything
// the CUDA path produced.
//
// What it computes: the renderer that the paper's joint Gaussian optimisation
// runs every iteration (Sec. 5.2: the Gaussian model is trained for 30 iterations
// per keyframe with a custom differentiable splat renderer; the primitive holds
// position, opacity, rotation, scale and SH coefficients, Sec. 7).  The paper
// gives no renderer internals, so every step below is the plain definition of
// EWA splatting with front-to-back alpha compositing, with the standard
// 3DGS rasterizer constants: +0.3 px^2 dilation of the 2D covariance, alpha
// clamped at 0.99, splats with alpha < 1/255 skipped, compositing stopped before
// the splat that would bring transmittance below 1e-4.
//
// Readings of points the paper leaves open (each is listed in the design notes):
//   camera      OpenCV convention, pose = world->camera (R, tau), centre = -R^T tau
//   pixels      pixel (u,v) covers [u,u+1)x[v,v+1); its centre is (u+1/2, v+1/2)
//   near plane  culled when t_z <= znear
//   J guard     t_x/t_z, t_y/t_z clamped to +-1.3 (W/2)/f_x, +-1.3 (H/2)/f_y
//   support     r = ceil(3 sqrt(lambda_max)); a splat touches a pixel only if the
//               pixel centre lies in [m-r, m+r]^2 (so the image does not depend
//               on the tile shape)
//   tile rect   the tiles of [m-h, m+h] per axis, h = min(r, the half-width of
//               the bounding box of the ellipse where alpha can reach 1/255,
//               widened by 0.1% + 0.05 px): only tiles where a pixel can pass
//               the alpha test hold the splat, so the image is unchanged
//   SH          real orthonormal SH up to l = 3 without Condon-Shortley phase,
//               index k = l^2 + l + m; rgb = max(0, sum_k c_k Y_k(d) + 1/2)
//   quaternion  (w,x,y,z), normalised inside the forward
//   pose grad   left perturbation T <- Exp(xi) T, xi = (v, omega)
//   depth ties  equal keys keep Gaussian-id order (stable sort of id-ordered
//               emission)
//
// Everything is double precision.  The forward is written once as a template on
// the scalar type, so the same code evaluated on forward-mode dual numbers gives
// exact directional derivatives that pin the hand-derived analytic backward.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ----------------------------------------------------------------------------
// Scalar types: double and first-order dual numbers a + b eps, eps^2 = 0.
// ----------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

const double kPi = 3.14159265358979323846;

// ----------------------------------------------------------------------------
// Real spherical harmonics, l <= 3, from the closed form.
//   Y_l^m = K_l^m * sqrt2^[m!=0] * (d^|m| P_l / dz^|m|)(z) * {Re, 1, Im}((x+iy)^|m|)
// with K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), P_l from Rodrigues'
// formula P_l(z) = 1/(2^l l!) d^l/dz^l (z^2-1)^l, no Condon-Shortley phase.
// (x+iy)^m = sin^m(theta) e^{i m phi} on the unit sphere, so this equals the
// usual sin^m(theta) P_l^(m)(cos theta) cos/sin(m phi) form.
// ----------------------------------------------------------------------------
struct ShTable {
  double poly[4][4][4];  // [l][m][p]: coefficient of z^p in d^m P_l / dz^m
  double norm[4][4];     // [l][m]: K_l^m, times sqrt(2) for m > 0
  ShTable() {
    std::memset(poly, 0, sizeof(poly));
    for (int l = 0; l <= 3; ++l) {
      for (int m = 0; m <= l; ++m) {
        // (z^2-1)^l = sum_k C(l,k) (-1)^(l-k) z^(2k); differentiate l+m times.
        for (int k = 0; k <= l; ++k) {
          int p = 2 * k - l - m;
          if (p < 0) continue;
          double c = binom(l, k) * ((l - k) % 2 ? -1.0 : 1.0);
          c *= fact(2 * k) / fact(p);
          c /= std::pow(2.0, l) * fact(l);
          poly[l][m][p] += c;
        }
        double K = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * fact(l - m) / fact(l + m));
        norm[l][m] = (m == 0) ? K : K * std::sqrt(2.0);
      }
    }
  }
  static double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }
  static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }
};
const ShTable& sh_table() { static ShTable t; return t; }

template <class S>
void sh_eval(int deg, S x, S y, S z, S* Y) {
  const ShTable& tb = sh_table();
  // powers of (x + i y)
  S re[4], im[4];
  re[0] = S(1.0); im[0] = S(0.0);
  for (int m = 1; m <= 3; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int l = 0; l <= deg; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      S q = S(0.0), zp = S(1.0);
      for (int p = 0; p <= l - am; ++p) { q += zp * S(tb.poly[l][am][p]); zp = zp * z; }
      S az = (m > 0) ? re[am] : (m < 0 ? im[am] : S(1.0));
      Y[l * l + l + m] = S(tb.norm[l][am]) * q * az;
    }
  }
}

// ----------------------------------------------------------------------------
// Inputs
// ----------------------------------------------------------------------------
struct Scene {
  int64_t n;
  int deg, nc;                 // SH degree, coefficients per channel ((deg+1)^2)
  const double* means;         // [n][3]
  const double* lsc;           // [n][3] log-scales
  const double* quat;          // [n][4] (w,x,y,z), not necessarily unit
  const double* opl;           // [n]    opacity logits
  const double* sh;            // [n][3][nc]
};

template <class S>
struct View {
  S R[9];        // world->camera rotation, row-major
  S tau[3];      // world->camera translation
  double fx, fy, cx, cy;
  int W, H;
  int TX, TY;    // tiles
  int wx0, wy0, ww, wh;  // composited pixel window (the whole image by default)
};

struct Cfg {
  double znear;
  int tw, th;
  double bg[3];
  int clamp_j;
  // decision margins used to flag pixels whose discrete decisions a
  // single-precision implementation cannot be expected to reproduce
  double m_px, m_rel, m_r, m_near, m_lim, m_sh, m_depth;
};

// Per (view, Gaussian) projected splat
template <class S>
struct Proj {
  bool vis;
  S mx, my, A, B, C, opa, rgb[3], depth;
  double r;                     // integer-valued support half-width (px)
  int xlo, ylo, xhi, yhi;       // tile rect
  int clampbits;                // rgb channel c clamped at 0 -> bit c
  bool img_amb;                 // a per-Gaussian decision is within margin
  bool grad_amb;                // derivative discontinuity within margin
  bool r_amb;                   // 3 sqrt(lambda) within margin of an integer
  bool bin_amb;                 // rect edge within margin of a tile boundary
};

template <class S>
void scene_param(const Scene& sc, int64_t i, const Scene* tg, S mu[3], S ls[3], S q[4], S& ol,
                 std::vector<S>& shc);

template <>
void scene_param<double>(const Scene& sc, int64_t i, const Scene*, double mu[3], double ls[3],
                         double q[4], double& ol, std::vector<double>& shc) {
  for (int k = 0; k < 3; ++k) { mu[k] = sc.means[3 * i + k]; ls[k] = sc.lsc[3 * i + k]; }
  for (int k = 0; k < 4; ++k) q[k] = sc.quat[4 * i + k];
  ol = sc.opl[i];
  shc.resize(3 * sc.nc);
  for (int k = 0; k < 3 * sc.nc; ++k) shc[k] = sc.sh[3 * sc.nc * i + k];
}

template <>
void scene_param<Dual>(const Scene& sc, int64_t i, const Scene* tg, Dual mu[3], Dual ls[3],
                       Dual q[4], Dual& ol, std::vector<Dual>& shc) {
  for (int k = 0; k < 3; ++k) {
    mu[k] = Dual(sc.means[3 * i + k], tg->means[3 * i + k]);
    ls[k] = Dual(sc.lsc[3 * i + k], tg->lsc[3 * i + k]);
  }
  for (int k = 0; k < 4; ++k) q[k] = Dual(sc.quat[4 * i + k], tg->quat[4 * i + k]);
  ol = Dual(sc.opl[i], tg->opl[i]);
  shc.resize(3 * sc.nc);
  for (int k = 0; k < 3 * sc.nc; ++k)
    shc[k] = Dual(sc.sh[3 * sc.nc * i + k], tg->sh[3 * sc.nc * i + k]);
}

// Rotation matrix of a unit quaternion (w,x,y,z), row-major.
template <class S>
void quat_to_rot(const S q[4], S Rq[9]) {
  S w = q[0], x = q[1], y = q[2], z = q[3];
  Rq[0] = S(1.0) - S(2.0) * (y * y + z * z); Rq[1] = S(2.0) * (x * y - w * z); Rq[2] = S(2.0) * (x * z + w * y);
  Rq[3] = S(2.0) * (x * y + w * z); Rq[4] = S(1.0) - S(2.0) * (x * x + z * z); Rq[5] = S(2.0) * (y * z - w * x);
  Rq[6] = S(2.0) * (x * z - w * y); Rq[7] = S(2.0) * (y * z + w * x); Rq[8] = S(1.0) - S(2.0) * (x * x + y * y);
}

bool near_int(double x, double rel) {
  double f = std::floor(x + 0.5);
  return std::fabs(x - f) <= rel * std::max(1.0, std::fabs(x));
}

// EWA projection of one Gaussian into one view (the per-Gaussian stage of the
// renderer).  Returns vis = false when culled.
template <class S>
Proj<S> project_one(const Scene& sc, const Scene* tg, int64_t i, const View<S>& vw, const Cfg& cf) {
  using std::exp; using std::sqrt;
  Proj<S> P;
  P.vis = false; P.img_amb = P.grad_amb = P.r_amb = P.bin_amb = false; P.clampbits = 0;
  P.r = 0; P.xlo = P.ylo = 0; P.xhi = P.yhi = -1;
  S mu[3], ls[3], q[4], ol;
  std::vector<S> shc;
  scene_param<S>(sc, i, tg, mu, ls, q, ol, shc);

  // camera-space centre t = R mu + tau
  S t[3];
  for (int r = 0; r < 3; ++r) t[r] = vw.R[3 * r] * mu[0] + vw.R[3 * r + 1] * mu[1] + vw.R[3 * r + 2] * mu[2] + vw.tau[r];
  if (std::fabs(val(t[2]) - cf.znear) <= cf.m_near * cf.znear) P.img_amb = P.bin_amb = true;
  if (!(val(t[2]) > cf.znear)) return P;

  // 3D covariance Sigma = Rq diag(e^{2s}) Rq^T
  S qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S qu[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
  S Rq[9];
  quat_to_rot(qu, Rq);
  S sc3[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
  S M[9];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * sc3[c];
  S Sig[9];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) {
    S a = S(0.0);
    for (int k = 0; k < 3; ++k) a += M[3 * r + k] * M[3 * c + k];
    Sig[3 * r + c] = a;
  }
  // camera-frame covariance R Sigma R^T
  S RS[9], Sc[9];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) {
    S a = S(0.0);
    for (int k = 0; k < 3; ++k) a += vw.R[3 * r + k] * Sig[3 * k + c];
    RS[3 * r + c] = a;
  }
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) {
    S a = S(0.0);
    for (int k = 0; k < 3; ++k) a += RS[3 * r + k] * vw.R[3 * c + k];
    Sc[3 * r + c] = a;
  }
  // perspective Jacobian at the (guarded) camera-space point
  S iz = S(1.0) / t[2];
  S u = t[0] * iz, w = t[1] * iz;
  if (cf.clamp_j) {
    double limx = 1.3 * 0.5 * vw.W / vw.fx, limy = 1.3 * 0.5 * vw.H / vw.fy;
    if (std::fabs(std::fabs(val(u)) - limx) <= cf.m_lim * limx) P.grad_amb = true;
    if (std::fabs(std::fabs(val(w)) - limy) <= cf.m_lim * limy) P.grad_amb = true;
    if (val(u) > limx) u = S(limx);
    if (val(u) < -limx) u = S(-limx);
    if (val(w) > limy) w = S(limy);
    if (val(w) < -limy) w = S(-limy);
  }
  S J[6] = {S(vw.fx) * iz, S(0.0), S(-vw.fx) * u * iz,
            S(0.0), S(vw.fy) * iz, S(-vw.fy) * w * iz};
  // 2D covariance J Sc J^T + 0.3 I
  S JS[6];
  for (int r = 0; r < 2; ++r) for (int c = 0; c < 3; ++c) {
    S a = S(0.0);
    for (int k = 0; k < 3; ++k) a += J[3 * r + k] * Sc[3 * k + c];
    JS[3 * r + c] = a;
  }
  S C2[4];
  for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) {
    S a = S(0.0);
    for (int k = 0; k < 3; ++k) a += JS[3 * r + k] * J[3 * c + k];
    C2[2 * r + c] = a;
  }
  S a = C2[0] + S(0.3), b = C2[1], c = C2[3] + S(0.3);
  S det = a * c - b * b;
  if (!(val(det) > 0.0)) return P;
  P.A = c / det; P.B = -b / det; P.C = a / det;
  P.mx = S(vw.fx) * t[0] * iz + S(vw.cx);
  P.my = S(vw.fy) * t[1] * iz + S(vw.cy);
  P.depth = t[2];
  // support radius from the largest eigenvalue
  double av = val(a), bv = val(b), cv = val(c);
  double lam = 0.5 * (av + cv) + std::sqrt(std::max(0.0, 0.25 * (av - cv) * (av - cv) + bv * bv));
  double rr = 3.0 * std::sqrt(lam);
  if (near_int(rr, cf.m_r)) P.r_amb = true;
  P.r = std::ceil(rr);
  if (P.r <= 0.0) return P;
  P.opa = S(1.0) / (S(1.0) + exp(-ol));
  // tile rect: alpha can reach 1/255 only where A dx^2 + 2B dx dy + C dy^2
  // <= k = 2 ln(255 opacity), an ellipse whose bounding box has half-widths
  // sqrt(k a), sqrt(k c) (a, c: diagonal of the dilated 2D covariance);
  // widened by 0.1% + 0.05 px, capped by the support box r
  double kk = 2.0 * std::log(255.0 * val(P.opa));
  if (std::fabs(kk) <= 1e-4) P.bin_amb = true;
  if (!(kk > 0.0)) return P;
  double hx = std::min(P.r, std::sqrt(kk * av) * 1.001 + 0.05);
  double hy = std::min(P.r, std::sqrt(kk * cv) * 1.001 + 0.05);
  double mxv = val(P.mx), myv = val(P.my);
  double fxl = (mxv - hx) / cf.tw, fxh = (mxv + hx) / cf.tw;
  double fyl = (myv - hy) / cf.th, fyh = (myv + hy) / cf.th;
  P.xlo = std::max(0, (int)std::floor(fxl));
  P.xhi = std::min(vw.TX - 1, (int)std::floor(fxh));
  P.ylo = std::max(0, (int)std::floor(fyl));
  P.yhi = std::min(vw.TY - 1, (int)std::floor(fyh));
  // a tile boundary within margin of a rect edge makes the rect FP32-ambiguous
  double mt = cf.m_px / std::min(cf.tw, cf.th);
  if (near_int(fxl, mt) || near_int(fxh, mt) || near_int(fyl, mt) || near_int(fyh, mt) || P.r_amb)
    P.bin_amb = true;
  if (P.xlo > P.xhi || P.ylo > P.yhi) return P;

  // view direction from the camera centre o_c = -R^T tau
  S oc[3];
  for (int k = 0; k < 3; ++k) oc[k] = -(vw.R[k] * vw.tau[0] + vw.R[3 + k] * vw.tau[1] + vw.R[6 + k] * vw.tau[2]);
  S dv[3] = {mu[0] - oc[0], mu[1] - oc[1], mu[2] - oc[2]};
  S dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  S Y[16];
  sh_eval<S>(sc.deg, dv[0] / dn, dv[1] / dn, dv[2] / dn, Y);
  for (int ch = 0; ch < 3; ++ch) {
    S acc = S(0.5);
    for (int k = 0; k < sc.nc; ++k) acc += shc[ch * sc.nc + k] * Y[k];
    if (std::fabs(val(acc)) <= cf.m_sh) P.grad_amb = true;
    if (val(acc) < 0.0) { acc = S(0.0); P.clampbits |= 1 << ch; }
    P.rgb[ch] = acc;
  }
  P.vis = true;
  return P;
}

// ----------------------------------------------------------------------------
// Binning: every visible (view, Gaussian) emits one entry per tile of its rect,
// in Gaussian-id order and row-major within the rect; key = (global tile << 32)
// | depth bits.  A stable sort on the key leaves equal keys in id order.
// ----------------------------------------------------------------------------
struct Entry { uint64_t key; uint32_t val; };

int64_t bin_entries(int V, int64_t N, const uint32_t* depth_bits, const int32_t* rect,
                    const int32_t* tiles, std::vector<Entry>& out, std::vector<int64_t>& tile_base) {
  tile_base.assign(V + 1, 0);
  for (int v = 0; v < V; ++v) tile_base[v + 1] = tile_base[v] + (int64_t)tiles[2 * v] * tiles[2 * v + 1];
  out.clear();
  for (int v = 0; v < V; ++v) {
    int TX = tiles[2 * v];
    for (int64_t i = 0; i < N; ++i) {
      const int32_t* rc = rect + 4 * (v * N + i);
      if (rc[0] > rc[2] || rc[1] > rc[3]) continue;  // culled
      for (int ty = rc[1]; ty <= rc[3]; ++ty)
        for (int tx = rc[0]; tx <= rc[2]; ++tx) {
          uint64_t g = (uint64_t)(tile_base[v] + (int64_t)ty * TX + tx);
          out.push_back({(g << 32) | depth_bits[v * N + i], (uint32_t)i});
        }
    }
  }
  std::stable_sort(out.begin(), out.end(), [](const Entry& x, const Entry& y) { return x.key < y.key; });
  return (int64_t)out.size();
}

// ----------------------------------------------------------------------------
// Rendering
// ----------------------------------------------------------------------------
struct Blended {
  int64_t i;          // Gaussian id
  int64_t k;          // position in the tile's list
  double alpha, T;    // alpha_i and transmittance before it
  double e;           // exp(power)
  double dx, dy;      // m - p
  bool clamped;       // alpha hit the 0.99 clamp
};

template <class S>
struct ViewOut {
  S* image;        // [3][wh][ww] (the view's pixel window)
  S* alpha;        // [wh][ww]
  uint8_t* flags;  // [wh][ww] or null
};

// One view: project, bin (by FP64 depth), composite.
// `on_pixel(tile, list length, pix, blended list, T_final)` is called after
// each pixel when `record` is set (the backward consumes the list at once, so
// memory stays O(list length)).
//
// Threads (OpenMP): the projection runs over Gaussians and the composite over
// tiles; every pixel belongs to one tile and every (view, Gaussian) record to
// one iteration, so outputs do not depend on the thread count.  on_pixel is
// called by the thread that owns the tile (the caller keeps per-tile state).
// tiles_out (optional) receives every tile's list, in blend order.
struct NoPixel {
  void operator()(size_t, size_t, size_t, const std::vector<Blended>&, double) const {}
};

template <class S, class F>
void render_view(const Scene& sc, const Scene* tg, const View<S>& vw, const Cfg& cf,
                 std::vector<Proj<S>>& proj, ViewOut<S> out, bool record, F&& on_pixel,
                 std::vector<std::vector<int64_t>>* tiles_out = nullptr) {
  const int64_t N = sc.n;
  proj.resize(N);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < N; ++i) proj[i] = project_one<S>(sc, tg, i, vw, cf);

  // per-tile lists ordered by (depth, id)
  std::vector<int64_t> order;
  for (int64_t i = 0; i < N; ++i) if (proj[i].vis) order.push_back(i);
  // Blend order: depth rounded to single precision (the precision of the sort
  // key), equal keys in Gaussian-id order.
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return (float)val(proj[x].depth) < (float)val(proj[y].depth);
  });
  std::vector<std::vector<int64_t>> tiles((size_t)vw.TX * vw.TY);
  for (int64_t i : order) {
    const Proj<S>& p = proj[i];
    for (int ty = p.ylo; ty <= p.yhi; ++ty)
      for (int tx = p.xlo; tx <= p.xhi; ++tx) tiles[(size_t)ty * vw.TX + tx].push_back(i);
  }
  const double a_min = 1.0 / 255.0, t_min = 1e-4;

  const int wx1 = vw.wx0 + vw.ww, wy1 = vw.wy0 + vw.wh;
  const int64_t n_tiles = (int64_t)vw.TX * vw.TY;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < n_tiles; ++t) {
      const int ty = (int)(t / vw.TX), tx = (int)(t % vw.TX);
      std::vector<Blended> bl;
      const std::vector<int64_t>& lst = tiles[(size_t)t];
      for (int py = std::max(vw.wy0, ty * cf.th); py < std::min(wy1, (ty + 1) * cf.th); ++py)
        for (int px = std::max(vw.wx0, tx * cf.tw); px < std::min(wx1, (tx + 1) * cf.tw); ++px) {
          const double pcx = px + 0.5, pcy = py + 0.5;
          S T = S(1.0);
          S Cc[3] = {S(0.0), S(0.0), S(0.0)};
          uint8_t fl = 0;
          double last_depth = -1.0;
          bl.clear();
          for (size_t li = 0; li < lst.size(); ++li) {
            const int64_t i = lst[li];
            const Proj<S>& p = proj[i];
            double mxv = val(p.mx), myv = val(p.my);
            // signed distance of the pixel centre to the support box edge
            double e = std::min(std::min(pcx - (mxv - p.r), (mxv + p.r) - pcx),
                                std::min(pcy - (myv - p.r), (myv + p.r) - pcy));
            S dx = p.mx - S(pcx), dy = p.my - S(pcy);
            S power = S(-0.5) * (p.A * dx * dx + p.C * dy * dy) - p.B * dx * dy;
            double araw = val(p.opa) * std::exp(val(power));
            bool matters = std::min(0.99, araw) >= a_min * (1.0 - cf.m_rel);
            double edge_m = p.r_amb ? 1.0 + cf.m_px : cf.m_px;
            if (matters && std::fabs(e) <= edge_m) fl |= 1;
            if (matters && p.img_amb) fl |= 1;
            if (e < 0.0) continue;
            if (val(power) > 0.0) continue;
            using std::exp;
            S ex = exp(power);
            S al = p.opa * ex;
            bool clamped = false;
            if (std::fabs(val(al) - 0.99) <= cf.m_rel * 0.99) fl |= 2;
            if (val(al) > 0.99) { al = S(0.99); clamped = true; }
            if (std::fabs(val(al) - a_min) <= cf.m_rel * a_min) fl |= 1;
            if (val(al) < a_min) continue;
            S Tn = T * (S(1.0) - al);
            if (std::fabs(val(Tn) - t_min) <= cf.m_rel * t_min) fl |= 1;
            if (val(Tn) < t_min) break;
            if (p.grad_amb) fl |= 2;
            if (last_depth >= 0.0 && val(p.depth) - last_depth <= cf.m_depth * val(p.depth)) fl |= 1;
            last_depth = val(p.depth);
            for (int ch = 0; ch < 3; ++ch) Cc[ch] += p.rgb[ch] * al * T;
            if (record) bl.push_back({i, (int64_t)li, val(al), val(T), val(ex), val(dx), val(dy), clamped});
            T = Tn;
          }
          const size_t pix = (size_t)(py - vw.wy0) * vw.ww + (px - vw.wx0);
          for (int ch = 0; ch < 3; ++ch) out.image[(size_t)ch * vw.ww * vw.wh + pix] = Cc[ch] + T * S(cf.bg[ch]);
          if (out.alpha) out.alpha[pix] = S(1.0) - T;
          if (out.flags) out.flags[pix] = fl;
          if (record) on_pixel((size_t)t, lst.size(), pix, bl, val(T));
        }
  }
  if (tiles_out) tiles_out->swap(tiles);
}

// Views from [V][12] poses, [V][4] intrinsics, [V][2] sizes and optional
// [V][4] pixel windows (x0, y0, w, h).
void load_views(int V, const double* poses, const double* intr, const int32_t* wh,
                const int32_t* win, const Cfg& cf, std::vector<View<double>>& views) {
  views.resize(V);
  for (int v = 0; v < V; ++v) {
    View<double>& w = views[v];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) w.R[3 * r + c] = poses[12 * v + 4 * r + c];
      w.tau[r] = poses[12 * v + 4 * r + 3];
    }
    w.fx = intr[4 * v]; w.fy = intr[4 * v + 1]; w.cx = intr[4 * v + 2]; w.cy = intr[4 * v + 3];
    w.W = wh[2 * v]; w.H = wh[2 * v + 1];
    w.TX = (w.W + cf.tw - 1) / cf.tw; w.TY = (w.H + cf.th - 1) / cf.th;
    if (win) {
      w.wx0 = win[4 * v]; w.wy0 = win[4 * v + 1]; w.ww = win[4 * v + 2]; w.wh = win[4 * v + 3];
    } else {
      w.wx0 = 0; w.wy0 = 0; w.ww = w.W; w.wh = w.H;
    }
  }
}

// Dual views: the pose moves along T(eps) = Exp(eps xi) T, xi = (v, omega) given
// per view in `tposes` [V][6].  To first order R(eps) = R + eps [omega]x R and
// tau(eps) = tau + eps ([omega]x tau + v), which is exact for dual numbers.
void load_dual_views(int V, const double* poses, const double* tposes, const double* intr,
                     const int32_t* wh, const int32_t* win, const Cfg& cf,
                     std::vector<View<Dual>>& views) {
  std::vector<View<double>> base;
  load_views(V, poses, intr, wh, win, cf, base);
  views.resize(V);
  for (int v = 0; v < V; ++v) {
    const double* xi = tposes + 6 * v;
    const double* om = xi + 3;
    double W[9] = {0, -om[2], om[1], om[2], 0, -om[0], -om[1], om[0], 0};
    View<Dual>& w = views[v];
    const View<double>& b = base[v];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) {
        double d = 0;
        for (int k = 0; k < 3; ++k) d += W[3 * r + k] * b.R[3 * k + c];
        w.R[3 * r + c] = Dual(b.R[3 * r + c], d);
      }
      double d = xi[r];
      for (int k = 0; k < 3; ++k) d += W[3 * r + k] * b.tau[k];
      w.tau[r] = Dual(b.tau[r], d);
    }
    w.fx = b.fx; w.fy = b.fy; w.cx = b.cx; w.cy = b.cy; w.W = b.W; w.H = b.H; w.TX = b.TX; w.TY = b.TY;
    w.wx0 = b.wx0; w.wy0 = b.wy0; w.ww = b.ww; w.wh = b.wh;
  }
}

Cfg make_cfg(double znear, int tw, int th, const double* bg, int clamp_j, const double* margins) {
  Cfg c;
  c.znear = znear; c.tw = tw; c.th = th; c.clamp_j = clamp_j;
  for (int k = 0; k < 3; ++k) c.bg[k] = bg ? bg[k] : 0.0;
  // default margins: generous against single-precision rounding of each decision
  // [support edge (px), alpha/transmittance thresholds (relative), 3 sqrt(lambda)
  //  near an integer (relative), near plane (relative), Jacobian guard
  //  (relative),
  //  SH colour clamp (absolute), depth gap between consecutive blended splats
  //  (relative; 0 = off: both sides order by the same single-precision key)]
  double d[7] = {5e-4, 3e-4, 1e-5, 1e-9, 1e-5, 1e-5, 0.0};
  if (margins) for (int k = 0; k < 7; ++k) d[k] = margins[k];
  c.m_px = d[0]; c.m_rel = d[1]; c.m_r = d[2]; c.m_near = d[3]; c.m_lim = d[4]; c.m_sh = d[5];
  c.m_depth = d[6];
  return c;
}

Scene make_scene(int64_t N, int deg, const double* means, const double* lsc, const double* quat,
                 const double* opl, const double* sh) {
  Scene s;
  s.n = N; s.deg = deg; s.nc = (deg + 1) * (deg + 1);
  s.means = means; s.lsc = lsc; s.quat = quat; s.opl = opl; s.sh = sh;
  return s;
}

// ----------------------------------------------------------------------------
// Analytic backward (hand-derived chain rule, matrix form), FP64.
// ----------------------------------------------------------------------------
void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
  for (int r = 0; r < n; ++r) for (int c = 0; c < m; ++c) {
    double a = 0; for (int j = 0; j < k; ++j) a += A[r * k + j] * B[j * m + c];
    C[r * m + c] = a;
  }
}
void transpose(const double* A, double* B, int n, int m) {
  for (int r = 0; r < n; ++r) for (int c = 0; c < m; ++c) B[c * n + r] = A[r * m + c];
}

struct Grad2D { double mx, my, A, B, C, opa, rgb[3]; };

// dL/d(parameters, pose) of one visible Gaussian in one view given the
// gradients of its 2D splat record.
void project_backward(const Scene& sc, int64_t i, const View<double>& vw, const Cfg& cf,
                      const Proj<double>& P, const Grad2D& g, double* gmeans, double* glsc,
                      double* gquat, double* gopl, double* gsh, double* gpose) {
  const double* mu = sc.means + 3 * i;
  const double* ls = sc.lsc + 3 * i;
  const double* q = sc.quat + 4 * i;
  const double ol = sc.opl[i];
  const double* shc = sc.sh + 3 * sc.nc * i;
  const double* R = vw.R;

  double t[3];
  for (int r = 0; r < 3; ++r) t[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + vw.tau[r];
  double dt[3] = {0, 0, 0};
  double dmu[3] = {0, 0, 0};
  double dvpose[3] = {0, 0, 0}, dom[3] = {0, 0, 0};

  // ---- colour: rgb = max(0, sum c Y(d) + 1/2), d = (mu - o_c)/|mu - o_c|
  double oc[3];
  for (int k = 0; k < 3; ++k) oc[k] = -(R[k] * vw.tau[0] + R[3 + k] * vw.tau[1] + R[6 + k] * vw.tau[2]);
  double wv[3] = {mu[0] - oc[0], mu[1] - oc[1], mu[2] - oc[2]};
  double wn = std::sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
  double d[3] = {wv[0] / wn, wv[1] / wn, wv[2] / wn};
  double Y[16];
  sh_eval<double>(sc.deg, d[0], d[1], d[2], Y);
  double dY[16] = {0};
  for (int ch = 0; ch < 3; ++ch) {
    if (P.clampbits & (1 << ch)) continue;
    for (int k = 0; k < sc.nc; ++k) {
      gsh[ch * sc.nc + k] += g.rgb[ch] * Y[k];
      dY[k] += g.rgb[ch] * shc[ch * sc.nc + k];
    }
  }
  // gradient of the basis along each axis, from dual numbers
  double dd[3] = {0, 0, 0};
  for (int ax = 0; ax < 3; ++ax) {
    Dual x(d[0], ax == 0), y(d[1], ax == 1), z(d[2], ax == 2);
    Dual Yd[16];
    sh_eval<Dual>(sc.deg, x, y, z, Yd);
    for (int k = 0; k < sc.nc; ++k) dd[ax] += dY[k] * Yd[k].d;
  }
  // through the normalisation: dw = (I - d d^T) dd / |w|
  double dproj = d[0] * dd[0] + d[1] * dd[1] + d[2] * dd[2];
  double dw[3];
  for (int k = 0; k < 3; ++k) dw[k] = (dd[k] - d[k] * dproj) / wn;
  for (int k = 0; k < 3; ++k) dmu[k] += dw[k];
  // w = mu - o_c moves with the pose as w + R^T v (first order): dL/dv += R dw
  for (int r = 0; r < 3; ++r) dvpose[r] += R[3 * r] * dw[0] + R[3 * r + 1] * dw[1] + R[3 * r + 2] * dw[2];

  // ---- opacity
  double o = 1.0 / (1.0 + std::exp(-ol));
  gopl[0] += g.opa * o * (1.0 - o);

  // ---- mean in pixels
  double iz = 1.0 / t[2];
  dt[0] += g.mx * vw.fx * iz;
  dt[1] += g.my * vw.fy * iz;
  dt[2] += -g.mx * vw.fx * t[0] * iz * iz - g.my * vw.fy * t[1] * iz * iz;

  // ---- conic -> 2D covariance: Q = S2^{-1}, G_S2 = -Q G_Q Q
  double Q[4] = {P.A, P.B, P.B, P.C};
  double GQ[4] = {g.A, 0.5 * g.B, 0.5 * g.B, g.C};
  double tmp[4], GS2[4];
  matmul(Q, GQ, tmp, 2, 2, 2);
  matmul(tmp, Q, GS2, 2, 2, 2);
  for (int k = 0; k < 4; ++k) GS2[k] = -GS2[k];

  // ---- recompute Sigma, Sc, J
  double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double qu[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
  double Rq[9];
  quat_to_rot(qu, Rq);
  double s3[3] = {std::exp(ls[0]), std::exp(ls[1]), std::exp(ls[2])};
  double M[9];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s3[c];
  double Mt[9], Sig[9];
  transpose(M, Mt, 3, 3);
  matmul(M, Mt, Sig, 3, 3, 3);
  double Rt[9], RS[9], Sc[9];
  transpose(R, Rt, 3, 3);
  matmul(R, Sig, RS, 3, 3, 3);
  matmul(RS, Rt, Sc, 3, 3, 3);
  double u = t[0] * iz, w = t[1] * iz;
  bool cu = false, cw = false;
  if (cf.clamp_j) {
    double limx = 1.3 * 0.5 * vw.W / vw.fx, limy = 1.3 * 0.5 * vw.H / vw.fy;
    if (u > limx) { u = limx; cu = true; }
    if (u < -limx) { u = -limx; cu = true; }
    if (w > limy) { w = limy; cw = true; }
    if (w < -limy) { w = -limy; cw = true; }
  }
  double J[6] = {vw.fx * iz, 0, -vw.fx * u * iz, 0, vw.fy * iz, -vw.fy * w * iz};

  // S2 = J Sc J^T (+0.3 I): G_Sc = J^T G_S2 J ; G_J = 2 G_S2 J Sc
  double Jt[6], t23[6], GSc[9], GJ[6];
  transpose(J, Jt, 2, 3);
  matmul(GS2, J, t23, 2, 2, 3);
  matmul(Jt, t23, GSc, 3, 2, 3);
  double JSc[6];
  matmul(J, Sc, JSc, 2, 3, 3);
  matmul(GS2, JSc, GJ, 2, 2, 3);
  for (int k = 0; k < 6; ++k) GJ[k] *= 2.0;

  // J entries as functions of t
  dt[2] += GJ[0] * (-vw.fx * iz * iz) + GJ[4] * (-vw.fy * iz * iz);
  if (cu) {
    dt[2] += GJ[2] * (vw.fx * u * iz * iz);
  } else {
    dt[0] += GJ[2] * (-vw.fx * iz * iz);
    dt[2] += GJ[2] * (2.0 * vw.fx * t[0] * iz * iz * iz);
  }
  if (cw) {
    dt[2] += GJ[5] * (vw.fy * w * iz * iz);
  } else {
    dt[1] += GJ[5] * (-vw.fy * iz * iz);
    dt[2] += GJ[5] * (2.0 * vw.fy * t[1] * iz * iz * iz);
  }

  // Sc = R Sigma R^T: G_Sigma = R^T G_Sc R ; pose rotation term from Sc G_Sc
  double t33[9], GSig[9];
  matmul(Rt, GSc, t33, 3, 3, 3);
  matmul(t33, R, GSig, 3, 3, 3);
  double MM[9];
  matmul(Sc, GSc, MM, 3, 3, 3);
  dom[0] += 2.0 * (MM[5] - MM[7]);
  dom[1] += 2.0 * (MM[6] - MM[2]);
  dom[2] += 2.0 * (MM[1] - MM[3]);

  // Sigma = M M^T, M = Rq diag(s): G_M = 2 G_Sigma M
  double GM[9];
  matmul(GSig, M, GM, 3, 3, 3);
  for (int k = 0; k < 9; ++k) GM[k] *= 2.0;
  for (int c = 0; c < 3; ++c) {
    double gs = 0;
    for (int r = 0; r < 3; ++r) gs += Rq[3 * r + c] * GM[3 * r + c];
    glsc[c] += gs * s3[c];
  }
  double GR[9];
  for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) GR[3 * r + c] = GM[3 * r + c] * s3[c];
  // rotation entries as functions of the unit quaternion
  const double W_ = qu[0], X = qu[1], Yq = qu[2], Z = qu[3];
  const double dRw[9] = {0, -2 * Z, 2 * Yq, 2 * Z, 0, -2 * X, -2 * Yq, 2 * X, 0};
  const double dRx[9] = {0, 2 * Yq, 2 * Z, 2 * Yq, -4 * X, -2 * W_, 2 * Z, 2 * W_, -4 * X};
  const double dRy[9] = {-4 * Yq, 2 * X, 2 * W_, 2 * X, 0, 2 * Z, -2 * W_, 2 * Z, -4 * Yq};
  const double dRz[9] = {-4 * Z, -2 * W_, 2 * X, 2 * W_, -4 * Z, 2 * Yq, 2 * X, 2 * Yq, 0};
  double dqu[4] = {0, 0, 0, 0};
  for (int k = 0; k < 9; ++k) {
    dqu[0] += GR[k] * dRw[k]; dqu[1] += GR[k] * dRx[k];
    dqu[2] += GR[k] * dRy[k]; dqu[3] += GR[k] * dRz[k];
  }
  double pr = qu[0] * dqu[0] + qu[1] * dqu[1] + qu[2] * dqu[2] + qu[3] * dqu[3];
  for (int k = 0; k < 4; ++k) gquat[k] += (dqu[k] - qu[k] * pr) / qn;

  // t = R mu + tau
  for (int c = 0; c < 3; ++c) dmu[c] += R[c] * dt[0] + R[3 + c] * dt[1] + R[6 + c] * dt[2];
  for (int k = 0; k < 3; ++k) gmeans[k] += dmu[k];
  // pose, left perturbation: t -> t + omega x t + v
  for (int k = 0; k < 3; ++k) dvpose[k] += dt[k];
  dom[0] += t[1] * dt[2] - t[2] * dt[1];
  dom[1] += t[2] * dt[0] - t[0] * dt[2];
  dom[2] += t[0] * dt[1] - t[1] * dt[0];
  for (int k = 0; k < 3; ++k) { gpose[k] += dvpose[k]; gpose[3 + k] += dom[k]; }
}

// SE(3) exponential of xi = (v, omega): rotation by Rodrigues, translation V v.
void se3_exp(const double* xi, double* Re, double* te) {
  const double* v = xi;
  const double* w = xi + 3;
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = std::sqrt(th2);
  double A, B, Cc;
  if (th < 1e-5) {
    A = 1.0 - th2 / 6.0; B = 0.5 - th2 / 24.0; Cc = 1.0 / 6.0 - th2 / 120.0;
  } else {
    A = std::sin(th) / th; B = (1.0 - std::cos(th)) / th2; Cc = (th - std::sin(th)) / (th2 * th);
  }
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  matmul(K, K, K2, 3, 3, 3);
  double Vm[9];
  for (int k = 0; k < 9; ++k) {
    double I = (k % 4 == 0) ? 1.0 : 0.0;
    Re[k] = I + A * K[k] + B * K2[k];
    Vm[k] = I + B * K[k] + Cc * K2[k];
  }
  for (int r = 0; r < 3; ++r) te[r] = Vm[3 * r] * v[0] + Vm[3 * r + 1] * v[1] + Vm[3 * r + 2] * v[2];
}

}  // namespace

// ============================================================================
// C entry points (ctypes)
// ============================================================================
extern "C" {

// Real SH basis Y_k(dir), k = l^2 + l + m, for n unit directions [n][3].
int orc_sh_basis(int deg, int64_t n, const double* dirs, double* out) {
  if (deg < 0 || deg > 3) return 1;
  int nc = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    double Y[16];
    sh_eval<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < nc; ++k) out[nc * i + k] = Y[k];
  }
  return 0;
}

// Projected records per (view, Gaussian), stride 20 doubles:
//  0 vis, 1 mx, 2 my, 3 A, 4 B, 5 C, 6 opacity, 7-9 rgb, 10 depth, 11 radius,
//  12-15 rect (xlo, ylo, xhi, yhi), 16 clamp bits, 17 img_amb, 18 grad_amb,
//  19 bin_amb
enum { PROJ_STRIDE = 20 };

static void write_proj(const Proj<double>& p, double* o) {
  o[0] = p.vis; o[1] = p.vis ? p.mx : 0; o[2] = p.vis ? p.my : 0;
  o[3] = p.vis ? p.A : 0; o[4] = p.vis ? p.B : 0; o[5] = p.vis ? p.C : 0;
  o[6] = p.vis ? p.opa : 0;
  for (int k = 0; k < 3; ++k) o[7 + k] = p.vis ? p.rgb[k] : 0;
  o[10] = p.vis ? p.depth : 0; o[11] = p.r;
  o[12] = p.xlo; o[13] = p.ylo; o[14] = p.xhi; o[15] = p.yhi;
  o[16] = p.clampbits; o[17] = p.img_amb; o[18] = p.grad_amb; o[19] = p.bin_amb;
}

// Forward render of V views.  windows (optional): [V][4] pixel windows
// (x0, y0, w, h) to composite; the projection and binning always cover the
// whole view.  image: windows concatenated, each [3][h][w]; alpha: each [h][w];
// flags (optional): each [h][w], bit 0 = the image value at
// this pixel hangs on a decision within margin, bit 1 = its derivative does.
// proj (optional): [V][N][PROJ_STRIDE].
int orc_render(int64_t N, int deg, const double* means, const double* lsc, const double* quat,
               const double* opl, const double* sh, int V, const double* poses, const double* intr,
               const int32_t* wh, const int32_t* windows, double znear, int tw, int th,
               const double* bg, int clamp_j, const double* margins, double* image, double* alpha,
               uint8_t* flags, double* proj) {
  if (N < 0 || deg < 0 || deg > 3 || V <= 0 || tw <= 0 || th <= 0) return 1;
  Scene sc = make_scene(N, deg, means, lsc, quat, opl, sh);
  Cfg cf = make_cfg(znear, tw, th, bg, clamp_j, margins);
  std::vector<View<double>> views;
  load_views(V, poses, intr, wh, windows, cf, views);
  size_t off_img = 0, off_px = 0;
  std::vector<Proj<double>> pj;
  for (int v = 0; v < V; ++v) {
    ViewOut<double> o{image + off_img, alpha ? alpha + off_px : nullptr, flags ? flags + off_px : nullptr};
    render_view<double>(sc, nullptr, views[v], cf, pj, o, false, NoPixel());
    if (proj) for (int64_t i = 0; i < N; ++i) write_proj(pj[i], proj + PROJ_STRIDE * (v * N + i));
    off_img += (size_t)3 * views[v].ww * views[v].wh;
    off_px += (size_t)views[v].ww * views[v].wh;
  }
  return 0;
}

// Forward render on dual numbers: the parameters move along the tangent
// (t_means, ...) and each pose along Exp(eps xi_v) T_v with xi_v = t_pose[v]
// (v, omega).  Writes the image value and its exact directional derivative.
int orc_render_dual(int64_t N, int deg, const double* means, const double* lsc, const double* quat,
                    const double* opl, const double* sh, const double* t_means, const double* t_lsc,
                    const double* t_quat, const double* t_opl, const double* t_sh, int V,
                    const double* poses, const double* t_pose, const double* intr, const int32_t* wh,
                    const int32_t* windows, double znear, int tw, int th, const double* bg,
                    int clamp_j, double* image, double* image_tan, double* alpha_tan) {
  if (N < 0 || deg < 0 || deg > 3 || V <= 0) return 1;
  Scene sc = make_scene(N, deg, means, lsc, quat, opl, sh);
  Scene tg = make_scene(N, deg, t_means, t_lsc, t_quat, t_opl, t_sh);
  Cfg cf = make_cfg(znear, tw, th, bg, clamp_j, nullptr);
  std::vector<View<Dual>> views;
  load_dual_views(V, poses, t_pose, intr, wh, windows, cf, views);
  size_t off_img = 0, off_px = 0;
  std::vector<Proj<Dual>> pj;
  for (int v = 0; v < V; ++v) {
    size_t np = (size_t)views[v].ww * views[v].wh;
    std::vector<Dual> img(3 * np), al(np);
    ViewOut<Dual> o{img.data(), al.data(), nullptr};
    render_view<Dual>(sc, &tg, views[v], cf, pj, o, false, NoPixel());
    for (size_t k = 0; k < 3 * np; ++k) { image[off_img + k] = img[k].v; image_tan[off_img + k] = img[k].d; }
    if (alpha_tan) for (size_t k = 0; k < np; ++k) alpha_tan[off_px + k] = al[k].d;
    off_img += 3 * np;
    off_px += np;
  }
  return 0;
}

// Analytic backward: given dL/dimage (same layout as image) and optionally
// dL/dalpha, accumulate dL/dparams (natural layouts) and dL/dpose [V][6]
// (v, omega).  With windows, dL/dimage covers the windows only (the loss
// gradient is zero elsewhere).  Gradient arrays are overwritten.
int orc_backward(int64_t N, int deg, const double* means, const double* lsc, const double* quat,
                 const double* opl, const double* sh, int V, const double* poses, const double* intr,
                 const int32_t* wh, const int32_t* windows, double znear, int tw, int th,
                 const double* bg, int clamp_j, const double* dimage, const double* dalpha,
                 double* gmeans, double* glsc,
                 double* gquat, double* gopl, double* gsh, double* gpose) {
  if (N < 0 || deg < 0 || deg > 3 || V <= 0) return 1;
  Scene sc = make_scene(N, deg, means, lsc, quat, opl, sh);
  Cfg cf = make_cfg(znear, tw, th, bg, clamp_j, nullptr);
  std::vector<View<double>> views;
  load_views(V, poses, intr, wh, windows, cf, views);
  const int nc = sc.nc;
  std::memset(gmeans, 0, sizeof(double) * 3 * N);
  std::memset(glsc, 0, sizeof(double) * 3 * N);
  std::memset(gquat, 0, sizeof(double) * 4 * N);
  std::memset(gopl, 0, sizeof(double) * N);
  std::memset(gsh, 0, sizeof(double) * 3 * nc * N);
  std::memset(gpose, 0, sizeof(double) * 6 * V);
  size_t off_img = 0, off_px = 0;
  std::vector<Proj<double>> pj;
  for (int v = 0; v < V; ++v) {
    const View<double>& vw = views[v];
    size_t np = (size_t)vw.ww * vw.wh;
    std::vector<double> img(3 * np), al(np);
    ViewOut<double> o{img.data(), al.data(), nullptr};
    // Per-pixel contributions are summed per tile first (pixels of the tile in
    // row-major order, each walked back to front), into part[tile][list
    // position]; the tiles are then added in tile order.  The order of every
    // sum is fixed by the tile lists alone, so any number of threads gives the
    // same bits.
    std::vector<std::vector<Grad2D>> part((size_t)vw.TX * vw.TY);
    auto per_pixel = [&](size_t tile, size_t list_len, size_t pix, const std::vector<Blended>& L, double Tfin) {
      std::vector<Grad2D>& P = part[tile];
      if (P.empty()) P.assign(list_len, Grad2D{0, 0, 0, 0, 0, 0, {0, 0, 0}});
      double gc[3];
      for (int ch = 0; ch < 3; ++ch) gc[ch] = dimage[off_img + ch * np + pix];
      double ga = dalpha ? dalpha[off_px + pix] : 0.0;
      // acc = colour contributed by everything behind splat k, background included
      double acc[3] = {Tfin * cf.bg[0], Tfin * cf.bg[1], Tfin * cf.bg[2]};
      for (int k = (int)L.size() - 1; k >= 0; --k) {
        const Blended& b = L[k];
        const Proj<double>& p = pj[b.i];
        Grad2D& G = P[(size_t)b.k];
        double dal = 0;
        for (int ch = 0; ch < 3; ++ch) {
          G.rgb[ch] += gc[ch] * b.alpha * b.T;
          // d/dalpha_k of  c_k alpha_k T_k + (later terms scale with 1/(1-alpha_k))
          dal += gc[ch] * (p.rgb[ch] * b.T - acc[ch] / (1.0 - b.alpha));
          acc[ch] += p.rgb[ch] * b.alpha * b.T;
        }
        dal += ga * Tfin / (1.0 - b.alpha);
        if (b.clamped) continue;
        // alpha = o e^power
        G.opa += dal * b.e;
        double dpow = dal * b.alpha;
        G.A += -0.5 * b.dx * b.dx * dpow;
        G.C += -0.5 * b.dy * b.dy * dpow;
        G.B += -b.dx * b.dy * dpow;
        // dx = mx - px
        G.mx += -(p.A * b.dx + p.B * b.dy) * dpow;
        G.my += -(p.C * b.dy + p.B * b.dx) * dpow;
      }
    };
    std::vector<std::vector<int64_t>> tiles;
    render_view<double>(sc, nullptr, vw, cf, pj, o, true, per_pixel, &tiles);
    std::vector<Grad2D> g2(N);
    std::memset(g2.data(), 0, sizeof(Grad2D) * N);
    for (size_t t = 0; t < tiles.size(); ++t) {
      const std::vector<Grad2D>& P = part[t];
      for (size_t k = 0; k < P.size(); ++k) {
        Grad2D& G = g2[tiles[t][k]];
        const Grad2D& q = P[k];
        G.mx += q.mx; G.my += q.my; G.A += q.A; G.B += q.B; G.C += q.C; G.opa += q.opa;
        for (int ch = 0; ch < 3; ++ch) G.rgb[ch] += q.rgb[ch];
      }
    }
    part.clear();
    // chain rule per Gaussian (independent), pose terms summed in Gaussian order
    std::vector<double> gp((size_t)6 * N, 0.0);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < N; ++i) {
      if (!pj[i].vis) continue;
      project_backward(sc, i, vw, cf, pj[i], g2[i], gmeans + 3 * i, glsc + 3 * i, gquat + 4 * i,
                       gopl + i, gsh + 3 * nc * i, gp.data() + 6 * i);
    }
    for (int64_t i = 0; i < N; ++i) {
      if (!pj[i].vis) continue;
      for (int k = 0; k < 6; ++k) gpose[6 * v + k] += gp[6 * i + k];
    }
    off_img += 3 * np;
    off_px += np;
  }
  return 0;
}

// Binning of given records: depth_bits [V*N] (IEEE single bits of positive
// depths), rect [V*N][4] (xlo, ylo, xhi, yhi; xlo > xhi marks culled), tiles
// [V][2] (TX, TY).  Writes sorted keys/vals (capacity cap) and ranges
// [sum TX*TY][2] ([start, end) per global tile).  Returns K, or -1 when K > cap.
int64_t orc_bin(int V, int64_t N, const uint32_t* depth_bits, const int32_t* rect,
                const int32_t* tiles, int64_t cap, uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
  std::vector<Entry> e;
  std::vector<int64_t> tb;
  int64_t K = bin_entries(V, N, depth_bits, rect, tiles, e, tb);
  if (K > cap) return -1;
  for (int64_t k = 0; k < K; ++k) { keys[k] = e[k].key; vals[k] = e[k].val; }
  int64_t G = tb[V];
  for (int64_t g = 0; g < G; ++g) { ranges[2 * g] = 0; ranges[2 * g + 1] = 0; }
  for (int64_t k = 0; k < K; ++k) {
    uint64_t g = e[k].key >> 32;
    if (k == 0 || (e[k - 1].key >> 32) != g) ranges[2 * g] = (uint32_t)k;
    if (k == K - 1 || (e[k + 1].key >> 32) != g) ranges[2 * g + 1] = (uint32_t)(k + 1);
  }
  return K;
}

// Adam with bias correction, in place, n elements; lr per element.
//   m = b1 m + (1-b1) g ; v = b2 v + (1-b2) g^2
//   p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
int orc_adam(int64_t n, double* p, const double* g, double* m, double* v, const double* lr,
             double b1, double b2, double eps, int step) {
  if (step < 1) return 1;
  double bc1 = 1.0 - std::pow(b1, step), bc2 = 1.0 - std::pow(b2, step);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    double mh = m[k] / bc1, vh = v[k] / bc2;
    p[k] -= lr[k] * mh / (std::sqrt(vh) + eps);
  }
  return 0;
}

// Pose step: Adam on xi (v, omega) with zero-based tangent, then T <- Exp(xi) T.
// poses [V][12] (R row-major 3x4 with tau in column 3), gpose/m/v [V][6].
int orc_pose_adam(int V, double* poses, const double* gpose, double* m, double* v, double lr,
                  double b1, double b2, double eps, int step) {
  if (step < 1) return 1;
  double bc1 = 1.0 - std::pow(b1, step), bc2 = 1.0 - std::pow(b2, step);
  for (int iv = 0; iv < V; ++iv) {
    double xi[6];
    for (int k = 0; k < 6; ++k) {
      int j = 6 * iv + k;
      m[j] = b1 * m[j] + (1.0 - b1) * gpose[j];
      v[j] = b2 * v[j] + (1.0 - b2) * gpose[j] * gpose[j];
      xi[k] = -lr * (m[j] / bc1) / (std::sqrt(v[j] / bc2) + eps);
    }
    double Re[9], te[3];
    se3_exp(xi, Re, te);
    double* P = poses + 12 * iv;
    double R0[9], t0[3];
    for (int r = 0; r < 3; ++r) { for (int c = 0; c < 3; ++c) R0[3 * r + c] = P[4 * r + c]; t0[r] = P[4 * r + 3]; }
    double Rn[9];
    matmul(Re, R0, Rn, 3, 3, 3);
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) P[4 * r + c] = Rn[3 * r + c];
      P[4 * r + 3] = Re[3 * r] * t0[0] + Re[3 * r + 1] * t0[1] + Re[3 * r + 2] * t0[2] + te[r];
    }
  }
  return 0;
}

// Threads used by the oracle's parallel loops (OpenMP; 1 = serial).  Results
// do not depend on it.  orc_get_threads returns the current setting (1 when
// built without OpenMP).
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// SE(3) exponential, for tests: xi [6] -> R [9], t [3].
int orc_se3_exp(const double* xi, double* R, double* t) { se3_exp(xi, R, t); return 0; }

}  // extern "C"
