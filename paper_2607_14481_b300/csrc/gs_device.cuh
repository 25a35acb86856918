// Device-side building blocks shared by the rasterizer kernels:
// double-single arithmetic for the screen-space mean, the per-launch view
// table, real SH of degree <= 3 with their gradients, and quaternion rotation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = GS_TILE;                  // default tile: 16x16 pixels
constexpr int kTilePixels = kTile * kTile;      // pixels of every supported tile shape (16x16, 32x8, 8x32)
constexpr float kAlphaMax = 0.99f;              // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;      // skip threshold
constexpr float kTransMin = 1e-4f;              // early-stop threshold
constexpr float kDilation = 0.3f;               // px^2 added to the 2D covariance
constexpr float kGuard = 1.3f;                  // Jacobian frustum guard factor

// ---------------------------------------------------------------------------
// Per-launch view table, passed by value as a kernel parameter.
// ---------------------------------------------------------------------------
struct ViewInfo {
  float fx, fy, cx, cy;
  int32_t W, H, TX, TY;
  int32_t tile_base;     // first global tile of this view
  int32_t pad;
  int64_t pix_base;      // first pixel of this view in concatenated per-pixel buffers
};

struct ViewTable {
  ViewInfo v[GS_MAX_VIEWS];
  int32_t views;
  int32_t total_tiles;
  int32_t tw, th;        // tile shape in pixels (TX = ceil(W / tw), TY = ceil(H / th))
};

// Supported tile shapes: 256 pixels, width 8, 16 or 32.
inline bool tile_shape_ok(int tw, int th) {
  return (tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 8 && th == 32);
}

// View owning global tile gt (binary search over tile_base).
// First statement of a kernel in a chain of programmatic dependent launches
// (launch_dependent): waits until the grid before it on the stream has
// completed and its writes are visible (a no-op for a kernel launched the
// ordinary way), then lets the next kernel of the chain be scheduled as this
// grid's blocks retire; that kernel's own chain_enter holds it until this
// grid has completed, so no read moves ahead of a write it depends on.
__device__ __forceinline__ void chain_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Hint that the line holding p will be read soon by this SM (no register,
// no wait; p must point into an allocation).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int gt) {
  int lo = 0, hi = vt.views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Double-single ("df") arithmetic: value = hi + lo with |lo| <= ulp(hi)/2,
// built from the error-free transformations TwoSum (Knuth) and TwoProduct via
// fused multiply-add (Dekker's product with an FMA).  Used for the camera-space
// point and the pixel-space mean, whose single-precision rounding would
// otherwise move splats by ~5e-5 px at 720p-1080p.
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  // r = a - q1 b, exactly enough for a second quotient digit
  df p = df_mul_f(b, q1);
  df r = df_add(a, df{-p.hi, -p.lo});
  float q2 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2);
}
// a0 b0 + a1 b1 + a2 b2 + c with single-precision operands
__device__ __forceinline__ df df_dot3_add(float a0, float b0, float a1, float b1, float a2,
                                          float b2, float c) {
  df s = df_two_prod(a0, b0);
  s = df_add(s, df_two_prod(a1, b1));
  s = df_add(s, df_two_prod(a2, b2));
  return df_add_f(s, c);
}
// value <= x ?
__device__ __forceinline__ bool df_le(df a, float x) {
  return a.hi < x || (a.hi == x && a.lo <= 0.0f);
}

// ---------------------------------------------------------------------------
// Real spherical harmonics up to l = 3 (orthonormal, no Condon-Shortley
// phase, index k = l^2 + l + m) at a unit direction (x, y, z):
//   l=0: 1/(2 sqrt pi)
//   l=1: sqrt(3/(4 pi)) (y, z, x)
//   l=2: 1/2 sqrt(15/pi) (xy, yz), 1/4 sqrt(5/pi) (3z^2-1), 1/2 sqrt(15/pi) xz,
//        1/4 sqrt(15/pi) (x^2-y^2)
//   l=3: 1/4 sqrt(35/(2pi)) y(3x^2-y^2), 1/2 sqrt(105/pi) xyz,
//        1/4 sqrt(21/(2pi)) y(5z^2-1), 1/4 sqrt(7/pi) z(5z^2-3),
//        1/4 sqrt(21/(2pi)) x(5z^2-1), 1/4 sqrt(105/pi) z(x^2-y^2),
//        1/4 sqrt(35/(2pi)) x(x^2-3y^2)
// Decimal values of the normalisations written out from those closed forms.
// ---------------------------------------------------------------------------
constexpr float kY00 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3e = 1.445305721320277f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = kY00;
  if (DEG >= 1) {
    Y[1] = kC1 * y; Y[2] = kC1 * z; Y[3] = kC1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = kC2a * y * z;
    Y[6] = kC2b * (3.0f * zz - 1.0f);
    Y[7] = kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = kC3a * y * (3.0f * xx - yy);
      Y[10] = kC3b * x * y * z;
      Y[11] = kC3c * y * (5.0f * zz - 1.0f);
      Y[12] = kC3d * z * (5.0f * zz - 3.0f);
      Y[13] = kC3c * x * (5.0f * zz - 1.0f);
      Y[14] = kC3e * z * (xx - yy);
      Y[15] = kC3a * x * (xx - 3.0f * yy);
    }
  }
}

// g . grad_xyz Y for the polynomial forms above (the radial part is removed
// by the caller's projection onto the sphere's tangent plane).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float* g,
                                              float& dx, float& dy, float& dz) {
  dx = 0.0f; dy = 0.0f; dz = 0.0f;
  if (DEG >= 1) {
    dy += kC1 * g[1]; dz += kC1 * g[2]; dx += kC1 * g[3];
  }
  if (DEG >= 2) {
    dx += kC2a * (y * g[4] + z * g[7]) + 2.0f * kC2c * x * g[8];
    dy += kC2a * (x * g[4] + z * g[5]) - 2.0f * kC2c * y * g[8];
    dz += kC2a * (y * g[5] + x * g[7]) + 6.0f * kC2b * z * g[6];
    if (DEG >= 3) {
      float xx = x * x, yy = y * y, zz = z * z;
      dx += kC3a * 6.0f * x * y * g[9] + kC3b * y * z * g[10] + kC3c * (5.0f * zz - 1.0f) * g[13] +
            kC3e * 2.0f * x * z * g[14] + kC3a * 3.0f * (xx - yy) * g[15];
      dy += kC3a * 3.0f * (xx - yy) * g[9] + kC3b * x * z * g[10] + kC3c * (5.0f * zz - 1.0f) * g[11] -
            kC3e * 2.0f * y * z * g[14] - kC3a * 6.0f * x * y * g[15];
      dz += kC3b * x * y * g[10] + kC3c * 10.0f * y * z * g[11] + kC3d * (15.0f * zz - 3.0f) * g[12] +
            kC3c * 10.0f * x * z * g[13] + kC3e * (xx - yy) * g[14];
    }
  }
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* Rq) {
  Rq[0] = 1.0f - 2.0f * (y * y + z * z); Rq[1] = 2.0f * (x * y - w * z); Rq[2] = 2.0f * (x * z + w * y);
  Rq[3] = 2.0f * (x * y + w * z); Rq[4] = 1.0f - 2.0f * (x * x + z * z); Rq[5] = 2.0f * (y * z - w * x);
  Rq[6] = 2.0f * (x * z - w * y); Rq[7] = 2.0f * (y * z + w * x); Rq[8] = 1.0f - 2.0f * (x * x + y * y);
}

// ---------------------------------------------------------------------------
// The Adam update of one element (shared by the standalone step and the
// per-Gaussian backward with the update fused in, so both give the same bits)
// ---------------------------------------------------------------------------
// 1 - beta^step: beta^step by exponentiation by squaring in double (only
// multiplications, so host and device give the same bits), rounded once.
__host__ __device__ __forceinline__ float bias_corr(float beta, int step) {
  double r = 1.0, b = (double)beta;
  for (unsigned e = (unsigned)step; e; e >>= 1) {
    if (e & 1u) r *= b;
    b *= b;
  }
  return (float)(1.0 - r);
}

// p -= lr * (m / bc1) / (sqrt(v / bc2) + eps), written as
// p -= (lr / bc1) * m / (sqrt(v) * rsqrt_bc2 + eps) with the step constants
// hoisted out of the element loop (step_size = lr / bc1).  Every operation is
// an explicit rounding (no contraction left to the compiler), so the result
// does not depend on the kernel it is inlined in.  False when the gradient
// or the second moment is not finite.
__device__ __forceinline__ bool adam_elem(float& p, float g, float& m, float& v, float step_size, float b1,
                                          float b2, float eps, float rs_bc2) {
  m = __fmaf_rn(b1, m, __fmul_rn(1.f - b1, g));
  v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.f - b2, g), g));
  p = __fsub_rn(p, __fmul_rn(step_size, __fdividef(m, __fmaf_rn(sqrtf(v), rs_bc2, eps))));
  return isfinite(g) && isfinite(v);
}

// ---------------------------------------------------------------------------
// Helpers of the level-of-detail hierarchies: order-preserving float <-> u32
// (for atomic min / max), 10-bit Morton quantisation in single precision, a
// symmetric 3x3 eigen-decomposition and a rotation-to-quaternion conversion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t float_order(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float float_unorder(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t quantise10(float x, float lo, float scale) {
  float f = floorf(__fmul_rn(__fsub_rn(x, lo), scale));
  if (!(f >= 0.f)) f = 0.f;
  if (f > 1023.f) f = 1023.f;
  return (uint32_t)f;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 (row-major A):
// A = V diag(lam) V^T with the eigenvectors in the columns of V.
__device__ __forceinline__ void jacobi3(float* A, float* lam, float* V) {
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    const float scale = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (!(off > 1e-14f * scale)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = A[3 * p + q];
      if (apq == 0.f) continue;
      const float theta = (A[3 * q + q] - A[3 * p + p]) / (2.f * apq);
      const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - s * akq;
        A[3 * k + q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - s * aqk;
        A[3 * q + k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
      }
    }
  }
  lam[0] = A[0];
  lam[1] = A[4];
  lam[2] = A[8];
}

// Unit quaternion (w,x,y,z), w >= 0, of a rotation matrix (row-major).
__device__ __forceinline__ float4 rot_to_quat(const float* R) {
  const float tr = R[0] + R[4] + R[8];
  float w, x, y, z;
  if (tr > 0.f) {
    const float s = sqrtf(tr + 1.f) * 2.f;
    w = 0.25f * s; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    const float s = sqrtf(1.f + R[0] - R[4] - R[8]) * 2.f;
    w = (R[7] - R[5]) / s; x = 0.25f * s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    const float s = sqrtf(1.f + R[4] - R[0] - R[8]) * 2.f;
    w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; y = 0.25f * s; z = (R[5] + R[7]) / s;
  } else {
    const float s = sqrtf(1.f + R[8] - R[0] - R[4]) * 2.f;
    w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; z = 0.25f * s;
  }
  if (w < 0.f) { w = -w; x = -x; y = -y; z = -z; }
  const float inv = 1.f / sqrtf(w * w + x * x + y * y + z * z);
  return make_float4(w * inv, x * inv, y * inv, z * inv);
}

// Screen size of a node of the progressive hierarchy, S = f_x 3 max scale /
// t_z (+inf at or behind the near plane), and whether it lies in view (its
// projected centre within the image widened by S).  Written with explicit
// round-to-nearest operations, so the reload pass and the projection's view
// cut take the same decisions.  R row-major, t: the world->camera pose.
__device__ __forceinline__ float hier_node_screen(const float* R, const float* t, float fx, float fy, float cx,
                                                  float cy, int W, int H, float znear, float4 m, float4 so,
                                                  bool& inview) {
  auto dot = [&](int r, float tr) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[3 * r], m.x), __fmul_rn(R[3 * r + 1], m.y)),
                               __fmul_rn(R[3 * r + 2], m.z)), tr);
  };
  const float tz = dot(2, t[2]);
  if (!(tz > znear)) {
    inview = false;
    return INFINITY;
  }
  const float tx = dot(0, t[0]), ty = dot(1, t[1]);
  const float S = __fdiv_rn(__fmul_rn(__fmul_rn(fx, 3.0f), expf(fmaxf(so.x, fmaxf(so.y, so.z)))), tz);
  const float u = __fadd_rn(__fdiv_rn(__fmul_rn(fx, tx), tz), cx);
  const float w = __fadd_rn(__fdiv_rn(__fmul_rn(fy, ty), tz), cy);
  inview = u >= -S && u <= __fadd_rn((float)W, S) && w >= -S && w <= __fadd_rn((float)H, S);
  return S;
}

// Pixel offset of a splat: dx = m - (p + 1/2) from the integer / fraction
// split of m.  The integer difference is exact, so dx is accurate to ~1 ulp.
__device__ __forceinline__ float splat_delta(float m_int, float m_frac, float p) {
  return (m_int - p) + (m_frac - 0.5f);
}

// Position of tile (tx, ty) inside a splat's rect, row-major; the pair of
// (view, Gaussian) for that tile sits at pair_off + this index.
__device__ __forceinline__ uint32_t rect_index(uint2 rect, int tx, int ty) {
  int x0 = rect.x & 0xffff, y0 = rect.x >> 16, x1 = rect.y & 0xffff;
  return (uint32_t)((ty - y0) * (x1 - x0 + 1) + (tx - x0));
}

}  // namespace gs
