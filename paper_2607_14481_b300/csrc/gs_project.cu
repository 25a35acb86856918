// EWA projection of every (view, Gaussian): the per-Gaussian stage of the
// splat renderer (Sec. 5.2).  One thread per (view, Gaussian); the Gaussian's
// parameters are read as coalesced float4 / planar-SH loads, the splat record
// is written as float4 structure-of-arrays.  HBM-bound: ~64 B (SH0) / 240 B
// (SH3) read and 64 B written per (view, Gaussian).
#include "gs_internal.h"

namespace gs {

namespace {

struct ProjectArgs {
  const float4* means4;
  const float4* scale_opa;
  const float4* quat;
  const float* sh;
  int64_t n;
  int64_t sh_stride;
  const float* poses;
  float znear;
  int clamp_j;
  float4* xy;
  float4* conic;
  float4* rgb;
  float* depth;
  uint2* rect;
  uint32_t* touched;
  uint32_t* aux;
  const int32_t* parent;  // level-of-detail cut (nullptr: every Gaussian is a candidate)
  int64_t n_leaf;
  float tau;
  // progressive hierarchy (h_active nullptr: none): the view cut at tau
  const int32_t* h_parent;
  const int32_t* h_child;
  const uint8_t* h_active;
  const uint32_t* h_n;
  int h_roots;            // 1: the render cut from the roots (h_active unused)
};

// Screen size of a node: f_x * 3 * max_k scale_k / t_z, infinite at or
// behind the near plane (never coarse enough).
__device__ __forceinline__ float screen_size(float tz, float4 so, float fx, float znear) {
  return tz <= znear ? INFINITY : fx * 3.0f * expf(fmaxf(so.x, fmaxf(so.y, so.z))) / tz;
}

template <int DEG>
__global__ void __launch_bounds__(256) k_project(const ProjectArgs a, const ViewTable vt) {
  constexpr int NC = (DEG + 1) * (DEG + 1);
  // the blocks of one chunk of Gaussians for every view are adjacent, so the
  // views of a chunk run close together and share its parameter and SH
  // lines in L2 (one DRAM read of them per step, not one per view)
  const int v = (int)(blockIdx.x % (unsigned)vt.views);
  const int64_t i = (int64_t)(blockIdx.x / (unsigned)vt.views) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t o = (int64_t)v * a.n + i;
  const ViewInfo vi = vt.v[v];
  const float* P = a.poses + 12 * v;
  const float R[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]};
  const float tc[3] = {P[3], P[7], P[11]};

  // the rotation and scale are loaded with the mean, so that the thread
  // waits for one memory round trip before the covariance, not two
  const float4 mu = a.means4[i], q = a.quat[i], so = a.scale_opa[i];
  // camera-space centre in double-single
  const df tz = df_dot3_add(R[6], mu.x, R[7], mu.y, R[8], mu.z, tc[2]);
  bool vis = !df_le(tz, a.znear);
  // the SH planes are read only once the splat is known to be visible, a
  // second dependent round trip: for a centre in front of the camera start
  // bringing them to L2 now
  if (vis) {
#pragma unroll
    for (int k = 0; k < 3 * NC; ++k)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(a.sh + (int64_t)k * a.sh_stride + i)));
  }
  df tx = {0.f, 0.f}, ty = {0.f, 0.f}, mx = {0.f, 0.f}, my = {0.f, 0.f};
  if (vis) {
    tx = df_dot3_add(R[0], mu.x, R[1], mu.y, R[2], mu.z, tc[0]);
    ty = df_dot3_add(R[3], mu.x, R[4], mu.y, R[5], mu.z, tc[1]);
    mx = df_add_f(df_mul_f(df_div(tx, tz), vi.fx), vi.cx);
    my = df_add_f(df_mul_f(df_div(ty, tz), vi.fy), vi.cy);
    // far off-screen (or non-finite) centres are culled before the split
    vis = fabsf(mx.hi) < 1e7f && fabsf(my.hi) < 1e7f;
  }
  if (vis && a.parent) {
    // level-of-detail cut: rendered iff (a leaf or S < tau) and every
    // ancestor has S >= tau
    bool sel = i < a.n_leaf || screen_size(tz.hi, so, vi.fx, a.znear) < a.tau;
    int32_t p = a.parent[i];
    for (int d = 0; d < 8 && sel && p >= 0 && p < a.n; ++d) {
      const float4 mp = a.means4[p];
      const float tzp = R[6] * mp.x + R[7] * mp.y + R[8] * mp.z + tc[2];
      sel = screen_size(tzp, a.scale_opa[p], vi.fx, a.znear) >= a.tau;
      p = a.parent[p];
    }
    vis = sel;
  }
  if (vis && a.h_roots) {
    // the render cut: descend from the roots while a node has children and
    // is coarser than tau; the nodes where the descent stops are drawn
    auto descends = [&](int64_t k) {
      if (a.h_child[4 * k] < 0) return false;
      bool in;
      const float S = hier_node_screen(R, tc, vi.fx, vi.fy, vi.cx, vi.cy, vi.W, vi.H, a.znear, a.means4[k],
                                       a.scale_opa[k], in);
      return S > a.tau;
    };
    bool sel = i < (int64_t)*a.h_n && a.h_parent[i] >= -1 && !descends(i);
    int32_t p = sel ? a.h_parent[i] : -1;
    for (int d = 0; p >= 0; ++d) {
      if (d >= 64 || !descends(p)) {
        sel = false;
        break;
      }
      p = a.h_parent[p];
    }
    vis = sel;
  } else if (vis && a.h_active) {
    // the active set refined for this view: rendered iff not expandable, and
    // either active or below an active ancestor through expandable nodes
    auto expandable = [&](int64_t k) {
      if (a.h_child[4 * k] < 0) return false;
      bool in;
      const float S = hier_node_screen(R, tc, vi.fx, vi.fy, vi.cx, vi.cy, vi.W, vi.H, a.znear, a.means4[k],
                                       a.scale_opa[k], in);
      return in && S > a.tau;
    };
    bool sel = i < (int64_t)*a.h_n && !expandable(i);
    if (sel && !a.h_active[i]) {
      int32_t p = a.h_parent[i];
      int d = 0;
      for (; p >= 0 && d < 64; ++d) {
        if (!expandable(p)) {
          sel = false;
          break;
        }
        if (a.h_active[p]) break;
        p = a.h_parent[p];
      }
      if (p < 0 || d >= 64) sel = false;
    }
    vis = sel;
  }
  float A = 0.f, B = 0.f, C = 0.f, r = 0.f, opa = 0.f;
  float mix = 0.f, miy = 0.f, mfx = 0.f, mfy = 0.f;
  int xlo = 1, ylo = 1, xhi = 0, yhi = 0;
  uint32_t auxbits = 0;
  if (vis) {
    // integer / fraction split of the pixel-space mean
    mix = floorf(mx.hi);
    mfx = (mx.hi - mix) + mx.lo;
    if (mfx < 0.f) { mix -= 1.f; mfx += 1.f; } else if (mfx >= 1.f) { mix += 1.f; mfx -= 1.f; }
    miy = floorf(my.hi);
    mfy = (my.hi - miy) + my.lo;
    if (mfy < 0.f) { miy -= 1.f; mfy += 1.f; } else if (mfy >= 1.f) { miy += 1.f; mfy -= 1.f; }

    const float qi = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float Rq[9];
    quat_rot(q.x * qi, q.y * qi, q.z * qi, q.w * qi, Rq);
    const float s[3] = {expf(so.x), expf(so.y), expf(so.z)};

    // perspective Jacobian with the frustum guard
    const float tzf = tz.hi, iz = 1.0f / tzf;
    float u = tx.hi * iz, w = ty.hi * iz;
    if (a.clamp_j) {
      const float limx = kGuard * 0.5f * (float)vi.W / vi.fx;
      const float limy = kGuard * 0.5f * (float)vi.H / vi.fy;
      if (u > limx) { u = limx; auxbits |= 8u; } else if (u < -limx) { u = -limx; auxbits |= 8u; }
      if (w > limy) { w = limy; auxbits |= 16u; } else if (w < -limy) { w = -limy; auxbits |= 16u; }
    }
    const float J00 = vi.fx * iz, J02 = -vi.fx * u * iz;
    const float J11 = vi.fy * iz, J12 = -vi.fy * w * iz;
    // T = J R (2x3); P = T Rq diag(s); 2D covariance = P P^T + 0.3 I
    const float T0[3] = {J00 * R[0] + J02 * R[6], J00 * R[1] + J02 * R[7], J00 * R[2] + J02 * R[8]};
    const float T1[3] = {J11 * R[3] + J12 * R[6], J11 * R[4] + J12 * R[7], J11 * R[5] + J12 * R[8]};
    float P0[3], P1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P0[c] = (T0[0] * Rq[c] + T0[1] * Rq[3 + c] + T0[2] * Rq[6 + c]) * s[c];
      P1[c] = (T1[0] * Rq[c] + T1[1] * Rq[3 + c] + T1[2] * Rq[6 + c]) * s[c];
    }
    const float ca = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2] + kDilation;
    const float cb = P0[0] * P1[0] + P0[1] * P1[1] + P0[2] * P1[2];
    const float cc = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2] + kDilation;
    const float det = ca * cc - cb * cb;
    vis = det > 0.f;
    if (vis) {
      const float id = 1.0f / det;
      A = cc * id; B = -cb * id; C = ca * id;
      const float hd = 0.5f * (ca - cc);
      const float lam = 0.5f * (ca + cc) + sqrtf(fmaxf(0.f, hd * hd + cb * cb));
      r = ceilf(3.0f * sqrtf(lam));
      opa = 1.0f / (1.0f + expf(-so.w));
      // tile rect: alpha can reach 1/255 only where A dx^2 + 2B dx dy + C dy^2
      // <= k = 2 ln(255 opacity), an ellipse whose bounding box has
      // half-widths sqrt(k ca), sqrt(k cc); widened by 0.1% + 0.05 px against
      // rounding and capped by the support box r, so that no tile where a
      // pixel passes the alpha test is left out (the image is unchanged)
      const float k = 2.0f * logf(255.0f * opa);
      vis = k > 0.f;
      if (vis) {
        const float hx = fminf(r, fmaf(sqrtf(k * ca), 1.001f, 0.05f));
        const float hy = fminf(r, fmaf(sqrtf(k * cc), 1.001f, 0.05f));
        const float mxf = mix + mfx, myf = miy + mfy;  // m = mi + frac, frac in [0,1)
        // tile edges are powers of two: the scale by their inverse is exact
        const float itw = 1.0f / (float)vt.tw, ith = 1.0f / (float)vt.th;
        xlo = max(0, (int)floorf((mxf - hx) * itw));
        xhi = min(vi.TX - 1, (int)floorf((mxf + hx) * itw));
        ylo = max(0, (int)floorf((myf - hy) * ith));
        yhi = min(vi.TY - 1, (int)floorf((myf + hy) * ith));
        vis = xlo <= xhi && ylo <= yhi;
      }
    }
  }
  float3 col = make_float3(0.f, 0.f, 0.f);
  if (vis) {
    // SH colour seen from the camera centre -R^T t
    const float oc0 = -(R[0] * tc[0] + R[3] * tc[1] + R[6] * tc[2]);
    const float oc1 = -(R[1] * tc[0] + R[4] * tc[1] + R[7] * tc[2]);
    const float oc2 = -(R[2] * tc[0] + R[5] * tc[1] + R[8] * tc[2]);
    float dx = mu.x - oc0, dy = mu.y - oc1, dz = mu.z - oc2;
    const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[NC];
    sh_basis<DEG>(dx, dy, dz, Y);
    float cv[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NC; ++k) acc += a.sh[(int64_t)(ch * NC + k) * a.sh_stride + i] * Y[k];
      acc += 0.5f;
      if (acc < 0.f) { acc = 0.f; auxbits |= 1u << ch; }
      cv[ch] = acc;
    }
    col = make_float3(cv[0], cv[1], cv[2]);
  }
  if (!vis) {
    A = B = C = opa = r = 0.f;
    mix = miy = mfx = mfy = 0.f;
    xlo = ylo = 1; xhi = yhi = 0;
    auxbits = 0;
  }
  a.xy[o] = make_float4(mix, miy, mfx, mfy);
  a.conic[o] = make_float4(A, B, C, opa);
  a.rgb[o] = make_float4(col.x, col.y, col.z, r);
  a.depth[o] = tz.hi;
  a.rect[o] = make_uint2((uint32_t)xlo | ((uint32_t)ylo << 16), (uint32_t)xhi | ((uint32_t)yhi << 16));
  a.touched[o] = vis ? (uint32_t)((xhi - xlo + 1) * (yhi - ylo + 1)) : 0u;
  a.aux[o] = auxbits;
}

}  // namespace

gs_status launch_project(const gs_params& p, const float* poses, const ViewTable& vt,
                         const gs_raster_cfg& cfg, const gs_splats& out, cudaStream_t s, const int32_t* parent,
                         int64_t n_leaf, float tau, const gs_hier* hier, bool hier_roots) {
  ProjectArgs a;
  a.means4 = reinterpret_cast<const float4*>(p.means4);
  a.scale_opa = reinterpret_cast<const float4*>(p.scale_opa);
  a.quat = reinterpret_cast<const float4*>(p.quat);
  a.sh = p.sh;
  a.n = p.n;
  a.sh_stride = p.sh_stride > 0 ? p.sh_stride : p.n;
  a.poses = poses;
  a.znear = cfg.znear;
  a.clamp_j = cfg.clamp_jacobian;
  a.xy = reinterpret_cast<float4*>(out.xy);
  a.conic = reinterpret_cast<float4*>(out.conic);
  a.rgb = reinterpret_cast<float4*>(out.rgb);
  a.depth = out.depth;
  a.rect = reinterpret_cast<uint2*>(out.rect);
  a.touched = out.touched;
  a.aux = out.aux;
  a.parent = parent;
  a.n_leaf = n_leaf;
  a.tau = tau;
  a.h_parent = hier ? hier->parent : nullptr;
  a.h_child = hier ? hier->child : nullptr;
  a.h_active = hier ? hier->active : nullptr;
  a.h_n = hier ? hier->n_nodes : nullptr;
  a.h_roots = hier && hier_roots ? 1 : 0;
  if (p.n == 0) return GS_OK;
  const unsigned grid = (unsigned)((p.n + 255) / 256) * (unsigned)vt.views;
  switch (p.sh_degree) {
    case 0: k_project<0><<<grid, 256, 0, s>>>(a, vt); break;
    case 1: k_project<1><<<grid, 256, 0, s>>>(a, vt); break;
    case 2: k_project<2><<<grid, 256, 0, s>>>(a, vt); break;
    default: k_project<3><<<grid, 256, 0, s>>>(a, vt); break;
  }
  return check_launch("k_project");
}

}  // namespace gs
