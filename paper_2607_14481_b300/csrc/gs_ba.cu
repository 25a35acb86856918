// Local bundle adjustment on the device (Sec. 5.1 "Local Bundle Adjustment",
// supplementary "Fast Bundle Adjustment"): every landmark keeps a fixed subset
// of at most M observing keyframes, so one Levenberg-Marquardt iteration is
//
//   k_ba_linearize  one group of G >= M lanes per landmark, one lane per
//                   observation slot: residual and Jacobians (pose, landmark,
//                   shared focal), the landmark's 3x3 block summed over the
//                   group, damped and factorised (V = L L^T), and per
//                   observation the Schur terms in the symmetric form
//                   Z = W L^-T (W = J_c^T J_X), so that the landmark's share
//                   of the reduced camera matrix is J_c^T J_c - Z Z^T.
//   k_ba_reduce     a few CTAs per block of the reduced system: a free
//                   keyframe's 6x6 diagonal block (with its right-hand side and
//                   focal column), a pair of free keyframes (-sum Z_a Z_b^T over
//                   the landmarks both observe), or the focal entry and the
//                   cost.  Entry lists are built once per solve, in landmark
//                   order; each thread owns one value of the block (coalesced
//                   record reads) and sums in double-float; deterministic, no
//                   atomics.
//   k_ba_solve      one CTA: assemble the dense reduced system in double-float,
//                   damp, scale to unit diagonal, invert it in float32 with the
//                   symmetric sweep (Gauss-Jordan) operator on 4x4 register
//                   blocks, then solve with double-float residual refinement;
//                   candidate keyframe poses.
//   k_ba_candidate  back-substitution dX = -L^-T (q + p_f df + sum Z^T dc),
//                   candidate cost; the last CTA to finish takes the
//                   accept/reject decision and updates lambda (no host sync).
//
// The work is small (20 keyframes, 10k landmarks, 8 slots: ~80k observations)
// and latency-bound.  Everything runs in float32, with double-float (value +
// rounding error) sums where cancellation needs them: sm_103a runs float64 at
// a small fraction of the float32 rate.
#include <algorithm>
#include <cmath>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kZ = 20;    // floats per observation: Z (6 rows x 3), 2 unused
constexpr int kD = 40;    // floats per observation: net 6x6 upper triangle (21), rhs (6), focal column (6),
                          // raw J_c^T J_c diagonal (6), 1 unused
constexpr int kLR = 16;   // floats per landmark: L^-1 (6), q = L^-1 g_p (3), p_f = L^-1 w_f (3), focal net,
                          // raw sum J_f^2, focal rhs, cost
constexpr int kBR = 48;   // (hi, lo) values per block result
constexpr int kSplitD = 16, kSplitP = 4, kSplitF = 32;  // CTAs per diagonal / pair / focal block
constexpr int kUnroll = 4;                             // independent record loads in flight per thread
constexpr int kRedThreads = 320;  // threads of a reduce CTA
constexpr int kMaxPairs = GS_BA_MAX_FREE * (GS_BA_MAX_FREE - 1) / 2;
constexpr int kMaxDim = 6 * GS_BA_MAX_FREE + 1;
constexpr int kSolveThreads = 1024;  // one thread per 4x4 block of the (padded) reduced system
constexpr int kRefine = 2;  // solves per iteration: one plus one refinement
constexpr int kMaxPad = (kMaxDim + 3) & ~3;
constexpr float kZmin = 1e-6f;
constexpr float kDmin = 1e-6f, kDmax = 1e32f;
constexpr float kPivotMin = 1e-7f;  // sweep pivot floor of the unit-diagonal scaled system

struct BaState {
  double lam;
  double cost;                          // cost at the current state
  float dc[kMaxPad];                    // keyframe/focal step of the current iteration
  float pose_cand[GS_BA_MAX_CAMS * 12];
  float f_cand;
  int accepted;                         // decision of the previous iteration
  int solve_ok;
  unsigned ticket;                      // CTAs of k_ba_candidate finished
};

struct BaArgs {
  int P, M, N, opt_focal, n_free, dim, n_pairs, iter;
  float cx, cy;
  int8_t free_of[GS_BA_MAX_CAMS];  // free index of keyframe k, -1 if fixed
  int8_t cam_of[GS_BA_MAX_FREE];   // keyframe of free index i
  uint8_t pa[kMaxPairs], pb[kMaxPairs];
  const int32_t* obs_in;
  int8_t* obs;  // validated slots
  const float2* uv;
  float* poses;
  float* points;
  float* focal;
  float* xcand;
  float* zrec;
  float* drec;      // diagonal-block records, keyframe-major: [free keyframe][list position]
  int32_t* dpos;    // list position of each observation slot of a free keyframe
  float* lrec;
  int32_t* lists;
  int32_t* counts;
  float2* bres;      // per split CTA
  float2* bfin;      // per block, splits combined
  unsigned* bticket; // split CTAs of a block finished
  float2* partials;
  BaState* st;
  double* trace;
  uint32_t* status;
};

// upper-triangle order of a 6x6 block: (0,0) (0,1) .. (0,5) (1,1) .. (5,5)
__constant__ int8_t c_tri_i[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__constant__ int8_t c_tri_j[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

// double-float accumulation: s + c carries the sum (Knuth's two-sum)
__device__ __forceinline__ void df_add(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// Sums NV double-float values over the CTA in a fixed order; thread v < NV
// returns value v as a normalised (hi, lo) pair (others 0).
template <int NV>
__device__ float2 block_sum_df(float (&s)[NV], float (&c)[NV], float (*sh)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s[v], off);
      const float c2 = __shfl_xor_sync(0xffffffffu, c[v], off);
      df_add(s[v], c[v], s2);
      c[v] += c2;
    }
    if (lane == 0) {
      sh[warp * NV + v][0] = s[v];
      sh[warp * NV + v][1] = c[v];
    }
  }
  __syncthreads();
  float hs = 0.f, hc = 0.f;
  if ((int)threadIdx.x < NV)
    for (int w = 0; w < nw; ++w) {
      df_add(hs, hc, sh[w * NV + threadIdx.x][0]);
      hc += sh[w * NV + threadIdx.x][1];
    }
  const float hi = hs + hc;
  return make_float2(hi, hc - (hi - hs));
}

__device__ __forceinline__ float clampf(float x) { return fminf(fmaxf(x, kDmin), kDmax); }

// Validates the observation slots (out-of-range or repeated keyframes become
// empty, with a status bit) and initialises the solver state.
__global__ void __launch_bounds__(256) k_ba_prepare(const BaArgs a, double lambda0) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  for (int b = l; b < a.n_free + a.n_pairs + 1; b += gridDim.x * blockDim.x) a.bticket[b] = 0u;
  if (l == 0) {
    a.st->lam = lambda0;
    a.st->accepted = 0;
    a.st->solve_ok = 0;
    a.st->ticket = 0;
  }
  if (l >= a.P) return;
  bool bad = false;
  for (int m = 0; m < a.M; ++m) {
    int k = a.obs_in[(size_t)l * a.M + m];
    if (k < -1 || k >= a.N) {
      bad = true;
      k = -1;
    }
    if (k >= 0)
      for (int j = 0; j < m; ++j)
        if (a.obs[(size_t)l * a.M + j] == k) {
          bad = true;
          k = -1;
          break;
        }
    a.obs[(size_t)l * a.M + m] = (int8_t)k;
  }
  if (bad) atomicOr(a.status, GS_BA_BAD_OBS);
}

// Entry lists of the diagonal (free keyframe) and pair blocks, in landmark
// order: CTA b scans all landmarks and compacts the matches.
__global__ void __launch_bounds__(256) k_ba_lists(const BaArgs a) {
  __shared__ int s_warp[8];
  const int b = blockIdx.x;
  const bool diag = b < a.n_free;
  const int ka = a.cam_of[diag ? b : a.pa[b - a.n_free]];
  const int kc = diag ? -1 : a.cam_of[a.pb[b - a.n_free]];
  int32_t* out = a.lists + (size_t)b * a.P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = 0;
  constexpr int kPer = 4;  // landmarks per thread and chunk, loaded before the compaction
  for (int l0 = 0; l0 < a.P; l0 += kPer * blockDim.x) {
    int sa[kPer], sc[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int l = l0 + u * blockDim.x + threadIdx.x;
      sa[u] = sc[u] = -1;
      if (l < a.P)
        for (int m = 0; m < a.M; ++m) {
          const int k = a.obs[(size_t)l * a.M + m];
          if (k == ka) sa[u] = m;
          if (k == kc) sc[u] = m;
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {  // compaction in landmark order
      const int l = l0 + u * blockDim.x + threadIdx.x;
      const bool hit = sa[u] >= 0 && (diag || sc[u] >= 0);
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (lane == 0) s_warp[warp] = __popc(bal);
      __syncthreads();
      int before = 0, total = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        before += w < warp ? s_warp[w] : 0;
        total += s_warp[w];
      }
      if (hit) {
        const int pos = base + before + __popc(bal & ((1u << lane) - 1u));
        out[pos] = diag ? (l << 4) | sa[u] : (l << 8) | (sa[u] << 4) | sc[u];
        if (diag) a.dpos[(size_t)l * a.M + sa[u]] = pos;
      }
      base += total;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) a.counts[b] = base;
}

template <int G>
__global__ void __launch_bounds__(256) k_ba_linearize(const BaArgs a) {
  const int gl = threadIdx.x & (G - 1);
  const int l = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
  const bool live = l < a.P;
  const BaState* st = a.st;
  const bool take = st->accepted != 0;
  float X0 = 0.f, X1 = 0.f, X2 = 0.f;
  if (live) {
    const float* src = take ? a.xcand : a.points;
    X0 = src[3 * l];
    X1 = src[3 * l + 1];
    X2 = src[3 * l + 2];
    if (take && gl == 0) {  // the previous candidate was accepted
      a.points[3 * l] = X0;
      a.points[3 * l + 1] = X1;
      a.points[3 * l + 2] = X2;
    }
  }
  const float f = *a.focal;
  const int k = (live && gl < a.M) ? (int)a.obs[(size_t)l * a.M + gl] : -1;
  float r0 = 0.f, r1 = 0.f, jf0 = 0.f, jf1 = 0.f;
  float jx0[3] = {0.f, 0.f, 0.f}, jx1[3] = {0.f, 0.f, 0.f};
  float jc0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, jc1[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // a free keyframe's slot always writes its records (zeros when the point
  // is behind the camera), so the later kernels never read stale entries
  const int fi = k >= 0 ? (int)a.free_of[k] : -1;
  if (k >= 0) {
    const float* T = a.poses + 12 * k;
    const float RX0 = fmaf(T[0], X0, fmaf(T[1], X1, T[2] * X2));
    const float RX1 = fmaf(T[4], X0, fmaf(T[5], X1, T[6] * X2));
    const float RX2 = fmaf(T[8], X0, fmaf(T[9], X1, T[10] * X2));
    const float x = RX0 + T[3], y = RX1 + T[7], z = RX2 + T[11];
    if (z > kZmin) {
      const float iz = 1.f / z;
      const float xn = x * iz, yn = y * iz, fz = f * iz;
      const float2 o = a.uv[(size_t)l * a.M + gl];
      r0 = fmaf(f, xn, a.cx) - o.x;
      r1 = fmaf(f, yn, a.cy) - o.y;
#pragma unroll
      for (int j = 0; j < 3; ++j) {  // d(u,v)/dX = dpi R
        jx0[j] = fz * fmaf(-xn, T[8 + j], T[j]);
        jx1[j] = fz * fmaf(-yn, T[8 + j], T[4 + j]);
      }
      if (fi >= 0) {  // d/dtheta of Exp(theta) R X is -[R X]x; d/dt is the identity
        jc0[0] = -fz * xn * RX1;
        jc0[1] = fz * fmaf(xn, RX0, RX2);
        jc0[2] = -fz * RX1;
        jc0[3] = fz;
        jc0[5] = -fz * xn;
        jc1[0] = -fz * fmaf(yn, RX1, RX2);
        jc1[1] = fz * yn * RX0;
        jc1[2] = fz * RX0;
        jc1[4] = fz;
        jc1[5] = -fz * yn;
      }
      if (a.opt_focal) {
        jf0 = xn;
        jf1 = yn;
      }
    }
  }
  // landmark block V = sum J_X^T J_X, g_p = sum J_X^T r, w_f = sum J_X^T J_f,
  // sum J_f^2, g_f = sum J_f r, cost = sum r^2 over the group
  float s[15];
  s[0] = fmaf(jx0[0], jx0[0], jx1[0] * jx1[0]);
  s[1] = fmaf(jx0[0], jx0[1], jx1[0] * jx1[1]);
  s[2] = fmaf(jx0[0], jx0[2], jx1[0] * jx1[2]);
  s[3] = fmaf(jx0[1], jx0[1], jx1[1] * jx1[1]);
  s[4] = fmaf(jx0[1], jx0[2], jx1[1] * jx1[2]);
  s[5] = fmaf(jx0[2], jx0[2], jx1[2] * jx1[2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    s[6 + j] = fmaf(jx0[j], r0, jx1[j] * r1);
    s[9 + j] = fmaf(jx0[j], jf0, jx1[j] * jf1);
  }
  s[12] = fmaf(jf0, jf0, jf1 * jf1);
  s[13] = fmaf(jf0, r0, jf1 * r1);
  s[14] = fmaf(r0, r0, r1 * r1);
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
    for (int v = 0; v < 15; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], off);

  // damped block V = L L^T; only L^-1 is kept (float32: V itself is a float32
  // sum, so a wider factorisation would not add accuracy)
  const float lamf = (float)fmin(st->lam, 1e30);
  const float v00 = fmaf(lamf, clampf(s[0]), s[0]), v11 = fmaf(lamf, clampf(s[3]), s[3]),
              v22 = fmaf(lamf, clampf(s[5]), s[5]);
  bool ok = v00 > 0.f;
  const float i00 = ok ? rsqrtf(v00) : 0.f;
  const float l10 = s[1] * i00, l20 = s[2] * i00;
  const float d11 = v11 - l10 * l10;
  ok = ok && d11 > 0.f;
  const float i11 = ok ? rsqrtf(d11) : 0.f;
  const float l21 = (s[4] - l20 * l10) * i11;
  const float d22 = v22 - l20 * l20 - l21 * l21;
  ok = ok && d22 > 0.f;
  const float i22 = ok ? rsqrtf(d22) : 0.f;
  float Li[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // L^-1: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
  if (ok) {
    Li[0] = i00;
    Li[1] = -l10 * i00 * i11;
    Li[2] = i11;
    Li[3] = (l10 * l21 * i11 - l20) * i00 * i22;
    Li[4] = -l21 * i11 * i22;
    Li[5] = i22;
  } else if (live && gl == 0) {
    atomicOr(a.status, GS_BA_DEGENERATE);  // frozen: no Schur terms, no step
  }
  const float q0 = Li[0] * s[6], q1 = fmaf(Li[1], s[6], Li[2] * s[7]),
              q2 = fmaf(Li[3], s[6], fmaf(Li[4], s[7], Li[5] * s[8]));
  const float p0 = Li[0] * s[9], p1 = fmaf(Li[1], s[9], Li[2] * s[10]),
              p2 = fmaf(Li[3], s[9], fmaf(Li[4], s[10], Li[5] * s[11]));

  if (fi >= 0) {
    const size_t o = (size_t)l * a.M + gl;
    float z[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float w0 = fmaf(jc0[i], jx0[0], jc1[i] * jx1[0]);
      const float w1 = fmaf(jc0[i], jx0[1], jc1[i] * jx1[1]);
      const float w2 = fmaf(jc0[i], jx0[2], jc1[i] * jx1[2]);
      z[i][0] = Li[0] * w0;
      z[i][1] = fmaf(Li[1], w0, Li[2] * w1);
      z[i][2] = fmaf(Li[3], w0, fmaf(Li[4], w1, Li[5] * w2));
    }
    float4* zo = reinterpret_cast<float4*>(a.zrec + o * kZ);
    zo[0] = make_float4(z[0][0], z[0][1], z[0][2], z[1][0]);
    zo[1] = make_float4(z[1][1], z[1][2], z[2][0], z[2][1]);
    zo[2] = make_float4(z[2][2], z[3][0], z[3][1], z[3][2]);
    zo[3] = make_float4(z[4][0], z[4][1], z[4][2], z[5][0]);
    zo[4] = make_float4(z[5][1], z[5][2], 0.f, 0.f);
    float d[kD];
#pragma unroll
    for (int e = 0; e < 21; ++e) {
      const int i = e < 6 ? 0 : e < 11 ? 1 : e < 15 ? 2 : e < 18 ? 3 : e < 20 ? 4 : 5;
      const int j = e - (i == 0 ? 0 : i == 1 ? 5 : i == 2 ? 9 : i == 3 ? 12 : i == 4 ? 14 : 15);
      const float zz = fmaf(z[i][0], z[j][0], fmaf(z[i][1], z[j][1], z[i][2] * z[j][2]));
      d[e] = fmaf(jc0[i], jc0[j], fmaf(jc1[i], jc1[j], -zz));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float zq = fmaf(z[i][0], q0, fmaf(z[i][1], q1, z[i][2] * q2));
      const float zp = fmaf(z[i][0], p0, fmaf(z[i][1], p1, z[i][2] * p2));
      d[21 + i] = zq - fmaf(jc0[i], r0, jc1[i] * r1);
      d[27 + i] = fmaf(jc0[i], jf0, fmaf(jc1[i], jf1, -zp));
      d[33 + i] = fmaf(jc0[i], jc0[i], jc1[i] * jc1[i]);
    }
    d[39] = 0.f;
    float4* dout = reinterpret_cast<float4*>(a.drec + ((size_t)fi * a.P + a.dpos[o]) * kD);
#pragma unroll
    for (int e = 0; e < kD / 4; ++e) dout[e] = make_float4(d[4 * e], d[4 * e + 1], d[4 * e + 2], d[4 * e + 3]);
  }
  if (live && gl == 0) {
    float4* lo = reinterpret_cast<float4*>(a.lrec + (size_t)l * kLR);
    lo[0] = make_float4(Li[0], Li[1], Li[2], Li[3]);
    lo[1] = make_float4(Li[4], Li[5], q0, q1);
    lo[2] = make_float4(q2, p0, p1, p2);
    const float pp = fmaf(p0, p0, fmaf(p1, p1, p2 * p2));
    const float pq = fmaf(p0, q0, fmaf(p1, q1, p2 * q2));
    lo[3] = make_float4(s[12] - pp, s[12], pq - s[13], s[14]);
  }
}

// CTA c covers one split of one block.  Diagonal block: thread (slot, g)
// adds values 4g..4g+3 of the records of entries slot, slot + 32, ... (float4
// reads of the keyframe-major records); pair block: thread (slot, i) adds row
// i of Z_a Z_c^T for its entries (Z_c read whole); focal block: thread
// (slot, v) adds value v of the landmark records.  Per-thread sums are float32
// over a few entries (double-float for the focal block, which carries the
// cost); slots are combined in double-float in a fixed order, and the last
// split CTA of a block to finish combines the splits' (hi, lo) results.
constexpr int kDiagSlots = kRedThreads / 10, kPairSlots = kRedThreads / 6, kFocSlots = kRedThreads / 4;
__global__ void __launch_bounds__(kRedThreads) k_ba_reduce(const BaArgs a) {
  __shared__ float red[kRedThreads * 6];  // per thread up to 6 values (pair rows)
  __shared__ float redc[kRedThreads];     // focal: double-float error terms
  __shared__ bool s_last;
  const int c = blockIdx.x, t = threadIdx.x;
  const int nd = a.n_free * kSplitD, npp = a.n_pairs * kSplitP;
  int nv, blk, chunk0, nsplit;
  if (c < nd) {  // diagonal block of free keyframe c / kSplitD
    const int b = c / kSplitD, sp = c % kSplitD;
    nv = 40;  // value 39 is the record's zero pad
    blk = b;
    chunk0 = b * kSplitD;
    nsplit = kSplitD;
    const int slot = t / 10, g = t % 10, stride = kSplitD * kDiagSlots;
    const float4* R = reinterpret_cast<const float4*>(a.drec + (size_t)b * a.P * kD) + g;
    const int n = a.counts[b];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e0 = sp * kDiagSlots + slot; e0 < n; e0 += kUnroll * stride) {
      float4 x[kUnroll];
      float w[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int e = e0 + u * stride;
        w[u] = e < n ? 1.f : 0.f;
        x[u] = R[(size_t)min(e, n - 1) * (kD / 4)];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        acc.x = fmaf(w[u], x[u].x, acc.x);
        acc.y = fmaf(w[u], x[u].y, acc.y);
        acc.z = fmaf(w[u], x[u].z, acc.z);
        acc.w = fmaf(w[u], x[u].w, acc.w);
      }
    }
    red[slot * 40 + 4 * g] = acc.x;
    red[slot * 40 + 4 * g + 1] = acc.y;
    red[slot * 40 + 4 * g + 2] = acc.z;
    red[slot * 40 + 4 * g + 3] = acc.w;
  } else if (c < nd + npp) {  // off-diagonal block: sum Z_a Z_c^T
    const int p = (c - nd) / kSplitP, sp = (c - nd) % kSplitP;
    nv = 36;
    blk = a.n_free + p;
    chunk0 = nd + p * kSplitP;
    nsplit = kSplitP;
    const int slot = t / 6, i = t % 6, stride = kSplitP * kPairSlots;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (slot < kPairSlots) {
      const int32_t* L = a.lists + (size_t)blk * a.P;
      const int n = a.counts[blk];
      for (int e0 = sp * kPairSlots + slot; e0 < n; e0 += kUnroll * stride) {
        // unconditional loads (past the end: the last entry, weighted 0), so
        // that the list reads, then the record reads, are in flight together
        int ent[kUnroll];
        float w[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u * stride;
          w[u] = e < n ? 1.f : 0.f;
          ent[u] = __ldg(L + min(e, n - 1));
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const size_t base = (size_t)(ent[u] >> 8) * a.M;
          const float* za = a.zrec + (base + ((ent[u] >> 4) & 15)) * kZ + 3 * i;
          const float4* zc4 = reinterpret_cast<const float4*>(a.zrec + (base + (ent[u] & 15)) * kZ);
          const float z0 = w[u] * za[0], z1 = w[u] * za[1], z2 = w[u] * za[2];
          float zc[20];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const float4 v = zc4[q];
            zc[4 * q] = v.x; zc[4 * q + 1] = v.y; zc[4 * q + 2] = v.z; zc[4 * q + 3] = v.w;
          }
#pragma unroll
          for (int j = 0; j < 6; ++j)
            acc[j] = fmaf(z0, zc[3 * j], fmaf(z1, zc[3 * j + 1], fmaf(z2, zc[3 * j + 2], acc[j])));
        }
      }
      #pragma unroll
      for (int j = 0; j < 6; ++j) red[slot * 36 + 6 * i + j] = acc[j];
    }
  } else {  // focal entry, its raw diagonal, its right-hand side, the cost
    const int sp = c - nd - npp;
    nv = 4;
    blk = a.n_free + a.n_pairs;
    chunk0 = nd + npp;
    nsplit = kSplitF;
    const int slot = t / 4, v = t % 4, stride = kSplitF * kFocSlots;
    float s = 0.f, cc = 0.f;
    for (int l0 = sp * kFocSlots + slot; l0 < a.P; l0 += kUnroll * stride) {
      float x[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int l = l0 + u * stride;
        x[u] = (l < a.P ? 1.f : 0.f) * a.lrec[(size_t)min(l, a.P - 1) * kLR + 12 + v];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) df_add(s, cc, x[u]);
    }
    red[t] = s;
    redc[t] = cc;
  }
  __syncthreads();
  if (t < nv) {
    const int slots = c < nd ? kDiagSlots : c < nd + npp ? kPairSlots : kFocSlots;
    float hs = 0.f, hc = 0.f;
    for (int q = 0; q < slots; ++q) {
      df_add(hs, hc, red[q * nv + t]);
      if (c >= nd + npp) hc += redc[q * nv + t];
    }
    const float hi = hs + hc;
    a.bres[(size_t)c * kBR + t] = make_float2(hi, hc - (hi - hs));
  }
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&a.bticket[blk], 1u) == (unsigned)nsplit - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (t < nv) {
    const volatile float2* R = a.bres;
    float hs = 0.f, hc = 0.f;
    for (int q = 0; q < nsplit; ++q) {
      const float ux = R[(size_t)(chunk0 + q) * kBR + t].x, uy = R[(size_t)(chunk0 + q) * kBR + t].y;
      df_add(hs, hc, ux);
      hc += uy;
    }
    const float hi = hs + hc;
    a.bfin[(size_t)blk * kBR + t] = make_float2(hi, hc - (hi - hs));
  }
  if (t == 0) a.bticket[blk] = 0u;
}

// Rodrigues: E = I + A K + B K^2 with K = [w]x, A = sin t / t, B = (1 - cos t) / t^2.
__device__ void exp_so3(float w0, float w1, float w2, float E[9]) {
  const float t2 = w0 * w0 + w1 * w1 + w2 * w2;
  float A, B;
  if (t2 < 1e-8f) {
    A = 1.f - t2 * (1.f / 6.f);
    B = 0.5f - t2 * (1.f / 24.f);
  } else {
    const float t = sqrtf(t2);
    float sn, cs;
    sincosf(t, &sn, &cs);
    A = sn / t;
    B = (1.f - cs) / t2;
  }
  E[0] = 1.f - B * (w1 * w1 + w2 * w2);
  E[1] = -A * w2 + B * w0 * w1;
  E[2] = A * w1 + B * w0 * w2;
  E[3] = A * w2 + B * w0 * w1;
  E[4] = 1.f - B * (w0 * w0 + w2 * w2);
  E[5] = -A * w0 + B * w1 * w2;
  E[6] = -A * w1 + B * w0 * w2;
  E[7] = A * w0 + B * w1 * w2;
  E[8] = 1.f - B * (w0 * w0 + w1 * w1);
}

__global__ void __launch_bounds__(kSolveThreads) k_ba_solve(const BaArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int n = a.dim, np = (n + 3) & ~3, nbk = np >> 2, nf = a.n_free, fidx = 6 * nf;
  float* Sh = sm;             // reduced system, double-float [np][np]
  float* Sl = Sh + np * np;
  float* Ai = Sl + np * np;   // inverse of the scaled system [np][np]
  float* rh = Ai + np * np;   // right-hand side, double-float
  float* rl = rh + np;
  float* xh = rl + np;        // solution, double-float
  float* xl = xh + np;
  float* dsc = xl + np;       // Jacobi scale
  float* raw = dsc + np;      // undamped diagonal of the camera block
  float* tmp = raw + np;      // [np]
  __shared__ int s_ok;
  BaState* st = a.st;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < np * np; e += nt) Sh[e] = Sl[e] = 0.f;
  for (int i = tid; i < np; i += nt) rh[i] = rl[i] = xh[i] = xl[i] = raw[i] = 0.f;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  // every value of the reduced system: loads first (independent), then placement
  const int nvals = nf * 39 + a.n_pairs * 36 + 4;
  constexpr int kPer = (GS_BA_MAX_FREE * 39 + kMaxPairs * 36 + 4 + kSolveThreads - 1) / kSolveThreads;
  float2 hv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = tid + u * nt;
    int src = -1;
    if (e < nf * 39) {
      src = (e / 39) * kBR + e % 39;
    } else if (e < nf * 39 + a.n_pairs * 36) {
      const int f = e - nf * 39;
      src = (nf + f / 36) * kBR + f % 36;
    } else if (e < nvals) {
      src = (nf + a.n_pairs) * kBR + (e - nf * 39 - a.n_pairs * 36);
    }
    hv[u] = src >= 0 ? a.bfin[src] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = tid + u * nt;
    const float2 h = hv[u];
    if (e < nf * 39) {
      const int fa = e / 39, v = e % 39, o = 6 * fa;
      if (v < 21) {
        const int i = o + c_tri_i[v], j = o + c_tri_j[v];
        Sh[i * np + j] = Sh[j * np + i] = h.x;
        Sl[i * np + j] = Sl[j * np + i] = h.y;
      } else if (v < 27) {
        rh[o + v - 21] = h.x;
        rl[o + v - 21] = h.y;
      } else if (v < 33) {
        if (a.opt_focal) {
          const int i = o + v - 27;
          Sh[i * np + fidx] = Sh[fidx * np + i] = h.x;
          Sl[i * np + fidx] = Sl[fidx * np + i] = h.y;
        }
      } else {
        raw[o + v - 33] = h.x;
      }
    } else if (e < nf * 39 + a.n_pairs * 36) {
      const int f = e - nf * 39, p = f / 36, v = f % 36;
      const int i = 6 * a.pa[p] + v / 6, j = 6 * a.pb[p] + v % 6;
      Sh[i * np + j] = Sh[j * np + i] = -h.x;
      Sl[i * np + j] = Sl[j * np + i] = -h.y;
    } else if (e < nvals) {
      const int v = e - nf * 39 - a.n_pairs * 36;
      if (v == 3) {
        st->cost = (double)h.x + (double)h.y;
      } else if (a.opt_focal) {
        if (v == 0) {
          Sh[fidx * np + fidx] = h.x;
          Sl[fidx * np + fidx] = h.y;
        } else if (v == 1) {
          raw[fidx] = h.x;
        } else {
          rh[fidx] = h.x;
          rl[fidx] = h.y;
        }
      }
    }
  }
  __syncthreads();
  // Marquardt damping and scaling to unit diagonal; padding rows are identity
  const float lamf = (float)fmin(st->lam, 1e30);
  for (int i = tid; i < np; i += nt) {
    if (i < n) {
      float h = Sh[i * np + i], l = Sl[i * np + i];
      df_add(h, l, lamf * clampf(raw[i]));
      const float hi = h + l;
      Sh[i * np + i] = hi;
      Sl[i * np + i] = l - (hi - h);
      if (!(hi > 0.f) || !isfinite(hi)) s_ok = 0;
      dsc[i] = hi > 0.f ? rsqrtf(hi) : 0.f;
    } else {
      Sh[i * np + i] = 1.f;
      dsc[i] = 1.f;
    }
  }
  __syncthreads();
  // symmetric block sweep (Gauss-Jordan on 4x4 pivot blocks): after pivoting
  // on every block K the matrix holds -A^-1.  Thread t owns the 4x4 block
  // (I, J) = (t / nbk, t % nbk) of the full matrix in registers, so the
  // owners of block row K are consecutive threads (one or two warps) and the
  // threads of a warp share one or two block rows.  By symmetry everything a
  // step needs comes from the pivot row: with D = A_KK, P_J = A_KJ and
  // W_J = D^-1 A_KJ,  A_IJ -= W_I^T P_J (I, J != K), A_IK <- W_I^T,
  // A_KJ <- W_J, A_KK <- -D^-1.  Look-ahead: the owners of row K + 1 update
  // their blocks first and prepare pivot K + 1 (publish P, invert D, form W)
  // behind a barrier of their own warps while the other warps finish step K;
  // one CTA barrier per step.
  constexpr int kRowPad = 20;  // floats per published 4x4 block (bank-conflict padding)
  __shared__ __align__(16) float s_P[2][kMaxPad / 4][kRowPad];  // pivot row blocks A_KJ
  __shared__ __align__(16) float s_W[2][kMaxPad / 4][kRowPad];  // W_J = D^-1 A_KJ
  __shared__ __align__(16) float s_D[2][16];                    // D^-1
  const bool own = tid < nbk * nbk;
  const int I = own ? tid / nbk : 0, J = own ? tid % nbk : 0;
  float A[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      A[r][c] = own ? Sh[(4 * I + r) * np + 4 * J + c] * dsc[4 * I + r] * dsc[4 * J + c] : 0.f;
  // prepare pivot block K: run by every thread of the warps that own row K
  auto prepare = [&](int K) {
    const int pb = K & 1, w0 = (K * nbk) >> 5, w1 = (K * nbk + nbk - 1) >> 5;
    const unsigned nbar = (unsigned)(w1 - w0 + 1) * 32u;
    const bool rowown = own && I == K;
    if (rowown) {
      float4* P4 = reinterpret_cast<float4*>(s_P[pb][J]);
#pragma unroll
      for (int r = 0; r < 4; ++r) P4[r] = make_float4(A[r][0], A[r][1], A[r][2], A[r][3]);
    }
    if (rowown && J == K) {  // D^-1 by the scalar sweep of the 4x4 pivot block
      float D[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) D[r][c] = A[r][c];
      bool dok = true;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float d = D[q][q];
        dok = dok && d > kPivotMin;
        const float inv = __fdividef(1.f, d);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (r != q && c != q) D[r][c] = fmaf(-D[r][q] * inv, D[q][c], D[r][c]);
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r != q) {
            D[r][q] *= inv;
            D[q][r] *= inv;
          }
        D[q][q] = -inv;
      }
      if (!dok) s_ok = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) s_D[pb][4 * r + c] = -D[r][c];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(nbar) : "memory");
    if (rowown) {  // W_J = D^-1 A_KJ
      float Dv[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) Dv[e] = s_D[pb][e];
      float4* W4 = reinterpret_cast<float4*>(s_W[pb][J]);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          w[c] = fmaf(Dv[4 * r], A[0][c], fmaf(Dv[4 * r + 1], A[1][c], fmaf(Dv[4 * r + 2], A[2][c], Dv[4 * r + 3] * A[3][c])));
        W4[r] = make_float4(w[0], w[1], w[2], w[3]);
      }
    }
  };
  const int warp = tid >> 5;
  if (s_ok && warp <= (nbk - 1) >> 5) prepare(0);
  __syncthreads();
  bool ok = s_ok != 0;
  for (int K = 0; K < nbk && ok; ++K) {
    const int pb = K & 1;
    if (own) {
      if (I != K && J != K) {  // A_IJ -= W_I^T P_J
        float W[16], Pj[16];
        const float4* W4 = reinterpret_cast<const float4*>(s_W[pb][I]);
        const float4* P4 = reinterpret_cast<const float4*>(s_P[pb][J]);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 w = W4[r], p = P4[r];
          W[4 * r] = w.x; W[4 * r + 1] = w.y; W[4 * r + 2] = w.z; W[4 * r + 3] = w.w;
          Pj[4 * r] = p.x; Pj[4 * r + 1] = p.y; Pj[4 * r + 2] = p.z; Pj[4 * r + 3] = p.w;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int m = 0; m < 4; ++m) A[r][c] = fmaf(-W[4 * m + r], Pj[4 * m + c], A[r][c]);
      } else if (I != K) {  // J == K: A_IK <- W_I^T
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) A[r][c] = s_W[pb][I][4 * c + r];
      } else if (J != K) {  // I == K: A_KJ <- W_J
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) A[r][c] = s_W[pb][J][4 * r + c];
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) A[r][c] = -s_D[pb][4 * r + c];
      }
    }
    if (K + 1 < nbk && warp >= ((K + 1) * nbk) >> 5 && warp <= ((K + 1) * nbk + nbk - 1) >> 5) prepare(K + 1);
    __syncthreads();
    ok = s_ok != 0;
  }
  if (ok && own)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) Ai[(4 * I + r) * np + 4 * J + c] = -A[r][c];
  __syncthreads();
  // x = D A^-1 D (b - S x), refined with double-float residuals; eight
  // threads per row
  constexpr int kTpr = kSolveThreads / 128;
  const int row = tid / kTpr, q = tid % kTpr;
  for (int pass = 0; pass < kRefine && ok; ++pass) {
    float s = 0.f, c = 0.f;
    if (row < n) {
      if (q == 0) {
        s = rh[row];
        c = rl[row];
      }
      if (pass > 0)
        for (int j = q; j < n; j += kTpr) {
          const float sh = Sh[row * np + j], sl = Sl[row * np + j], x0 = xh[j], x1 = xl[j];
          const float p = sh * x0;
          const float pe = fmaf(sh, x0, -p);  // exact error of the product
          df_add(s, c, -p);
          c -= pe + fmaf(sh, x1, sl * x0);
        }
    }
#pragma unroll
    for (int off = 1; off < kTpr; off <<= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
      const float c2 = __shfl_xor_sync(0xffffffffu, c, off);
      df_add(s, c, s2);
      c += c2;
    }
    if (q == 0 && row < np) tmp[row] = row < n ? (s + c) * dsc[row] : 0.f;
    __syncthreads();
    float y = 0.f;
    if (row < np)
      for (int j = q; j < np; j += kTpr) y = fmaf(Ai[row * np + j], tmp[j], y);
#pragma unroll
    for (int off = 1; off < kTpr; off <<= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
    if (q == 0 && row < n) {
      float h = xh[row], l = xl[row];
      df_add(h, l, y * dsc[row]);
      const float hi = h + l;
      xh[row] = hi;
      xl[row] = l - (hi - h);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) st->dc[i] = ok ? xh[i] + xl[i] : 0.f;
  // candidate keyframes and focal
  for (int k = tid; k < a.N; k += nt) {
    const float* T = a.poses + 12 * k;
    float* C = st->pose_cand + 12 * k;
    const int fi = a.free_of[k];
    if (fi < 0 || !ok) {
      for (int e = 0; e < 12; ++e) C[e] = T[e];
      continue;
    }
    const int o = 6 * fi;
    float E[9];
    exp_so3(xh[o] + xl[o], xh[o + 1] + xl[o + 1], xh[o + 2] + xl[o + 2], E);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int cidx = 0; cidx < 3; ++cidx)
        C[4 * r + cidx] = fmaf(E[3 * r], T[cidx], fmaf(E[3 * r + 1], T[4 + cidx], E[3 * r + 2] * T[8 + cidx]));
      C[4 * r + 3] = T[4 * r + 3] + (xh[o + 3 + r] + xl[o + 3 + r]);
    }
  }
  if (tid == 0) {
    st->f_cand = (ok && a.opt_focal) ? *a.focal + (xh[fidx] + xl[fidx]) : *a.focal;
    st->solve_ok = ok ? 1 : 0;
    if (!ok) atomicOr(a.status, GS_BA_SOLVE_FAILED);
  }
}

template <int G>
__global__ void __launch_bounds__(256) k_ba_candidate(const BaArgs a) {
  __shared__ float sh[8][2];
  __shared__ float s_dc[kMaxPad];
  __shared__ bool s_last;
  BaState* st = a.st;
  const int gl = threadIdx.x & (G - 1);
  const int l = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
  const bool live = l < a.P;
  const bool ok = st->solve_ok != 0;
  for (int i = threadIdx.x; i < a.dim; i += blockDim.x) s_dc[i] = st->dc[i];
  __syncthreads();
  float cs = 0.f, cc = 0.f;
  if (ok) {
    const int k = (live && gl < a.M) ? (int)a.obs[(size_t)l * a.M + gl] : -1;
    const int fi = k >= 0 ? a.free_of[k] : -1;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;  // Z^T dc of this observation
    if (fi >= 0) {
      const float* z = a.zrec + ((size_t)l * a.M + gl) * kZ;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float d = s_dc[6 * fi + i];
        t0 = fmaf(z[3 * i], d, t0);
        t1 = fmaf(z[3 * i + 1], d, t1);
        t2 = fmaf(z[3 * i + 2], d, t2);
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, off);
      t1 += __shfl_xor_sync(0xffffffffu, t1, off);
      t2 += __shfl_xor_sync(0xffffffffu, t2, off);
    }
    float X0 = 0.f, X1 = 0.f, X2 = 0.f;
    if (live) {
      const float* Lr = a.lrec + (size_t)l * kLR;
      const float df = a.opt_focal ? s_dc[6 * a.n_free] : 0.f;
      const float u0 = Lr[6] + fmaf(Lr[9], df, t0);
      const float u1 = Lr[7] + fmaf(Lr[10], df, t1);
      const float u2 = Lr[8] + fmaf(Lr[11], df, t2);
      // dX = -L^-T u
      X0 = a.points[3 * l] - fmaf(Lr[0], u0, fmaf(Lr[1], u1, Lr[3] * u2));
      X1 = a.points[3 * l + 1] - fmaf(Lr[2], u1, Lr[4] * u2);
      X2 = a.points[3 * l + 2] - Lr[5] * u2;
      if (gl == 0) {
        a.xcand[3 * l] = X0;
        a.xcand[3 * l + 1] = X1;
        a.xcand[3 * l + 2] = X2;
      }
    }
    float e = 0.f;
    if (k >= 0) {
      const float* T = st->pose_cand + 12 * k;
      const float x = fmaf(T[0], X0, fmaf(T[1], X1, T[2] * X2)) + T[3];
      const float y = fmaf(T[4], X0, fmaf(T[5], X1, T[6] * X2)) + T[7];
      const float z = fmaf(T[8], X0, fmaf(T[9], X1, T[10] * X2)) + T[11];
      if (z > kZmin) {
        const float iz = 1.f / z, f = st->f_cand;
        const float2 o = a.uv[(size_t)l * a.M + gl];
        const float r0 = fmaf(f, x * iz, a.cx) - o.x;
        const float r1 = fmaf(f, y * iz, a.cy) - o.y;
        e = fmaf(r0, r0, r1 * r1);
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (live && gl == 0) cs = e;
  }
  float s1[1] = {cs}, c1[1] = {cc};
  const float2 part = block_sum_df<1>(s1, c1, reinterpret_cast<float(*)[2]>(sh));
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x] = part;
    __threadfence();
    s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // last CTA: candidate cost summed over the CTAs' partials in a fixed order,
  // then the decision and lambda
  __threadfence();
  {
    const volatile float2* pv = a.partials;
    float ps = 0.f, pc = 0.f;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
      const float hx = pv[i].x, hy = pv[i].y;
      df_add(ps, pc, hx);
      pc += hy;
    }
    s1[0] = ps;
    c1[0] = pc;
  }
  __syncthreads();
  const float2 tot = block_sum_df<1>(s1, c1, reinterpret_cast<float(*)[2]>(sh));
  if (threadIdx.x == 0) {
    double Ec = (double)tot.x + (double)tot.y;
    const double E = st->cost;
    if (!ok) Ec = INFINITY;
    const bool acc = ok && Ec < E;
    if (a.trace) {
      double* tr = a.trace + 4 * (size_t)a.iter;
      tr[0] = E;
      tr[1] = Ec;
      tr[2] = st->lam;
      tr[3] = acc ? 1.0 : 0.0;
    }
    st->lam = acc ? st->lam * 0.1 : st->lam * 10.0;
    st->accepted = acc ? 1 : 0;
    st->ticket = 0;
    if (acc && a.opt_focal) *a.focal = st->f_cand;
  }
  __syncthreads();
  if (st->accepted)  // keyframe poses of the accepted candidate (fixed ones are equal)
    for (int e = threadIdx.x; e < 12 * a.N; e += blockDim.x)
      if (a.free_of[e / 12] >= 0) a.poses[e] = st->pose_cand[e];
}

__global__ void __launch_bounds__(256) k_ba_finish(const BaArgs a) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= a.P || !a.st->accepted) return;
  a.points[3 * l] = a.xcand[3 * l];
  a.points[3 * l + 1] = a.xcand[3 * l + 1];
  a.points[3 * l + 2] = a.xcand[3 * l + 2];
}

struct BaLayout {
  size_t st, obs, xcand, zrec, drec, dpos, lrec, lists, counts, bres, bfin, bticket, partials, total;
};

int max_free(int N) { return std::min(N, GS_BA_MAX_FREE); }
int groups_per_landmark(int M) { return M <= 4 ? 4 : M <= 8 ? 8 : 16; }

BaLayout ba_layout(int N, int P, int M) {
  const int fm = max_free(N);
  const size_t nb = (size_t)fm + (size_t)fm * (fm - 1) / 2 + 1;
  const size_t chunks = (size_t)fm * kSplitD + (size_t)fm * (fm - 1) / 2 * kSplitP + kSplitF;
  const size_t blocks = (size_t)P * groups_per_landmark(M) / 256 + 2;
  BaLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.st = take(sizeof(BaState));
  L.obs = take((size_t)P * M);
  L.xcand = take(sizeof(float) * 3 * (size_t)P);
  L.zrec = take(sizeof(float) * kZ * (size_t)P * M);
  L.drec = take(sizeof(float) * kD * (size_t)P * fm);
  L.dpos = take(sizeof(int32_t) * (size_t)P * M);
  L.lrec = take(sizeof(float) * kLR * (size_t)P);
  L.lists = take(sizeof(int32_t) * (nb - 1) * (size_t)P);
  L.counts = take(sizeof(int32_t) * nb);
  L.bres = take(sizeof(float2) * kBR * chunks);
  L.bfin = take(sizeof(float2) * kBR * nb);
  L.bticket = take(sizeof(unsigned) * nb);
  L.partials = take(sizeof(float2) * blocks);
  L.total = o;
  return L;
}

size_t solve_smem(int n) {
  const size_t np = (size_t)((n + 3) & ~3);
  return sizeof(float) * (3 * np * np + 8 * np);
}

template <int G>
gs_status launch_iters(BaArgs& a, int iters, size_t smem, cudaStream_t s) {
  const unsigned lin_grid = (unsigned)std::max<int64_t>(1, ((int64_t)a.P * G + 255) / 256);
  const unsigned nchunks = (unsigned)(a.n_free * kSplitD + a.n_pairs * kSplitP + kSplitF);
  for (int it = 0; it < iters; ++it) {
    a.iter = it;
    k_ba_linearize<G><<<lin_grid, 256, 0, s>>>(a);
    k_ba_reduce<<<nchunks, kRedThreads, 0, s>>>(a);
    k_ba_solve<<<1, kSolveThreads, smem, s>>>(a);
    k_ba_candidate<G><<<lin_grid, 256, 0, s>>>(a);
  }
  return check_launch("bundle adjustment iteration");
}

}  // namespace

size_t ba_workspace_bytes(int N, int P, int M) { return ba_layout(N, P, M).total; }

gs_status launch_ba(const gs_ba_problem& pr, float* poses, float* points, float* focal, int iters, double lambda0,
                    double* trace, uint32_t* status, void* ws, cudaStream_t s) {
  const BaLayout L = ba_layout(pr.num_cams, pr.num_points, pr.obs_per_point);
  unsigned char* w = static_cast<unsigned char*>(ws);
  BaArgs a{};
  a.P = pr.num_points;
  a.M = pr.obs_per_point;
  a.N = pr.num_cams;
  a.opt_focal = pr.opt_focal ? 1 : 0;
  a.cx = pr.cx;
  a.cy = pr.cy;
  int nf = 0;
  for (int k = 0; k < GS_BA_MAX_CAMS; ++k) a.free_of[k] = -1;
  for (int k = 0; k < pr.num_cams; ++k)
    if (!pr.fixed[k]) {
      a.free_of[k] = (int8_t)nf;
      a.cam_of[nf++] = (int8_t)k;
    }
  a.n_free = nf;
  a.dim = 6 * nf + a.opt_focal;
  int p = 0;
  for (int i = 0; i < nf; ++i)
    for (int j = i + 1; j < nf; ++j) {
      a.pa[p] = (uint8_t)i;
      a.pb[p++] = (uint8_t)j;
    }
  a.n_pairs = p;
  a.obs_in = pr.obs_cam;
  a.obs = reinterpret_cast<int8_t*>(w + L.obs);
  a.uv = reinterpret_cast<const float2*>(pr.obs_uv);
  a.poses = poses;
  a.points = points;
  a.focal = focal;
  a.xcand = reinterpret_cast<float*>(w + L.xcand);
  a.zrec = reinterpret_cast<float*>(w + L.zrec);
  a.drec = reinterpret_cast<float*>(w + L.drec);
  a.dpos = reinterpret_cast<int32_t*>(w + L.dpos);
  a.lrec = reinterpret_cast<float*>(w + L.lrec);
  a.lists = reinterpret_cast<int32_t*>(w + L.lists);
  a.counts = reinterpret_cast<int32_t*>(w + L.counts);
  a.bres = reinterpret_cast<float2*>(w + L.bres);
  a.bfin = reinterpret_cast<float2*>(w + L.bfin);
  a.bticket = reinterpret_cast<unsigned*>(w + L.bticket);
  a.partials = reinterpret_cast<float2*>(w + L.partials);
  a.st = reinterpret_cast<BaState*>(w + L.st);
  a.trace = trace;
  a.status = status;

  const size_t smem = solve_smem(a.dim);
  if (cudaFuncSetAttribute(k_ba_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return check_launch("k_ba_solve shared memory");
  k_ba_prepare<<<(unsigned)std::max(1, (a.P + 255) / 256), 256, 0, s>>>(a, lambda0);
  if (nf + a.n_pairs > 0) k_ba_lists<<<(unsigned)(nf + a.n_pairs), 256, 0, s>>>(a);
  gs_status st;
  switch (groups_per_landmark(a.M)) {
    case 4: st = launch_iters<4>(a, iters, smem, s); break;
    case 8: st = launch_iters<8>(a, iters, smem, s); break;
    default: st = launch_iters<16>(a, iters, smem, s); break;
  }
  if (st != GS_OK) return st;
  k_ba_finish<<<(unsigned)std::max(1, (a.P + 255) / 256), 256, 0, s>>>(a);
  return check_launch("k_ba_finish");
}

}  // namespace gs
