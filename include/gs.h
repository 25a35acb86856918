/*
 * gs.h -- C ABI of the B300 differentiable 3D Gaussian-splat rasterizer.
 *
 * The operation is the renderer that the paper's joint optimisation runs every
 * iteration (Sec. 5.2: the Gaussian model is trained for 30 iterations per
 * keyframe with a custom differentiable splat renderer, render -> loss ->
 * optimise), split into the calls a training step makes:
 *
 *   gs_project     EWA projection + SH colour of every (view, Gaussian)
 *   gs_bin_sort    per-tile duplication and (tile, depth) sort, tile ranges
 *   gs_render_fwd  front-to-back alpha compositing per tile
 *   gs_render_bwd  analytic backward to all parameters and the camera poses
 *   gs_render_fused  composite + image loss + per-pixel backward of a
 *                  training step in one persistent launch over all views'
 *                  tiles (then gs_render_bwd_gaussians)
 *   gs_adam_step   fused Adam over the parameter arena (+ optional pose step)
 *
 * The primitive (Sec. 7: position, opacity, rotation, scale, SH coefficients)
 * and the renderer's fixed rules are those of the standard 3DGS rasterizer:
 * 2D covariance dilated by 0.3 px^2, alpha = min(0.99, o exp(power)), splats
 * with alpha < 1/255 skipped, compositing stopped before the splat that would
 * bring transmittance below 1e-4.  Readings where the paper is silent:
 *   - OpenCV camera axes; pose = world->camera [R | t]; centre = -R^T t;
 *   - pixel (u,v) has centre (u+1/2, v+1/2), principal point in the same units;
 *   - culled when t_z <= znear;
 *   - support half-width r = ceil(3 sqrt(lambda_max)); a splat touches a pixel
 *     only when the pixel centre lies in [m-r, m+r]^2, so the image does not
 *     depend on the tile shape;
 *   - real SH without Condon-Shortley phase, k = l^2 + l + m,
 *     rgb = max(0, sum_k c_k Y_k(dir) + 1/2), dir from the camera centre;
 *   - quaternion (w,x,y,z), normalised inside the forward;
 *   - pose gradient for the left perturbation T <- Exp(xi) T, xi = (v, omega);
 *   - equal (tile, depth) keys keep Gaussian-id order.
 *
 * Conventions for every call:
 *   - Pointers named *_dev or documented as device memory are device pointers
 *     owned by the caller; the library never frees them.  Host pointers are
 *     read during the call only.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream); no call synchronises the stream.
 *   - A call returns GS_OK once its kernels are enqueued.  Argument errors
 *     return GS_ERR_INVALID and enqueue nothing; a failing CUDA call returns
 *     GS_ERR_CUDA.  gs_last_error() gives the message of the calling thread's
 *     last failure.
 *   - Conditions only the device can see (pair capacity exceeded, non-finite
 *     gradient) are recorded in the caller's status words (gs_bins.counts and
 *     gs_adam_cfg.status), read by the caller after the stream completes.
 *   - Float arithmetic is IEEE single precision except where stated.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

typedef int gs_status;
#define GS_OK 0
#define GS_ERR_INVALID 1  /* bad argument: nothing was enqueued */
#define GS_ERR_OOM 2      /* workspace smaller than the size query returned */
#define GS_ERR_CUDA 3     /* a CUDA runtime call failed */
#define GS_ERR_TIMEOUT 4  /* a bounded device wait expired */
#define GS_ERR_NONFINITE 5
#define GS_ERR_BUSY 6

#define GS_MAX_VIEWS 64   /* views per call */
#define GS_TILE 16        /* default tile edge in pixels (16x16 tiles) */

typedef void* gs_stream;  /* cudaStream_t */

/* Gaussian parameters, device memory, structure of arrays:
 *   means4    [n][4]  x, y, z, (ignored)
 *   scale_opa [n][4]  log-scale x, y, z, opacity logit (opacity = sigmoid)
 *   quat      [n][4]  w, x, y, z (any non-zero norm; normalised inside)
 *   sh        [3*nc][n] planar: plane (channel*nc + k) holds coefficient k of
 *             that colour channel for every Gaussian; nc = (sh_degree+1)^2
 * sh_stride: distance in floats between consecutive SH planes (0 means n;
 * a larger stride lets a capacity-sized arena hold a growing scene).
 * All four base pointers must be 16-byte aligned. */
typedef struct {
  const float* means4;
  const float* scale_opa;
  const float* quat;
  const float* sh;
  int64_t n;
  int32_t sh_degree; /* 0..3 */
  int64_t sh_stride;
} gs_params;

/* Gradients in exactly the layout of gs_params (the ignored 4th component of
 * means4 receives 0). */
typedef struct {
  float* means4;
  float* scale_opa;
  float* quat;
  float* sh;
  int64_t n;
  int32_t sh_degree;
  int64_t sh_stride;
} gs_grads;

/* Intrinsics and image size of one view, host memory. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t width, height;
} gs_camera;

typedef struct {
  int32_t tile_w, tile_h; /* tile shape in pixels: 16x16, 32x8 or 8x32 (every
                             shape has 256 pixels; the image does not depend
                             on it, gradients only through rounding order) */
  float bg[3];            /* background colour behind the last splat */
  float znear;            /* near plane (> 0) */
  int32_t clamp_jacobian; /* 1: guard t_x/t_z, t_y/t_z at +-1.3 (W/2)/fx, (H/2)/fy */
  uint32_t schedule;      /* GS_SCHED_* bits (0 = defaults); set by the autotuners */
} gs_raster_cfg;

/* Schedule of the blend kernels (no effect on any result):
 *   GS_SCHED_FWD_LONGEST_FIRST / GS_SCHED_BWD_LONGEST_FIRST: the composite /
 *     backward takes the tiles in gs_bins.tile_order (longest lists first);
 *   GS_SCHED_FWD_BATCH(b): splats staged in shared memory per batch by the
 *     composite, b = 0: 128, 1: 64, 2: 256;
 *   GS_SCHED_BWD_BATCH(b): the same for the single-pass backward, 0: 128, 1: 64;
 *   GS_SCHED_FUSED_LONGEST_FIRST: gs_render_fused hands out its (view, tile)
 *     items in gs_bins.tile_order (longest lists of all views first) instead
 *     of view-major order;
 *   GS_SCHED_FUSED_BATCH(b): splats per batch of gs_render_fused, 0: 128, 1: 64,
 *     2: 32. */
#define GS_SCHED_FWD_LONGEST_FIRST 0x1u
#define GS_SCHED_BWD_LONGEST_FIRST 0x2u
#define GS_SCHED_FUSED_LONGEST_FIRST 0x4u
#define GS_SCHED_FWD_BATCH(b) ((uint32_t)(b) << 4)
#define GS_SCHED_BWD_BATCH(b) ((uint32_t)(b) << 8)
#define GS_SCHED_FUSED_BATCH(b) ((uint32_t)(b) << 12)

/* Projected splats of V views, device memory, each array [V][n] (view-major):
 *   xy       float4  m = (x_int + x_frac, y_int + y_frac): the pixel-space
 *                    mean split into an integer part and a fraction in [0,1),
 *                    computed in double-single arithmetic so that it is
 *                    accurate to ~1e-6 px at any image size
 *   conic    float4  A, B, C of the inverse 2D covariance, opacity
 *   rgb      float4  r, g, b, support half-width r (integer valued)
 *   depth    float   camera-space z, correctly rounded (the sort key)
 *   rect     uint2   (x_lo | y_lo << 16, x_hi | y_hi << 16): inclusive tiles
 *   touched  uint32  tiles in rect; 0 = culled
 *   aux      uint32  bits 0-2: rgb channel clamped at 0; bit 3/4: Jacobian
 *                    guard active in x/y
 * Size in bytes of all arrays together: gs_splats_bytes(). */
typedef struct {
  float* xy;
  float* conic;
  float* rgb;
  float* depth;
  uint32_t* rect;
  uint32_t* touched;
  uint32_t* aux;
  int64_t n;
  int32_t views;
} gs_splats;

/* Sorted tile lists, device memory:
 *   vals      [capacity] Gaussian id of each (tile, Gaussian) pair, ordered by
 *             (global tile, depth, Gaussian id)
 *   ranges    [num_tiles][2] [start, end) of each global tile in vals; global
 *             tile = sum of the tile counts of earlier views + ty*TX + tx
 *   pair_off  [V][n] position of the first pair of each (view, Gaussian) in
 *             emission order (pairs of one Gaussian are contiguous there)
 *   keys      optional [capacity] (global tile << 32 | depth bits), sorted;
 *             NULL = not written
 *   counts    [4] status words written by the device: [0] visible
 *             (view, Gaussian) items, [1] pairs K, [2] status bits: 1 = K >
 *             capacity (the lists are then truncated and must not be
 *             rendered), 2 = an index read from an earlier stage was out of
 *             range and its access was skipped (an internal error), [3]
 *             min(K, capacity)
 *   tile_order optional [num_tiles]: written by gs_bin_sort, the tiles
 *             ordered by decreasing list length (bucketed by powers of two;
 *             empty tiles last); the composite and backward kernels then
 *             take the longest lists first, so the long ones do not trail at
 *             the end of the grid.  The order within a bucket is not fixed;
 *             every output is independent of it.  NULL = natural order. */
typedef struct {
  uint32_t* vals;
  uint32_t* ranges;
  uint32_t* pair_off;
  uint64_t* keys;
  uint32_t* counts;
  int64_t capacity;
  int64_t num_tiles;
  uint32_t* tile_order;
} gs_bins;

/* One Adam parameter group: elements [begin, end) of the arena; element e
 * uses learning rate lr[(e - begin) & 3] (so one float4 group can give its
 * four lanes different rates, e.g. log-scales and the opacity logit).  Groups
 * must not overlap. */
typedef struct {
  int64_t begin, end;
  float lr[4];
} gs_adam_group;

#define GS_MAX_ADAM_GROUPS 64

typedef struct {
  const gs_adam_group* groups; /* host array */
  int32_t num_groups;          /* 1..GS_MAX_ADAM_GROUPS */
  float beta1, beta2, eps;
  uint32_t* status;            /* optional device word: set to 1 when a
                                  non-finite gradient or moment is met */
  /* optional pose step (pose == NULL: skipped): Adam on the twist xi of each
   * view, then pose <- Exp(xi) pose */
  float* pose;                 /* [V][12] device, [R | t] row-major */
  const float* dpose;          /* [V][6] device, (v, omega) */
  float* pose_m;               /* [V][6] device */
  float* pose_v;               /* [V][6] device */
  int32_t views;
  float pose_lr;
  int32_t pose_step;           /* bias-correction step of the pose moments
                                  (0 = the parameters' step) */
  /* optional device step counters, for replaying a captured step: when
   * step_dev is set, the `step` argument is ignored, the update uses
   * *step_dev + 1 and then increments *step_dev; when pose_steps_dev ([V])
   * is set, view v's pose update uses pose_steps_dev[v] + 1 and increments it. */
  int32_t* step_dev;
  int32_t* pose_steps_dev;
  /* optional device word: when nonzero at run time the whole update (and the
   * step counters) is skipped, e.g. the bins status of the step, so a step
   * whose tile lists overflowed leaves the optimiser state untouched */
  const uint32_t* skip_dev;
} gs_adam_cfg;

/* ---------------------------------------------------------------------- */

/* Message of the calling thread's last failing call ("" if none).  Copies at
 * most len-1 bytes and a terminating NUL into buf; returns the full length. */
GS_API size_t gs_last_error(char* buf, size_t len);

/* Library version and the compute capability it was built for. */
GS_API int32_t gs_version(void);
GS_API int32_t gs_built_arch(void);

/* Bytes of the gs_splats arrays for n Gaussians and V views, laid out by
 * gs_splats_carve in one allocation (every array 256-byte aligned). */
GS_API size_t gs_splats_bytes(int64_t n, int32_t views);
/* Fill `out` with pointers into `base` (device, >= gs_splats_bytes, 256-byte
 * aligned). */
GS_API gs_status gs_splats_carve(void* base, int64_t n, int32_t views, gs_splats* out);

/* EWA projection (Sec. 5.2's renderer, per-Gaussian stage) of n Gaussians into
 * V views.  poses_dev [V][12] device ([R | t], world->camera); cams host [V].
 * Per (view, Gaussian): t = R mu + t_cam (double-single); culled if
 * t_z <= znear; Sigma = Rq diag(e^{2s}) Rq^T; 2D covariance
 * J R Sigma R^T J^T + 0.3 I; conic = its inverse; r = ceil(3 sqrt(lambda_max));
 * colour from SH at dir = normalise(mu - centre).  Tile rect: per axis the
 * tiles of [m - h, m + h], where h = min(r, the half-width of the bounding
 * box of the ellipse A dx^2 + 2B dx dy + C dy^2 <= 2 ln(255 opacity) on which
 * alpha can reach 1/255, widened by 0.1% + 0.05 px); a splat with
 * opacity <= 1/255 is culled.  Every pixel that can blend the splat lies in
 * a tile of its rect, so the image equals that of the [m-r, m+r]^2 rect.
 * Writes every field of `out` for every (view, Gaussian). */
GS_API gs_status gs_project(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                     int32_t views, const gs_raster_cfg* cfg, gs_splats* out, gs_stream stream);

/* Loop-closure update (Sec. 5.5: every Gaussian keeps the keyframe that
 * added it and receives the Sim(3) correction of that keyframe, with scale
 * and rotation updated accordingly).  For Gaussian i with k = kf_dev[i] >= 0
 * and the correction sim3_dev[k] = (qw, qx, qy, qz, tx, ty, tz, s) (rotation
 * as a quaternion of any non-zero norm, s > 0):
 *   mean' = s R mean + t;  log-scales' = log-scales + log s;
 *   quaternion' = q_S q (Hamilton product; the input's norm is kept).
 * Opacity and SH are unchanged (the paper updates scale and rotation; the SH
 * coefficients are not rotated), and so are the Adam moments.  kf_dev < 0:
 * not moved; kf_dev >= num_kf: not moved and bit 0 of *status_dev set.
 * params: writable parameter arrays (gs_params layout), n Gaussians; kf_dev
 * int32 [n], sim3_dev float [num_kf][8], status_dev uint32: device. */
GS_API gs_status gs_sim3_update(gs_grads* params, const int32_t* kf_dev, const float* sim3_dev, int32_t num_kf,
                                uint32_t* status_dev, gs_stream stream);

/* Leaf Gaussians per keyframe (Sec. 6.2: keyframes are sampled for
 * optimisation in proportion to the active leaves they generated):
 * counts_dev[k] = #{i < n : kf_dev[i] == k} for k < num_kf; other ids are not
 * counted.  counts_dev: device uint32 [num_kf], overwritten. */
GS_API gs_status gs_keyframe_counts(const int32_t* kf_dev, int64_t n, int32_t num_kf, uint32_t* counts_dev,
                                    gs_stream stream);

/* ---------------------------------------------------------------------------
 * Local bundle adjustment (Sec. 5.1 "Local Bundle Adjustment" and the
 * supplementary "Fast Bundle Adjustment"): N keyframes, n_f of them fixed, K
 * landmarks, each observed by a fixed subset of at most M keyframes, the
 * shared focal length optimised; per-observation residual/Jacobian kernels and
 * a dense Schur complement over the free keyframes.
 *
 * Readings where the paper is silent: pinhole u = f x/z + cx, v = f y/z + cy
 * with (x, y, z) = R X + t (pose world->camera, row-major [R | t]); residual in
 * pixels, cost = sum of squared residuals, no robust kernel; an observation
 * with z <= 1e-6 contributes nothing.  Update R <- Exp(dtheta) R, t <- t + dt,
 * X <- X + dX, f <- f + df.  Levenberg-Marquardt with Marquardt's scaling:
 * (H + lambda D) delta = -g, D = diag(H) clamped to [1e-6, 1e32]; a candidate
 * with a lower cost is accepted and lambda /= 10, otherwise lambda *= 10.
 * One iteration = one linearisation, one damped solve, one decision; the
 * iteration count is fixed.
 *
 * Precision: residuals, Jacobians and per-observation Schur terms in float32;
 * sums over observations in double-float (float32 value + error term), the
 * reduced camera system in float64 with Jacobi scaling, factorised in float32
 * and refined with float64 residuals; each landmark's 3x3 block factorised in
 * float64.
 * --------------------------------------------------------------------------- */
#define GS_BA_MAX_CAMS 64   /* keyframes per problem */
#define GS_BA_MAX_FREE 20   /* keyframes that are optimised */
#define GS_BA_MAX_OBS 16    /* observation slots per landmark */
/* status bits (device word, OR-ed) */
#define GS_BA_BAD_OBS 0x1u        /* a slot named a keyframe out of range or twice: slot ignored */
#define GS_BA_SOLVE_FAILED 0x2u   /* a reduced system was not positive definite: step rejected */
#define GS_BA_DEGENERATE 0x4u     /* a landmark's damped 3x3 block was not positive definite: landmark kept */

typedef struct gs_ba_problem {
  int32_t num_cams;       /* N, 1..GS_BA_MAX_CAMS */
  int32_t num_points;     /* K >= 0 */
  int32_t obs_per_point;  /* M, 1..GS_BA_MAX_OBS */
  int32_t opt_focal;      /* 1: the shared focal length is optimised, 0: kept */
  float cx, cy;           /* principal point, fixed */
  const int32_t* obs_cam; /* device int32 [K][M]: keyframe of each slot, -1 = empty */
  const float* obs_uv;    /* device float32 [K][M][2]: observed pixel position */
  uint8_t fixed[GS_BA_MAX_CAMS]; /* host flags: 1 = keyframe fixed (not optimised) */
} gs_ba_problem;

/* Workspace bytes of gs_ba_solve for a problem of this size. */
GS_API size_t gs_ba_workspace_bytes(int32_t num_cams, int32_t num_points, int32_t obs_per_point);
/* Runs `iters` Levenberg-Marquardt iterations from the given state, starting
 * with lambda = lambda0 (> 0).  poses: device float32 [N][12] (in/out; fixed
 * keyframes are never written), points: device float32 [K][3] (in/out),
 * focal: device float32 [1] (in/out).  trace (optional): device float64
 * [iters][4] = (cost at the current state, candidate cost (+inf when the
 * solve failed), lambda used, 1 if accepted else 0).  status: device uint32,
 * GS_BA_* bits OR-ed in.  No host synchronisation and no allocation: the call
 * can be captured in a CUDA graph.  GS_ERR_INVALID: sizes out of range, more
 * than GS_BA_MAX_FREE free keyframes, NULL arrays, lambda0 not > 0;
 * GS_ERR_OOM: ws_bytes below gs_ba_workspace_bytes. */
GS_API gs_status gs_ba_solve(const gs_ba_problem* prob, float* poses, float* points, float* focal, int32_t iters,
                             double lambda0, double* trace, uint32_t* status, void* ws, size_t ws_bytes,
                             gs_stream stream);

/* Level-of-detail hierarchy (Sec. 6: coarse nodes hold the parameters of a
 * merged group of children; rendering descends from the roots until a node's
 * screen size falls below tau pixels or a leaf is reached).  Three levels:
 * the n_leaf leaves, level 1 (one node per 8 leaves) and level 2 (one node
 * per 8 level-1 nodes).  Readings where the paper is silent or differs: it
 * merges 4 nearest neighbours by a KL criterion; here the leaves are grouped
 * by Morton order of their means (10 bits per axis over their bounding box,
 * quantised in single precision, equal codes in index order), runs of 8
 * consecutive leaves (then of 8 consecutive level-1 nodes) share a parent, and
 * a parent is the moment-matching merge of its children with weights
 * w = opacity: the mixture's mean and covariance, opacity-weighted SH and
 * opacity min(0.99, sum w o / sum w); its rotation and scales are the
 * eigenvectors and square-root eigenvalues of the covariance.
 * Node numbering: leaves [0, n_leaf), level 1 [n_leaf, n_leaf + n1),
 * level 2 after them; gs_lod_nodes(n_leaf) = n_leaf + n1 + n2. */
GS_API int64_t gs_lod_nodes(int64_t n_leaf);
/* Workspace bytes of gs_lod_build. */
GS_API size_t gs_lod_build_workspace(int64_t n_leaf);
/* Builds levels 1 and 2 over the first n_leaf Gaussians of `nodes` (writable
 * parameter arrays in the layout of gs_params, nodes->n >= gs_lod_nodes(n_leaf))
 * and writes the coarse nodes after the leaves.  parent_dev: device int32
 * [gs_lod_nodes(n_leaf)], overwritten: parent node, -1 for level 2.
 * ws: device, >= gs_lod_build_workspace bytes, 256-byte aligned. */
GS_API gs_status gs_lod_build(gs_grads* nodes, int64_t n_leaf, int32_t* parent_dev, void* ws, size_t ws_bytes,
                              gs_stream stream);
/* gs_project over all nodes->n nodes of a hierarchy with the level-of-detail
 * cut of every view applied: a node is projected iff (it is a leaf, index <
 * n_leaf, or its screen size S = f_x * 3 * max scale / t_z is below tau) and
 * every ancestor has S >= tau; S is infinite at or behind the near plane.
 * Other nodes are culled (touched = 0).  The rest of the pipeline
 * (gs_bin_sort, gs_render_fwd) is unchanged. */
GS_API gs_status gs_project_lod(const gs_params* nodes, int64_t n_leaf, const int32_t* parent_dev, float tau,
                                const float* poses_dev, const gs_camera* cams, int32_t views,
                                const gs_raster_cfg* cfg, gs_splats* out, gs_stream stream);

/* ---------------------------------------------------------------------------
 * Progressive hierarchy (Sec. 6.1 "Adaptive Gaussian Merging and Retrieval",
 * Sec. 6.2): an active set of nodes (leaves and merged intermediate nodes)
 * that is a cut of the forest; nodes live in the rows of the parameter arena
 * (gs_grads layout, capacity rows), the first *n_nodes of them in use.
 * Readings where the paper is silent or differs: groups are a candidate and
 * its 3 nearest candidates (the paper's 4 closest), found exactly within
 * chunks of 64 candidates consecutive in Morton order (its fast KNN); the
 * KL-divergence merge is read as the moment-matching merge of
 * gs_lod_build; a node is in view when t_z > znear and its projected centre
 * lies within the image widened by its screen size.
 * --------------------------------------------------------------------------- */
typedef struct {
  int32_t* parent;    /* [capacity] parent node, -1 = root; -2 marks a row that holds no node yet
                         (an unused slot below n_nodes: never drawn, never merged) */
  int32_t* child;     /* [capacity][4] child nodes, -1 = none */
  uint8_t* active;    /* [capacity] 1 = in the active set */
  uint32_t* n_nodes;  /* device word: arena rows in use (new nodes are appended) */
  uint32_t* info;     /* optional device [8]: analyse: n_nodes, triggered, candidates, active,
                         pulled parents, new groups, grouped candidates, status (1 = no room);
                         refine: [0] = nodes replaced by their children */
  int64_t capacity;   /* rows of the arena and of the arrays above */
} gs_hier;

/* Workspace bytes of gs_hier_analyze / gs_hier_refine. */
GS_API size_t gs_hier_workspace(int64_t capacity);
/* One analysis from a keyframe's camera (pose_dev: device float [12]
 * world->camera, cam: host).  Screen size S = f_x 3 max scale / t_z of every
 * active node (+inf at or behind znear); candidates S < tau_l (the paper's
 * 0.5 px).  Only when more than 20% of the active nodes are candidates:
 * inactive parents whose children are all candidates are pulled (active
 * again, children inactive); the remaining candidates without a parent are
 * grouped with their 3 nearest candidates (Morton order of their means, 10
 * bits per axis over their bounding box, stable; chunks of 64; squared
 * single-precision distances, ties by Morton position; greedy in Morton
 * order, a candidate left alone stays ungrouped) and every group of 2-4
 * becomes a new active node (moment-matching merge of its children, numbered
 * after the existing nodes in Morton order of its first child) with its
 * children inactive.  adam_m / adam_v (optional, gs_grads layout): the Adam
 * moments of the arena, zeroed for every node whose active flag changes.  No
 * host synchronisation; when the new nodes would not fit the capacity
 * nothing is merged and info[7] bit 0 is set. */
GS_API gs_status gs_hier_analyze(gs_grads* nodes, gs_hier* h, const gs_grads* adam_m, const gs_grads* adam_v,
                                 const float* pose_dev, const gs_camera* cam, float znear, float tau_l, void* ws,
                                 size_t ws_bytes, gs_stream stream);
/* Reload (Sec. 6.1, tau_h = 1 px in the paper): up to `passes` passes; in each,
 * every active node with children that is in view with S > tau_h (state
 * before the pass) is replaced by its children.  Passes after one that
 * changed nothing do nothing. */
GS_API gs_status gs_hier_refine(gs_grads* nodes, gs_hier* h, const gs_grads* adam_m, const gs_grads* adam_v,
                                const float* pose_dev, const gs_camera* cam, float znear, float tau_h,
                                int32_t passes, void* ws, size_t ws_bytes, gs_stream stream);
/* gs_project over the first nodes->n rows with each view's cut of the
 * hierarchy: a node is projected iff it belongs to the active set refined for
 * that view (the reload applied without changing the state): an active node
 * that is not expandable (no children, not in view, or S <= tau_h), or an
 * inactive one that is not expandable and whose path up to its first active
 * ancestor consists of expandable nodes.  Other nodes are culled. */
GS_API gs_status gs_project_hier(const gs_params* nodes, const gs_hier* h, float tau_h, const float* poses_dev,
                                 const gs_camera* cams, int32_t views, const gs_raster_cfg* cfg, gs_splats* out,
                                 gs_stream stream);
/* gs_project over the first nodes->n rows with each view's render cut of the
 * stored hierarchy (Sec. 6.2): starting at the roots (parent -1), the descent
 * goes on through every node that has children and is coarser than tau
 * (S > tau; S = +inf at or behind the near plane), and stops at the others,
 * which are projected: node i is projected iff it does not descend and every
 * ancestor does.  The active set is not read (h->active may be NULL); rows
 * >= *h->n_nodes are culled. */
GS_API gs_status gs_project_hier_render(const gs_params* nodes, const gs_hier* h, float tau,
                                        const float* poses_dev, const gs_camera* cams, int32_t views,
                                        const gs_raster_cfg* cfg, gs_splats* out, gs_stream stream);

/* Workspace bytes of gs_bin_sort. */
GS_API size_t gs_bin_sort_workspace(int64_t n, int32_t views, int64_t capacity);

/* Tile binning: every visible (view, Gaussian) emits one pair per tile of its
 * rect; pairs are sorted by (global tile, depth bits) with equal keys in
 * Gaussian-id order, and each tile's [start, end) range is written.  The sort
 * is a counting sort by tile (each pair takes a place in its tile list with
 * one atomic; a scan over the tiles gives the list starts) followed by a sort
 * of every tile's own (depth bits, id) keys by one warp (in registers, below
 * 256 pairs) or CTA (in shared memory up to 4096 pairs, else by a CTA-wide
 * stable radix sort); the keys of one tile
 * are distinct, so the result does not depend on the atomics' order.  At most
 * 2^25 tiles over all views.  No host synchronisation: K stays on the device
 * (counts).  ws: device, >= gs_bin_sort_workspace bytes, 256-byte aligned. */
GS_API gs_status gs_bin_sort(const gs_splats* splats, const gs_camera* cams, int32_t views,
                      const gs_raster_cfg* cfg, gs_bins* out, void* ws, size_t ws_bytes,
                      gs_stream stream);

/* Bytes of the static scratch behind gs_bin_sort_noalloc: enough for, e.g.,
 * n * views <= 65536 items with capacity <= 262144 pairs.  The library also
 * exports the value as the data symbol gs_noalloc_scratch_bytes. */
#define GS_NOALLOC_SCRATCH_BYTES (8u << 20)
GS_API extern const uint64_t gs_noalloc_scratch_bytes;

/* gs_bin_sort without a workspace argument and without allocating anything
 * (no cudaMalloc / cudaFree, no allocating library).  The paper has no
 * counterpart: this entry point serves callers that cannot allocate device
 * memory (a C host whose device buffers come from an owner's pool, a
 * latency-critical thread where an allocation may synchronise the device, a
 * caller held to a fixed memory budget).  The workspace is one file-scope
 * device array of GS_NOALLOC_SCRATCH_BYTES inside libgs; its device address
 * is looked up (cudaGetSymbolAddress, with that device current) on every
 * call made outside stream capture, so a cudaDeviceReset between calls
 * leaves no stale address; a call made while its stream is capturing uses
 * the address found by an earlier call on the device (GS_ERR_INVALID when
 * there was none).  Results are identical to gs_bin_sort's.
 * Errors: GS_ERR_OOM (with a message) when gs_bin_sort_workspace(n, views,
 * capacity) exceeds the scratch; gs_bin_sort's own checks otherwise.
 * Nothing in the scratch has to start at zero (the call writes every word it
 * reads).  All calls on a device share the one scratch: two calls whose
 * device work overlaps (different streams, or host threads without
 * ordering) race on it and give wrong results, so order them on one stream.
 * Because the lookup cannot run under capture, make the first call on a
 * device before any stream capture. */
GS_API gs_status gs_bin_sort_noalloc(const gs_splats* splats, const gs_camera* cams, int32_t views,
                                     const gs_raster_cfg* cfg, gs_bins* out, gs_stream stream);

/* Forward compositing, one CTA per tile: per pixel, splats in list
 * order; skip when the centre is outside [m-r, m+r]^2, power > 0 or
 * alpha < 1/255; stop before a splat that would make T < 1e-4;
 * C += rgb alpha T; image = C + T bg.
 * image: device, views concatenated, each [3][H][W]; alpha (optional):
 * device, each [H][W], 1 - final transmittance. */
GS_API gs_status gs_render_fwd(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                        int32_t views, const gs_raster_cfg* cfg, float* image, float* alpha,
                        gs_stream stream);

/* Workspace bytes of gs_render_bwd. */
GS_API size_t gs_render_bwd_workspace(int64_t n, int32_t views, int64_t capacity);

/* Backward of gs_project + gs_render_fwd for the loss gradients dL_dimage
 * (layout of image) and optional dL_dalpha (layout of alpha).  image
 * (optional, device, layout of gs_render_fwd's image) is the forward's output
 * for these very splats and tile lists.  When image is given and dL_dalpha is
 * NULL, one front-to-back pass per tile repeats the forward's decisions and
 * takes the colour behind each splat as image minus the colour composited so
 * far (dC/dalpha_i of the front-to-back composite needs only that and T_i).
 * Otherwise the forward
 * pass is replayed to recover the final transmittance and the last blended
 * splat (no per-pixel state is stored), then splats are walked back to front
 * recovering T_i = T_{i+1} / (1 - alpha_i).  The two forms agree to rounding
 * (they take the same decisions).  Per (tile, splat) the
 * gradients of m, conic, opacity and rgb are reduced over the tile's pixels by
 * warp shuffles and shared memory (no global atomics) and stored per pair;
 * a per-Gaussian pass sums its pairs in a fixed order and applies the chain
 * rule to every parameter and the camera pose.  Deterministic: equal inputs
 * give bit-identical outputs.  grads: overwritten (all n Gaussians).
 * dL_dpose (optional): [V][6] device, (v, omega), overwritten. */
GS_API gs_status gs_render_bwd(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                        int32_t views, const gs_splats* splats, const gs_bins* bins,
                        const gs_raster_cfg* cfg, const float* dL_dimage, const float* dL_dalpha,
                        const float* image, gs_grads* grads, float* dL_dpose, void* ws,
                        size_t ws_bytes, gs_stream stream);

/* The two halves of gs_render_bwd, for callers that time or overlap them:
 * gs_render_bwd_pixels runs the per-tile pass and leaves the per-pair
 * gradients in ws; gs_render_bwd_gaussians then applies the per-Gaussian
 * pass.  Calling them in this order with the same arguments is exactly
 * gs_render_bwd. */
GS_API gs_status gs_render_bwd_pixels(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                                      int32_t views, const gs_raster_cfg* cfg, const float* dL_dimage,
                                      const float* dL_dalpha, const float* image, int64_t n, void* ws,
                                      size_t ws_bytes, gs_stream stream);
GS_API gs_status gs_render_bwd_gaussians(const gs_params* params, const float* poses_dev,
                                         const gs_camera* cams, int32_t views, const gs_splats* splats,
                                         const gs_bins* bins, const gs_raster_cfg* cfg, gs_grads* grads,
                                         float* dL_dpose, void* ws, size_t ws_bytes, gs_stream stream);

/* Adam settings of gs_render_bwd_gaussians_adam: one learning rate per lane
 * of the float4 parameters and per SH plane (ch * nc + k), the betas and
 * epsilon of gs_adam_cfg; the step: *step_dev + 1 when step_dev is not NULL
 * (read, not incremented: a following gs_adam_step with the same step_dev
 * increments it), else `step` (>= 1); skip_dev (optional): nonzero = no
 * update; status (optional): bit 0 set when a gradient or a second moment is
 * not finite.  update_mask: bit 0 means4, bit 1 scale_opa, bit 2 quat, bit 3
 * the SH planes; parameters left out keep their values and moments. */
typedef struct {
  float lr_means4[4], lr_scale_opa[4], lr_quat[4];
  float lr_sh[48];
  float beta1, beta2, eps;
  int32_t step;
  uint32_t update_mask;
  const int32_t* step_dev;
  const uint32_t* skip_dev;
  uint32_t* status;
} gs_adam_params_cfg;

/* gs_render_bwd_gaussians with the Adam update of the parameters fused in
 * (the second half of a training step, Sec. 5.2): the kernel that turns each
 * Gaussian's colour gradients into SH gradients finishes its gradient and
 * applies to every parameter of that Gaussian the element update of
 * gs_adam_step (same arithmetic, same bits), so the SH gradients never reach
 * memory and the update takes no pass of its own.  params: read and
 * written (gs_grads layout of the parameters); m, v: Adam moments, same
 * shape (sh_stride may differ from params'); grads: receives the gradients
 * of means4, scale_opa and quat (its sh planes are not written); dL_dpose as
 * in gs_render_bwd_gaussians (the pose step stays with gs_adam_step, which
 * takes num_groups = 0 for the poses alone).  Equal to
 * gs_render_bwd_gaussians followed by gs_adam_step with one group per
 * parameter kind covering rows [0, n) and the same rates. */
GS_API gs_status gs_render_bwd_gaussians_adam(gs_grads* params, const float* poses_dev, const gs_camera* cams,
                                              int32_t views, const gs_splats* splats, const gs_bins* bins,
                                              const gs_raster_cfg* cfg, gs_grads* grads, gs_grads* adam_m,
                                              gs_grads* adam_v, const gs_adam_params_cfg* adam,
                                              float* dL_dpose, void* ws, size_t ws_bytes, gs_stream stream);

/* Workspace bytes of gs_render_fused: the gs_render_bwd workspace (same
 * layout at its start, so the same buffer then serves
 * gs_render_bwd_gaussians) plus a work counter and one float per tile. */
GS_API size_t gs_render_fused_workspace(int64_t n, int32_t views, int64_t capacity, int64_t num_tiles);

/* The per-pixel half of a training step in one persistent launch (the batched
 * iteration of the joint optimisation, Sec. 5.2: sampled views rendered,
 * compared with their images and back-propagated together).  A grid of as
 * many CTAs as the device holds at once takes (view, tile) items from a
 * device counter, in view-major order or, with GS_SCHED_FUSED_LONGEST_FIRST,
 * in gs_bins.tile_order (longest lists of all views first); per item it
 * composites the tile (as gs_render_fwd), writes image (and alpha when not
 * NULL), takes the image loss of its pixels against target (loss_kind 0:
 * L1, mean |image - target|; 1: mean squared error; the mean over all views'
 * pixels and channels, as gs_image_loss) and runs the single front-to-back
 * backward of gs_render_bwd_pixels with that loss gradient, the composite's
 * colour kept in registers.  No per-pixel state is stored besides the image.
 * The per-pair gradients are left in ws for gs_render_bwd_gaussians (same n,
 * views, bins, ws).  *loss_dev receives the loss; per tile its terms are
 * summed in a fixed order and the tiles in tile order (deterministic; equal
 * to gs_image_loss's value up to summation order).  Items do not wait for
 * one another (each tile's list is complete when the launch starts).
 * image, target: device, layout of gs_render_fwd's image; loss_dev: device
 * float; ws: >= gs_render_fused_workspace(n, views, bins->capacity,
 * bins->num_tiles) bytes, 256-byte aligned. */
GS_API gs_status gs_render_fused(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                                 int32_t views, const gs_raster_cfg* cfg, const float* target, int32_t loss_kind,
                                 float* image, float* alpha, float* loss_dev, int64_t n, void* ws, size_t ws_bytes,
                                 gs_stream stream);

/* Autotuner of the blend schedule: times every composite schedule (tile
 * order natural / longest lists first x 128 / 64 / 256 splats per batch) and
 * every single-pass backward schedule (order x 128 / 64) on the caller's
 * current splats and tile lists, `reps` launches each after one warm-up, and
 * writes the fastest of each into cfg->schedule (other bits unchanged).
 * Longest-first candidates need bins->tile_order.  image: device, the image's
 * size (overwritten; on return it holds the composite of the chosen
 * schedule); dL_dimage: device upstream gradient; ws: the gs_render_bwd
 * workspace (n Gaussians).  times_ms (optional, host, 10 floats): mean time
 * of each candidate, the 6 composite ones first (NaN where skipped).
 * Synchronises on its own events (bounded wait, GS_ERR_TIMEOUT): not for use
 * under stream capture.  Schedules change no result. */
GS_API gs_status gs_autotune_blend(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                                   int32_t views, gs_raster_cfg* cfg, float* image, const float* dL_dimage,
                                   int64_t n, void* ws, size_t ws_bytes, int32_t reps, float* times_ms,
                                   gs_stream stream);

/* Autotuner of the fused pass (the batched iteration's knobs: tile shape,
 * splats per shared-memory batch, work order).  For each tile shape (16x16,
 * 32x8, 8x32) the caller's Gaussians are projected and binned again; each
 * candidate shape x batch (128, 64, 32) x order (view-major, longest lists first
 * when bins->tile_order is given) is timed over `reps` runs of gs_project +
 * gs_bin_sort + gs_render_fused after one warm-up, with CUDA events.  A shape
 * whose lists exceed bins->capacity, whose tiles exceed ranges_tiles (the
 * entries bins->ranges and bins->tile_order hold) or whose workspace exceeds
 * ws_bytes is skipped.  On return cfg holds the fastest tile shape and fused
 * schedule (other schedule bits unchanged), bins->num_tiles that shape's tile
 * count, and splats / bins / image / loss the results of that configuration.
 * times_ms (optional, host, 18 floats): mean time of each candidate in the
 * order shape (16x16, 32x8, 8x32) x batch (128, 64, 32) x order (view-major,
 * longest first); NaN where skipped.  bin_ws: the gs_bin_sort workspace; ws:
 * the gs_render_fused workspace.  Synchronises (bounded waits,
 * GS_ERR_TIMEOUT): not for use under stream capture.  The image does not
 * depend on the choice; gradients only through summation order. */
GS_API gs_status gs_autotune_fused(const gs_params* params, const float* poses_dev, const gs_camera* cams,
                                   int32_t views, gs_raster_cfg* cfg, gs_splats* splats, gs_bins* bins,
                                   int64_t ranges_tiles, void* bin_ws, size_t bin_ws_bytes, const float* target,
                                   int32_t loss_kind, float* image, float* loss_dev, void* ws, size_t ws_bytes,
                                   int32_t reps, float* times_ms, gs_stream stream);

/* Fused Adam over one flat float arena of n elements (parameters p, gradients
 * g, moments m, v; all device, 16-byte aligned), in one launch for all groups
 * (the standard Adam update, bias-corrected):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * Elements outside every group are left unchanged.  step >= 1 (unless
 * cfg->step_dev is set). */
GS_API gs_status gs_adam_step(float* p, const float* g, float* m, float* v, int64_t n,
                       const gs_adam_cfg* cfg, int32_t step, gs_stream stream);

/* Work counts of one forward composite (diagnostics for roofline accounting;
 * no image is written): stats_dev[0] = (pixel, splat) pairs the kernel tests
 * (after its conservative per-warp culling), up to and including the splat
 * that stops a pixel; [1] = pairs blended; [2] = sum over tiles of the
 * backward's reverse-walk length (list positions up to the last blended
 * splat of any pixel of the tile); [3] = sum over tiles of the list length;
 * [4] = pairs the plain per-pixel loop evaluates: for every pixel, the list
 * entries of its tile up to and including the splat that stops it (the whole
 * list when none does).  stats_dev: device, 5 uint64, 8-byte aligned,
 * overwritten. */
GS_API gs_status gs_render_stats(const gs_splats* splats, const gs_bins* bins, const gs_camera* cams,
                                 int32_t views, const gs_raster_cfg* cfg, uint64_t* stats_dev,
                                 gs_stream stream);

/* Image loss of a training step over `count` floats (all views' images):
 * kind 0 = L1, mean |image - target|; kind 1 = mean squared error.  The paper
 * names its rendering loss without defining it; these are the two readings
 * offered.  Writes the loss to *loss_dev (device float) and, if dL_dimage is
 * not NULL, its gradient (same layout as image).  ws: device, >=
 * gs_image_loss_workspace() bytes, 256-byte aligned.  Deterministic. */
GS_API size_t gs_image_loss_workspace(void);
GS_API gs_status gs_image_loss(const float* image, const float* target, int64_t count, int32_t kind,
                               float* dL_dimage, float* loss_dev, void* ws, size_t ws_bytes,
                               gs_stream stream);

/* ------------------------------------------------------------------------
 * Streaming session (the live-capture mode of §5.2: optimisation runs
 * asynchronously while frames keep arriving).  A session owns the Gaussians,
 * their gradients and Adam moments (capacity max_gaussians, SH planes strided
 * by the capacity), and a pool of batch contexts (device buffers for one
 * batch in flight each).  Requests (render or train, one camera each) are
 * queued by gs_session_submit from any thread; a worker thread forms batches
 * of up to max_batch_views requests as soon as a context is free and enqueues
 * each batch without waiting for earlier ones (continuous batching); a
 * completion thread finishes requests as their batch's event fires (bounded
 * wait).  Render views of a batch see the parameters before the batch's
 * update; all train views of a batch share one Adam step over every active
 * Gaussian.  The number of contexts is what the HBM budget admits (at most
 * max_inflight); queued requests wait for a free context.  A batch whose tile
 * lists overflow skips its update on the device, grows its pair capacity
 * within the budget and runs again.
 * Streams: writes of the parameters (train parts, adds, loop closures,
 * hierarchy builds) run in issue order on the session's stream; each batch
 * context renders on its own stream.  A render part waits for the writes
 * issued before it and a write waits for the render parts issued before it,
 * so every render sees exactly the updates submitted ahead of it, while render
 * parts run beside one another and beside the forward and backward of a
 * later train part.  Train parts use gs_render_fused.
 * ------------------------------------------------------------------------ */
typedef struct gs_session gs_session;

#define GS_REQUEST_RENDER 0
#define GS_REQUEST_TRAIN 1
/* gs_request.flags: the train target is page-locked host memory (cudaHostAlloc
   or cudaHostRegister) that the caller leaves allocated and unchanged until
   the request has completed (gs_session_wait, or gs_session_times returning
   GS_OK); the session copies it to the device from there instead of taking a
   copy during submit (a camera frame already written to pinned memory is not
   copied twice) */
#define GS_REQUEST_BORROW_TARGET 1

typedef struct {
  int64_t max_gaussians;     /* device capacity (fixed for the session) */
  int32_t sh_degree;
  int32_t max_batch_views;   /* requests per batch, 1..GS_MAX_VIEWS */
  int32_t max_width, max_height;
  int32_t max_inflight;      /* batch contexts wanted (>= 1) */
  uint64_t hbm_budget_bytes; /* all device memory of the session */
  double pair_factor;        /* initial pair capacity = pair_factor * max_gaussians (0 = 4) */
  gs_raster_cfg raster;
  float lr_means, lr_scale, lr_opacity, lr_quat, lr_sh_dc, lr_sh_rest;
  float beta1, beta2, eps;
  int32_t loss_kind;         /* 0 = L1, 1 = MSE */
  int32_t lod;               /* 1: a progressive hierarchy (gs_session_analyze); renders draw its render
                                cut (descent from the roots), trains each view's cut of the active set */
  float lod_tau;             /* reload / cut threshold in pixels (> 0; the paper's tau_h = tau = 1); merging
                                takes nodes below lod_tau / 2 (the paper's tau_l = 0.5) */
} gs_session_config;

typedef struct {
  int32_t kind;              /* GS_REQUEST_RENDER or GS_REQUEST_TRAIN */
  gs_camera cam;             /* within the session's maximum resolution */
  float pose[12];            /* world->camera [R | t], row-major 3x4 */
  const float* target;       /* train: host [3][H][W], copied during submit (unless borrowed, flags) */
  float* image_out;          /* render: host [3][H][W], filled before the request completes (may be NULL) */
  double arrival_s;          /* arrival time on gs_session_now()'s clock; 0 = submit time */
  int32_t flags;             /* 0 or GS_REQUEST_BORROW_TARGET */
} gs_request;

typedef struct {
  int64_t submitted, completed, failed, queued, inflight;
  int64_t iterations;        /* Adam steps taken (batches with train views) */
  int64_t batches;           /* batches issued, capacity retries included */
  int64_t retries;           /* batch parts issued again after a pair-capacity overflow */
  int64_t lod_builds;        /* hierarchy analyses swapped in (progressive hierarchy) */
  int64_t gaussians;         /* active Gaussians */
  double pixels;             /* pixels of completed requests */
  double p50_ms, p99_ms, mean_ms, max_ms;  /* arrival -> completion, completed requests */
  double wall_s;             /* since creation */
  uint64_t hbm_in_use, hbm_budget;
  int32_t contexts;
  int64_t train_beside_render;  /* train parts issued while a render part was in flight: their
                                   forward and backward ran beside it on the device */
} gs_stats;

typedef struct {
  size_t fixed_bytes;        /* arenas of parameters, gradients, moments */
  size_t context_bytes;      /* one batch context at the initial pair capacity */
  int64_t initial_pair_capacity;
  int32_t contexts;          /* contexts the budget admits (<= max_inflight) */
} gs_session_plan_info;

/* Seconds on the steady clock the session timestamps requests with. */
GS_API double gs_session_now(void);
/* Memory plan of a configuration (host only; GS_ERR_OOM if the budget holds
 * no batch context). */
GS_API gs_status gs_session_plan(const gs_session_config* cfg, gs_session_plan_info* out);
/* Creates a session on the current device (allocates its device memory,
 * starts its two threads). */
GS_API gs_status gs_session_create(const gs_session_config* cfg, gs_session** out);
/* Appends `count` Gaussians (host arrays in natural layout: means [count][3],
 * log-scales [count][3], quaternions [count][4] (w,x,y,z), opacity logits
 * [count], SH [count][3][nc]); batches submitted later see them.
 * GS_ERR_OOM beyond the capacity. */
GS_API gs_status gs_session_add_gaussians(gs_session* s, int64_t count, const float* means,
                                          const float* log_scales, const float* quats,
                                          const float* opa_logits, const float* sh);
/* Gaussians added after this call are tagged with keyframe kf (< 0: none;
 * the default): the keyframe whose correction moves them at a loop closure. */
GS_API gs_status gs_session_set_keyframe(gs_session* s, int32_t kf);
/* Loop closure (Sec. 5.5): every Gaussian tagged with keyframe k < num_kf
 * moves with the correction sim3[k] = (qw, qx, qy, qz, tx, ty, tz, s) (host
 * [num_kf][8], s > 0) as gs_sim3_update does; untagged Gaussians and tags >=
 * num_kf stay.  With a hierarchy every node moves, merged nodes with the
 * keyframe most common among their children (Sec. 6.1).  Enqueued on the
 * session stream after the batches already issued (it never waits for them),
 * before any later one. */
GS_API gs_status gs_session_loop_closure(gs_session* s, int32_t num_kf, const float* sim3);
/* Keyframe sampling weights (Sec. 6.2): keyframe k < num_kf is drawn for
 * optimisation with probability proportional to the active leaf Gaussians it
 * generated; keyframes whose count is below frac * the largest count are
 * offloaded (probability 0), except that the min_keep keyframes with the
 * largest counts (ties: smaller id) always stay (the paper: frac = 0.05,
 * min_keep = 50).  Counts are taken after everything enqueued so far; the
 * call waits for them (bounded).  p_out: host double [num_kf];
 * counts_out / kept_out (optional): host uint32 / uint8 [num_kf]. */
GS_API gs_status gs_session_keyframe_weights(gs_session* s, int32_t num_kf, int32_t min_keep, float frac,
                                             double* p_out, uint32_t* counts_out, uint8_t* kept_out);
/* Queues a request; *id identifies it for poll/wait.  Never blocks on GPU work. */
GS_API gs_status gs_session_submit(gs_session* s, const gs_request* req, int64_t* id);
/* *done = 1 when the request finished (its status is returned), else 0. */
GS_API gs_status gs_session_poll(gs_session* s, int64_t id, int32_t* done);
/* Waits up to timeout_ms for a request; GS_ERR_TIMEOUT if it is still pending. */
GS_API gs_status gs_session_wait(gs_session* s, int64_t id, int32_t timeout_ms);
/* Arrival and completion time (gs_session_now's clock, seconds) of a finished
 * request; GS_ERR_BUSY (no message) while it is pending. */
GS_API gs_status gs_session_times(gs_session* s, int64_t id, double* arrival_s, double* done_s);
/* Waits up to timeout_ms until nothing is queued or in flight (and a pending
 * hierarchy analysis has completed and been swapped in). */
GS_API gs_status gs_session_drain(gs_session* s, int32_t timeout_ms);
/* on != 0 pauses admission: submitted requests queue up and no new batch is
 * formed (batches in flight complete); on == 0 resumes, and the queued
 * requests are batched together.  For a client that submits one frame's
 * requests as a group.  Waiting on a held request times out; destroying a
 * held session still drains its queue. */
GS_API gs_status gs_session_hold(gs_session* s, int32_t on);
GS_API gs_status gs_session_stats(gs_session* s, gs_stats* out);
/* Copies the active parameters to host arrays in the library layout (each
 * pointer may be NULL): means4 [n][4], scale_opa [n][4], quat [n][4], sh
 * [3*nc][n].  Drains first. */
GS_API gs_status gs_session_read_params(gs_session* s, float* means4, float* scale_opa, float* quat, float* sh);
/* Checkpoint (parameters, Adam moments, step, active count) to a file and
 * back; both drain first.  A resumed session continues bit-identically. */
GS_API gs_status gs_session_save(gs_session* s, const char* path);
GS_API gs_status gs_session_load(gs_session* s, const char* path);
/* Analysis of the session's progressive hierarchy (lod = 1) from a new
 * keyframe's camera (cam host, pose12 host [R | t]): gs_hier_analyze with
 * tau_l = lod_tau / 2, then gs_hier_refine with tau_h = lod_tau, into the
 * back buffer of the active set, enqueued on the session stream after
 * everything issued so far.  Render parts keep using the front buffer while it
 * runs (double buffering); once it has completed, the next batch formed swaps
 * the buffers (the Adam moments of nodes whose flag changed are zeroed and
 * every new merged node takes its children's most common keyframe tag).
 * Leaves occupy rows [0, max_gaussians), merged nodes the rows after them;
 * trains use each view's cut of the front active set, so merged nodes are
 * trained; renders draw the render cut of the hierarchy (gs_project_hier_render
 * at lod_tau: descent from the roots while a node is coarser than lod_tau).  GS_ERR_BUSY (nothing issued) while the previous
 * analysis has not completed; GS_ERR_INVALID without a hierarchy.
 * Checkpoints (gs_session_save / load) are not supported with a hierarchy. */
GS_API gs_status gs_session_analyze(gs_session* s, const gs_camera* cam, const float* pose12);
/* The session's hierarchy (lod = 1) after draining (a pending analysis is
 * waited for and swapped in): *rows = node rows in use (leaf slots
 * [0, max_gaussians), merged nodes after them); with any array non-NULL,
 * copies rows [0, *rows) in the library layout (as gs_session_read_params;
 * sh [3*nc][*rows]), parent [rows], child [rows][4] and the front active
 * flags [rows].  GS_ERR_INVALID: no hierarchy, or max_rows < *rows with an
 * array given. */
GS_API gs_status gs_session_read_hierarchy(gs_session* s, int64_t max_rows, int64_t* rows, float* means4,
                                           float* scale_opa, float* quat, float* sh, int32_t* parent,
                                           int32_t* child, uint8_t* active);
/* Host-side fault injection for tests: the session's next `count` device
 * allocations fail as if the device were out of memory (no device fault is
 * made).  A batch whose pair buffers cannot grow finishes its requests with
 * GS_ERR_OOM and keeps serving at its old capacity. */
GS_API gs_status gs_session_inject_alloc_failures(gs_session* s, int32_t count);
/* Drains the queue, stops the threads, frees everything. */
GS_API gs_status gs_session_destroy(gs_session* s);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
