"""Seeded synthetic scenes, cameras and trajectories.

The paper's captures (MipNeRF360, TUM, StaticHikes, CityWalk ...) are not
available, so every input is drawn here with the shapes of those captures:
Gaussian counts of 0.5-2M for medium scenes (the paper's hierarchy memory
evaluation reports 1.3-2.1M), 720p-1080p views, forward-moving or
inward-facing trajectories.

This module holds random draws and camera placement only.  It contains none of
the renderer's arithmetic, so it can feed both the CUDA path and the CPU oracle.
All arrays are float32 (the precision the renderer consumes); the oracle upcasts
the same values to float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np


@dataclass
class Scene:
    """Gaussian primitives in natural layout (Sec. 7: position, opacity,
    rotation, scale and SH coefficients per primitive)."""
    means: np.ndarray        # [N,3]
    log_scales: np.ndarray   # [N,3]
    quats: np.ndarray        # [N,4] (w,x,y,z), not normalised
    opa_logits: np.ndarray   # [N]
    sh: np.ndarray           # [N,3,C], C = (degree+1)^2

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(np.sqrt(self.sh.shape[2]))) - 1

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opa_logits.copy(), self.sh.copy())

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx], self.log_scales[idx], self.quats[idx],
                     self.opa_logits[idx], self.sh[idx])


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).
    R, t map world to camera: x_cam = R x_world + t."""
    R: np.ndarray            # [3,3] float32
    t: np.ndarray            # [3]   float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def pose12(self) -> np.ndarray:
        """[R | t] as 12 values, row-major 3x4, in the dtype R and t carry."""
        R = np.asarray(self.R)
        t = np.asarray(self.t)
        return np.concatenate([R, t[:, None]], axis=1).reshape(12)

    @property
    def pixels(self) -> int:
        return self.width * self.height


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_scene(n: int, seed: int, sh_degree: int, mean_lo: Sequence[float],
                 mean_hi: Sequence[float], log_scale_mu: float, log_scale_sigma: float,
                 sh_rest_sigma: float = 0.05) -> Scene:
    """Means uniform in a box, log-scales N(mu, sigma^2) per axis, quaternions
    N(0, I4) (normalised by the renderer), opacity logits N(0,1) (so the
    opacity is sigmoid of a standard normal), SH DC uniform in [0,1], higher
    bands N(0, sh_rest_sigma^2)."""
    g = _rng(seed)
    lo = np.asarray(mean_lo, np.float64)
    hi = np.asarray(mean_hi, np.float64)
    means = (lo + (hi - lo) * g.random((n, 3))).astype(np.float32)
    log_scales = g.normal(log_scale_mu, log_scale_sigma, (n, 3)).astype(np.float32)
    quats = g.normal(0.0, 1.0, (n, 4)).astype(np.float32)
    # keep quaternions away from zero norm (a measure-zero event, redrawn)
    bad = np.linalg.norm(quats, axis=1) < 1e-3
    while bad.any():
        quats[bad] = g.normal(0.0, 1.0, (int(bad.sum()), 4)).astype(np.float32)
        bad = np.linalg.norm(quats, axis=1) < 1e-3
    opa_logits = g.normal(0.0, 1.0, n).astype(np.float32)
    nc = (sh_degree + 1) ** 2
    sh = np.zeros((n, 3, nc), np.float32)
    sh[:, :, 0] = g.random((n, 3)).astype(np.float32)
    if nc > 1:
        sh[:, :, 1:] = g.normal(0.0, sh_rest_sigma, (n, 3, nc - 1)).astype(np.float32)
    return Scene(means, log_scales, quats, opa_logits, sh)


def look_at(eye, target, fx, fy, cx, cy, width, height, up=(0.0, -1.0, 0.0)) -> Camera:
    """Camera at `eye` looking at `target`; world 'up' is -y (image y grows down)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    return Camera(R.astype(np.float32), t.astype(np.float32), float(fx), float(fy),
                  float(cx), float(cy), int(width), int(height))


def _small_rotation(g: np.random.Generator, sigma_deg: float) -> np.ndarray:
    a = np.deg2rad(g.normal(0.0, sigma_deg, 3))
    cx, sx, cy, sy, cz, sz = np.cos(a[0]), np.sin(a[0]), np.cos(a[1]), np.sin(a[1]), np.cos(a[2]), np.sin(a[2])
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rx @ Ry @ Rz


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def plain_small(seed: int = 7):
    """4,096 Gaussians in [-1,1]^3, log-scales N(-3.5, 0.4^2), SH degree 0;
    one 128x128 camera with f = 120 at distance 3 looking at the origin
    (R = I, t = (0,0,3)); a seeded U[0,1] target image."""
    sc = random_scene(4096, seed, 0, (-1, -1, -1), (1, 1, 1), -3.5, 0.4)
    cam = Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 3], np.float32),
                 120.0, 120.0, 64.0, 64.0, 128, 128)
    target = _rng(seed + 1).random((3, 128, 128)).astype(np.float32)
    return sc, [cam], [target]


def box_scene(n: int, seed: int, sh_degree: int = 3) -> Scene:
    """Gaussians in a 20 x 5 x 20 m box (y is the 5 m vertical), log-scales
    N(-4, 0.5^2), SH degree 3 with higher bands N(0, 0.05^2)."""
    return random_scene(n, seed, sh_degree, (-10, -2.5, -10), (10, 2.5, 10), -4.0, 0.5)


def forward_trajectory(n_poses: int, seed: int, width: int = 1280, height: int = 720,
                       f: float = 1000.0) -> List[Camera]:
    """Poses moving along +z from z = -9 to z = +9 looking +z, jittered by
    N(0, 0.02 m) in position and N(0, 0.5 deg) per rotation axis."""
    g = _rng(seed)
    cams = []
    zs = np.linspace(-9.0, 9.0, n_poses) if n_poses > 1 else np.array([-9.0])
    for z in zs:
        eye = np.array([0.0, 0.0, z]) + g.normal(0.0, 0.02, 3)
        R = _small_rotation(g, 0.5)
        t = -R @ eye
        cams.append(Camera(R.astype(np.float32), t.astype(np.float32), f, f,
                           width / 2.0, height / 2.0, width, height))
    return cams


def diffcheck(seed: int = 2007):
    """256 Gaussians in [-0.5,0.5]^3, log-scales N(-2.5, 0.3^2), SH degree 3;
    three 64x64 views, f = 60, on a 30 degree arc at distance 2.5 looking at
    the origin; a seeded U[0,1] target per view."""
    sc = random_scene(256, seed, 3, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), -2.5, 0.3)
    cams = []
    for a in np.deg2rad([-15.0, 0.0, 15.0]):
        eye = (2.5 * np.sin(a), 0.0, -2.5 * np.cos(a))
        cams.append(look_at(eye, (0, 0, 0), 60.0, 60.0, 32.0, 32.0, 64, 64))
    g = _rng(seed + 1)
    targets = [g.random((3, 64, 64)).astype(np.float32) for _ in cams]
    return sc, cams, targets


RESOLUTIONS = ((960, 540), (1280, 720), (1600, 900), (1920, 1080))


def loop_views(n_views: int, seed: int, radius: float = 12.0, height: float = -1.5):
    """Inward-facing loop of radius 12 m at height 1.5 m (y = -1.5, y points
    down) looking at the centre; each view's resolution drawn from 540p-1080p,
    f = 0.78 W."""
    g = _rng(seed)
    cams = []
    for k in range(n_views):
        a = 2.0 * np.pi * k / n_views
        w, h = RESOLUTIONS[int(g.integers(0, len(RESOLUTIONS)))]
        eye = (radius * np.sin(a), height, -radius * np.cos(a))
        f = 0.78 * w
        cams.append(look_at(eye, (0, 0, 0), f, f, w / 2.0, h / 2.0, w, h))
    return cams


def perturbed(sc: Scene, seed: int, sigma: float = 0.01) -> Scene:
    """Copy of a scene with means moved by N(0, sigma^2): used to render
    targets that carry structure."""
    out = sc.copy()
    out.means = (out.means + _rng(seed).normal(0.0, sigma, out.means.shape)).astype(np.float32)
    return out


def random_records(views: Sequence[tuple], n: int, seed: int, tie_levels: int = 0):
    """Synthetic per-(view, Gaussian) bin inputs for the binning stage alone:
    positive depths (as float32), tile rects inside each view's tile grid and a
    culled share.  `views` holds (tiles_x, tiles_y).  With tie_levels > 0 the
    depths take only that many distinct values, forcing key ties."""
    g = _rng(seed)
    V = len(views)
    depth = np.zeros((V, n), np.float32)
    rect = np.zeros((V, n, 4), np.int32)
    for v, (tx, ty) in enumerate(views):
        if tie_levels > 0:
            levels = (0.2 + 50.0 * g.random(tie_levels)).astype(np.float32)
            depth[v] = levels[g.integers(0, tie_levels, n)]
        else:
            depth[v] = (0.2 + 50.0 * g.random(n) ** 2).astype(np.float32)
        # footprints: mostly 1-3 tiles wide, a heavy tail of large ones
        wx = np.minimum(tx, g.geometric(0.55, n) + (g.random(n) < 0.01) * g.integers(0, tx, n))
        wy = np.minimum(ty, g.geometric(0.55, n) + (g.random(n) < 0.01) * g.integers(0, ty, n))
        x0 = g.integers(0, tx, n)
        y0 = g.integers(0, ty, n)
        x1 = np.minimum(tx - 1, x0 + wx - 1)
        y1 = np.minimum(ty - 1, y0 + wy - 1)
        culled = g.random(n) < 0.3
        rect[v, :, 0] = np.where(culled, 1, x0)
        rect[v, :, 1] = np.where(culled, 1, y0)
        rect[v, :, 2] = np.where(culled, 0, x1)
        rect[v, :, 3] = np.where(culled, 0, y1)
    return depth, rect


# ---------------------------------------------------------------------------
# Streaming workload: a camera walking a 200 m loop; every frame brings new
# Gaussians in its frustum and a handful of mixed-resolution requests
# ---------------------------------------------------------------------------
STREAM_RESOLUTIONS = ((960, 540), (1280, 720), (1600, 900), (1920, 1080))


def stream_camera(k: int, n_frames: int, width: int = 1920, height: int = 1080, loop_m: float = 200.0,
                  height_m: float = -1.5) -> Camera:
    """Frame k's camera on a loop of loop_m metres (radius loop_m / 2 pi, at
    height 1.5 m with y down), looking along the direction of travel;
    f = 0.78 W, principal point at the image centre."""
    r = loop_m / (2 * np.pi)
    a = 2 * np.pi * k / max(1, n_frames)
    eye = np.array([r * np.cos(a), height_m, r * np.sin(a)])
    fwd = np.array([-np.sin(a), 0.0, np.cos(a)])
    return look_at(eye, eye + fwd, 0.78 * width, 0.78 * width, width / 2, height / 2, width, height)


def with_resolution(cam: Camera, width: int, height: int) -> Camera:
    """The same pose with another image size (f = 0.78 W)."""
    return Camera(cam.R, cam.t, 0.78 * width, 0.78 * width, width / 2, height / 2, int(width), int(height))


def frustum_gaussians(cam: Camera, n: int, seed: int, sh_degree: int = 3, depth=(1.0, 8.0)) -> Scene:
    """n Gaussians spawned in the camera's frustum: a uniform pixel, depth
    U(1, 8) m, log-scale log(1.5 depth / f) + N(0, 0.2^2) per axis (about 1.5
    px on screen), random rotation, opacity logit N(0, 1), SH DC U[0, 1] and
    higher bands N(0, 0.05^2)."""
    g = _rng(seed)
    u = g.uniform(0, cam.width, n)
    v = g.uniform(0, cam.height, n)
    z = g.uniform(depth[0], depth[1], n)
    pc = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], axis=1)
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    means = ((pc - t) @ R).astype(np.float32)  # R^T (p - t)
    log_scales = (np.log(1.5 * z / cam.fx)[:, None] + g.normal(0, 0.2, (n, 3))).astype(np.float32)
    quats = g.normal(size=(n, 4)).astype(np.float32)
    opa = g.normal(0.0, 1.0, n).astype(np.float32)
    nc = (sh_degree + 1) ** 2
    sh = np.zeros((n, 3, nc), np.float32)
    sh[:, :, 0] = g.uniform(0, 1, (n, 3))
    if nc > 1:
        sh[:, :, 1:] = g.normal(0.0, 0.05, (n, 3, nc - 1))
    return Scene(means, log_scales, quats, opa, sh)


def frustum_clusters(cam: Camera, n: int, seed: int, per_cluster: int = 4, sh_degree: int = 3,
                     depth=(1.0, 8.0)) -> Scene:
    """n Gaussians in groups of per_cluster that overlap one another, as
    neighbouring Gaussians on a reconstructed surface do: the group centres
    and every Gaussian's size, rotation, opacity and colour as
    frustum_gaussians; members offset from their centre by N(0, s^2) per axis,
    s = exp(the member's mean log-scale)."""
    k = n // per_cluster
    base = frustum_gaussians(cam, k, seed, sh_degree, depth)
    g = _rng(seed + 104729)
    members = frustum_gaussians(cam, k * per_cluster, seed + 1, sh_degree, depth)
    centres = np.repeat(base.means, per_cluster, axis=0)
    ls = np.repeat(base.log_scales, per_cluster, axis=0) + g.normal(0, 0.1, (k * per_cluster, 3)).astype(np.float32)
    s = np.exp(ls.mean(axis=1))[:, None]
    means = (centres + g.normal(0, 1.0, (k * per_cluster, 3)) * s).astype(np.float32)
    return Scene(means, ls.astype(np.float32), members.quats, members.opa_logits, members.sh)


def stream_frame(k: int, n_frames: int, seed: int):
    """Frame k of the stream: (camera at 1080p, U{10k..50k} new Gaussians in
    its frustum, requests [(kind, width, height)] with U{1..8} requests, each
    render (kind 0) or train (kind 1) with probability 1/2 and a resolution
    drawn from 540p..1080p)."""
    g = _rng(seed * 1000003 + k)
    cam = stream_camera(k, n_frames)
    new = frustum_gaussians(cam, int(g.integers(10_000, 50_001)), seed * 7919 + k)
    reqs = []
    for _ in range(int(g.integers(1, 9))):
        w, h = STREAM_RESOLUTIONS[int(g.integers(0, len(STREAM_RESOLUTIONS)))]
        reqs.append((0 if g.random() < 0.5 else 1, w, h))
    return cam, new, reqs


# ---------------------------------------------------------------------------
# Local bundle adjustment problem (Sec. 5.3: N = 20 keyframes, n_f = 4 of them
# fixed, K = 10,000 landmarks, each observed by a fixed subset of keyframes)
# ---------------------------------------------------------------------------

def ba_problem(seed: int, n_cams: int = 20, n_points: int = 10_000, obs_per_point: int = 8, n_fixed: int = 4,
               width: int = 1280, height: int = 720, noise_px: float = 0.5, rot_sigma: float = 0.01,
               trans_sigma: float = 0.05, point_sigma: float = 0.05, focal_err: float = 0.02):
    """Synthetic local BA problem: keyframes on a gently curving path looking
    forward, landmarks in the volume they see, each landmark observed by a
    fixed random subset of obs_per_point of the keyframes that see it, observations = true
    projections + N(0, noise_px^2); the first n_fixed keyframes are fixed and
    exact, the others start with pose noise, landmarks with position noise,
    the shared focal length with a relative error.  Poses are world->camera
    [R | t] row-major float32 [N][12]."""
    if not 1 <= obs_per_point <= n_cams:
        raise ValueError("obs_per_point must be in [1, n_cams]")
    g = _rng(seed)
    f_true = 0.8 * width
    cams = []
    for k in range(n_cams):
        a = 0.3 * k / max(1, n_cams - 1)
        eye = np.array([4.0 * np.sin(a), -0.2 * np.sin(2.1 * a), 0.35 * k])
        fwd = np.array([np.sin(a + 0.15), 0.0, np.cos(a + 0.15)])
        cams.append(look_at(eye, eye + fwd, f_true, f_true, width / 2, height / 2, width, height))
    # landmarks: in front of a random keyframe, inside its view; kept when at
    # least obs_per_point keyframes see it (depth > 1, inside the image), and
    # observed by a random fixed subset of obs_per_point of those keyframes
    Rs = np.stack([np.asarray(c.R, np.float64) for c in cams])
    ts = np.stack([np.asarray(c.t, np.float64) for c in cams])
    pts = np.zeros((0, 3))
    obs_cam = np.zeros((0, obs_per_point), np.int32)
    while pts.shape[0] < n_points:
        m = 2 * n_points
        k = g.integers(0, n_cams, m)
        u, v, z = g.uniform(0.1 * width, 0.9 * width, m), g.uniform(0.1 * height, 0.9 * height, m), g.uniform(3.0, 12.0, m)
        pc = np.stack([(u - width / 2) * z / f_true, (v - height / 2) * z / f_true, z], axis=1)
        P = np.einsum("mji,mj->mi", Rs[k], pc - ts[k])
        Xc = np.einsum("kij,mj->mki", Rs, P) + ts[None]
        uu = f_true * Xc[..., 0] / np.maximum(Xc[..., 2], 1e-9) + width / 2
        vv = f_true * Xc[..., 1] / np.maximum(Xc[..., 2], 1e-9) + height / 2
        vis = (Xc[..., 2] > 1.0) & (uu > 0) & (uu < width) & (vv > 0) & (vv < height)
        ok = vis.sum(axis=1) >= obs_per_point
        P, vis = P[ok], vis[ok]
        key = np.where(vis, g.random(vis.shape), 2.0)
        sel = np.sort(np.argsort(key, axis=1, kind="stable")[:, :obs_per_point], axis=1).astype(np.int32)
        pts = np.concatenate([pts, P])[:n_points]
        obs_cam = np.concatenate([obs_cam, sel])[:n_points]
    Xc = np.einsum("lkij,lkj->lki", Rs[obs_cam], np.broadcast_to(pts[:, None, :], obs_cam.shape + (3,))) + ts[obs_cam]
    uv = np.stack([f_true * Xc[..., 0] / Xc[..., 2] + width / 2, f_true * Xc[..., 1] / Xc[..., 2] + height / 2], axis=-1)
    uv = uv + g.normal(0.0, noise_px, uv.shape)
    poses_true = np.concatenate([Rs, ts[:, :, None]], axis=2).reshape(n_cams, 12)
    poses0 = poses_true.copy()
    for k in range(n_fixed, n_cams):
        R = Rs[k] @ _small_rotation(g, np.rad2deg(rot_sigma))
        t = ts[k] + g.normal(0.0, trans_sigma, 3)
        poses0[k] = np.concatenate([R, t[:, None]], axis=1).reshape(12)
    pts0 = pts + g.normal(0.0, point_sigma, pts.shape)
    return {"poses_true": poses_true.astype(np.float32), "points_true": pts.astype(np.float32), "f_true": f_true,
            "poses0": poses0.astype(np.float32), "points0": pts0.astype(np.float32),
            "f0": f_true * (1.0 + focal_err), "obs_cam": obs_cam, "obs_uv": uv.astype(np.float32),
            "cx": width / 2, "cy": height / 2, "n_fixed": n_fixed}
