"""FP64 CPU oracle of the differentiable splat rasterizer (ctypes wrapper).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It loads
oracle/_build/liboracle.so (built from gs_oracle.cpp by oracle/build.py) and
shares nothing with the CUDA path.  Every function takes scenes and cameras in
natural layout (paper_2607_14481_b300.synth.Scene / Camera) and upcasts them to
float64.  The local bundle adjustment oracle is the separate module
oracle/ba.py (numpy/scipy).
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d = C.POINTER(C.c_double)
        i32 = C.POINTER(C.c_int32)
        u8 = C.POINTER(C.c_uint8)
        u32 = C.POINTER(C.c_uint32)
        u64 = C.POINTER(C.c_uint64)
        L.orc_sh_basis.argtypes = [C.c_int, C.c_int64, d, d]
        L.orc_render.argtypes = [C.c_int64, C.c_int, d, d, d, d, d, C.c_int, d, d, i32, i32, C.c_double,
                                 C.c_int, C.c_int, d, C.c_int, d, d, d, u8, d]
        L.orc_render_dual.argtypes = [C.c_int64, C.c_int, d, d, d, d, d, d, d, d, d, d, C.c_int, d, d,
                                      d, i32, i32, C.c_double, C.c_int, C.c_int, d, C.c_int, d, d, d]
        L.orc_backward.argtypes = [C.c_int64, C.c_int, d, d, d, d, d, C.c_int, d, d, i32, i32, C.c_double,
                                   C.c_int, C.c_int, d, C.c_int, d, d, d, d, d, d, d, d]
        L.orc_bin.argtypes = [C.c_int, C.c_int64, u32, i32, i32, C.c_int64, u64, u32, u32]
        L.orc_bin.restype = C.c_int64
        L.orc_adam.argtypes = [C.c_int64, d, d, d, d, d, C.c_double, C.c_double, C.c_double, C.c_int]
        L.orc_pose_adam.argtypes = [C.c_int, d, d, d, d, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int]
        L.orc_se3_exp.argtypes = [d, d, d]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        L.orc_get_threads.argtypes = []
        L.orc_get_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (OpenMP; results do not depend
    on it).  Returns the setting in force."""
    return int(lib().orc_set_threads(int(n)))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _p(a: np.ndarray, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


PROJ_FIELDS = ("vis", "mx", "my", "A", "B", "C", "opacity", "r", "g", "b", "depth", "radius",
               "xlo", "ylo", "xhi", "yhi", "clamp", "img_amb", "grad_amb", "bin_amb")


class _Inputs:
    def __init__(self, scene, cams, znear, tile, bg, clamp_j, windows=None):
        self.N = scene.n
        self.deg = scene.sh_degree
        self.means = _f64(scene.means)
        self.lsc = _f64(scene.log_scales)
        self.quat = _f64(scene.quats)
        self.opl = _f64(scene.opa_logits)
        self.sh = _f64(scene.sh)
        self.V = len(cams)
        self.poses = _f64(np.stack([c.pose12() for c in cams]))
        self.intr = _f64([[c.fx, c.fy, c.cx, c.cy] for c in cams])
        self.wh = np.ascontiguousarray(np.array([[c.width, c.height] for c in cams], np.int32))
        self.znear = float(znear)
        self.tw, self.th = int(tile[0]), int(tile[1])
        self.bg = _f64(bg)
        self.clamp_j = int(bool(clamp_j))
        self.cams = cams
        if windows is None:
            self.win = None
            self.sizes = [(c.width, c.height) for c in cams]
        else:
            self.win = np.ascontiguousarray(np.array(windows, np.int32).reshape(self.V, 4))
            for c, w in zip(cams, self.win):
                assert 0 <= w[0] and 0 <= w[1] and w[2] > 0 and w[3] > 0
                assert w[0] + w[2] <= c.width and w[1] + w[3] <= c.height
            self.sizes = [(int(w[2]), int(w[3])) for w in self.win]

    def win_ptr(self):
        return _p(self.win, C.c_int32) if self.win is not None else None

    def npix(self) -> int:
        return int(sum(w * h for w, h in self.sizes))

    def scene_args(self):
        return (self.N, self.deg, _p(self.means), _p(self.lsc), _p(self.quat), _p(self.opl), _p(self.sh))

    def split_views(self, flat: np.ndarray, per_pixel: int) -> List[np.ndarray]:
        out, off = [], 0
        for w, h in self.sizes:
            n = per_pixel * w * h
            a = flat[off:off + n]
            out.append(a.reshape((per_pixel, h, w)) if per_pixel > 1 else a.reshape((h, w)))
            off += n
        return out


def sh_basis(degree: int, dirs) -> np.ndarray:
    """Real SH basis values [n, (degree+1)^2] at unit directions [n,3]."""
    d = _f64(dirs).reshape(-1, 3)
    nc = (degree + 1) ** 2
    out = np.zeros((d.shape[0], nc))
    rc = lib().orc_sh_basis(int(degree), d.shape[0], _p(d), _p(out))
    assert rc == 0
    return out


def render(scene, cams, znear=0.2, tile=(16, 16), bg=(0.0, 0.0, 0.0), clamp_j=True,
           margins: Optional[Sequence[float]] = None, want_proj=False, windows=None) -> Dict:
    """Forward render.  Returns image (list of [3,H,W]), alpha (list of [H,W]),
    flags (list of [H,W] uint8: bit 0 = the image value depends on a decision
    within margin, bit 1 = its derivative does) and optionally proj
    [V,N,len(PROJ_FIELDS)].  windows: optional per-view (x0, y0, w, h) pixel
    windows; the outputs then cover the windows only."""
    a = _Inputs(scene, cams, znear, tile, bg, clamp_j, windows)
    P = a.npix()
    img = np.zeros(3 * P)
    alpha = np.zeros(P)
    flags = np.zeros(P, np.uint8)
    proj = np.zeros((a.V, a.N, len(PROJ_FIELDS))) if want_proj else None
    mg = _f64(margins) if margins is not None else None
    rc = lib().orc_render(*a.scene_args(), a.V, _p(a.poses), _p(a.intr), _p(a.wh, C.c_int32), a.win_ptr(),
                          a.znear, a.tw, a.th, _p(a.bg), a.clamp_j, _p(mg) if mg is not None else None,
                          _p(img), _p(alpha), _p(flags, C.c_uint8),
                          _p(proj) if proj is not None else None)
    assert rc == 0
    out = {"image": a.split_views(img, 3), "alpha": a.split_views(alpha, 1),
           "flags": a.split_views(flags, 1)}
    if proj is not None:
        out["proj"] = proj
    return out


def backward(scene, cams, dimage: Sequence[np.ndarray], dalpha: Optional[Sequence[np.ndarray]] = None,
             znear=0.2, tile=(16, 16), bg=(0.0, 0.0, 0.0), clamp_j=True, windows=None) -> Dict:
    """Analytic FP64 gradients of sum(dimage * image) + sum(dalpha * alpha)
    w.r.t. every parameter (natural layout) and every pose ([V,6], (v, omega)
    of the left perturbation T <- Exp(xi) T).  With windows, dimage/dalpha
    cover the windows and the loss gradient is zero outside them."""
    a = _Inputs(scene, cams, znear, tile, bg, clamp_j, windows)
    di = _f64(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in dimage]))
    da = (_f64(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in dalpha]))
          if dalpha is not None else None)
    N, nc = a.N, (a.deg + 1) ** 2
    g = {"means": np.zeros((N, 3)), "log_scales": np.zeros((N, 3)), "quats": np.zeros((N, 4)),
         "opa_logits": np.zeros(N), "sh": np.zeros((N, 3, nc)), "pose": np.zeros((a.V, 6))}
    rc = lib().orc_backward(*a.scene_args(), a.V, _p(a.poses), _p(a.intr), _p(a.wh, C.c_int32), a.win_ptr(),
                            a.znear, a.tw, a.th, _p(a.bg), a.clamp_j, _p(di), _p(da) if da is not None else None,
                            _p(g["means"]), _p(g["log_scales"]), _p(g["quats"]), _p(g["opa_logits"]),
                            _p(g["sh"]), _p(g["pose"]))
    assert rc == 0
    return g


def render_dual(scene, tangent: Dict[str, np.ndarray], pose_tangent: np.ndarray, cams, znear=0.2,
                tile=(16, 16), bg=(0.0, 0.0, 0.0), clamp_j=True, windows=None) -> Dict:
    """Forward render on dual numbers.  `tangent` holds arrays shaped like the
    scene's (keys means, log_scales, quats, opa_logits, sh); pose_tangent is
    [V,6] (v, omega).  Returns image values and their exact directional
    derivatives (lists of [3,H,W]) and the alpha derivative."""
    a = _Inputs(scene, cams, znear, tile, bg, clamp_j, windows)
    t = {k: _f64(tangent[k]) for k in ("means", "log_scales", "quats", "opa_logits", "sh")}
    tp = _f64(pose_tangent).reshape(a.V, 6)
    P = a.npix()
    img = np.zeros(3 * P)
    img_t = np.zeros(3 * P)
    al_t = np.zeros(P)
    rc = lib().orc_render_dual(*a.scene_args(), _p(t["means"]), _p(t["log_scales"]), _p(t["quats"]),
                               _p(t["opa_logits"]), _p(t["sh"]), a.V, _p(a.poses), _p(tp), _p(a.intr),
                               _p(a.wh, C.c_int32), a.win_ptr(), a.znear, a.tw, a.th, _p(a.bg), a.clamp_j,
                               _p(img), _p(img_t), _p(al_t))
    assert rc == 0
    return {"image": a.split_views(img, 3), "image_tan": a.split_views(img_t, 3),
            "alpha_tan": a.split_views(al_t, 1)}


def bin_records(depth: np.ndarray, rect: np.ndarray, tiles: Sequence[tuple]):
    """Reference binning of given records: depth [V,N] float32 (positive),
    rect [V,N,4] int (xlo, ylo, xhi, yhi; xlo > xhi = culled), tiles [(TX,TY)].
    Returns (keys uint64 [K], vals uint32 [K], ranges uint32 [G,2])."""
    depth = np.ascontiguousarray(depth, np.float32)
    bits = np.ascontiguousarray(depth.view(np.uint32))
    rect = np.ascontiguousarray(rect, np.int32)
    V, N = depth.shape
    tl = np.ascontiguousarray(np.array(tiles, np.int32).reshape(V, 2))
    G = int(sum(int(tx) * int(ty) for tx, ty in tl))
    cap = 0
    for v in range(V):
        r = rect[v]
        ok = (r[:, 0] <= r[:, 2]) & (r[:, 1] <= r[:, 3])
        cap += int(((r[:, 2] - r[:, 0] + 1) * (r[:, 3] - r[:, 1] + 1) * ok).sum())
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros((G, 2), np.uint32)
    K = lib().orc_bin(V, N, _p(bits, C.c_uint32), _p(rect, C.c_int32), _p(tl, C.c_int32), cap,
                      _p(keys, C.c_uint64), _p(vals, C.c_uint32), _p(ranges, C.c_uint32))
    assert K == cap
    return keys[:K], vals[:K], ranges


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """In-place bias-corrected Adam on float64 arrays; lr scalar or per element."""
    n = p.size
    lr_a = _f64(np.broadcast_to(np.asarray(lr, np.float64), (n,)))
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _f64(g)
    rc = lib().orc_adam(n, _p(p), _p(gg), _p(m), _p(v), _p(lr_a), b1, b2, eps, int(step))
    assert rc == 0


def pose_adam(poses, gpose, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """In-place pose step on float64 arrays: Adam on xi, then T <- Exp(xi) T.
    poses [V,12] ([R | t] row-major), gpose/m/v [V,6]."""
    for a in (poses, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _f64(gpose)
    rc = lib().orc_pose_adam(poses.shape[0], _p(poses), _p(gg), _p(m), _p(v), lr, b1, b2, eps, int(step))
    assert rc == 0


def se3_exp(xi) -> tuple:
    """SE(3) exponential of xi = (v, omega): returns (R [3,3], t [3])."""
    x = _f64(xi).reshape(6)
    R = np.zeros(9)
    t = np.zeros(3)
    lib().orc_se3_exp(_p(x), _p(R), _p(t))
    return R.reshape(3, 3), t


# ---------------------------------------------------------------------------
# Losses (outside the renderer, which consumes dL/dimage)
# ---------------------------------------------------------------------------

def l1_loss(images: Sequence[np.ndarray], targets: Sequence[np.ndarray]):
    """Mean absolute error over all views' pixels and channels; returns
    (loss, [dL/dimage per view])."""
    n = sum(t.size for t in targets)
    loss = sum(np.abs(np.asarray(i, np.float64) - t).sum() for i, t in zip(images, targets)) / n
    grads = [np.sign(np.asarray(i, np.float64) - t) / n for i, t in zip(images, targets)]
    return loss, grads


def mse_loss(images: Sequence[np.ndarray], targets: Sequence[np.ndarray]):
    """Mean squared error over all views' pixels and channels."""
    n = sum(t.size for t in targets)
    d = [np.asarray(i, np.float64) - t for i, t in zip(images, targets)]
    loss = sum((x * x).sum() for x in d) / n
    return loss, [2.0 * x / n for x in d]


# ---------------------------------------------------------------------------
# Level-of-detail hierarchy (gs_lod_oracle.cpp)
# ---------------------------------------------------------------------------

def _lod_lib():
    L = lib()
    if not hasattr(L, "_lod_ready"):
        d = C.POINTER(C.c_double)
        i64 = C.POINTER(C.c_int64)
        L.orc_lod_morton.argtypes = [C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_uint32), i64]
        L.orc_lod_merge.argtypes = [C.c_int, d, d, d, d, d, C.c_int, d, d, d, d, d, d]
        L.orc_lod_build.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_float), d, d, d, d, d, i64, i64,
                                    d, d, d, d, d, d]
        L.orc_lod_build.restype = C.c_int64
        L.orc_lod_cut.argtypes = [C.c_int64, C.c_int64, d, d, i64, d, C.c_double, C.c_double, C.c_double,
                                  d, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8)]
        L._lod_ready = True
    return L


def lod_morton(means32):
    """Morton codes (10 bits per axis over the bounding box, single-precision
    quantisation) and the (code, index) order of float32 points [n, 3]."""
    m = np.ascontiguousarray(means32, np.float32)
    n = m.shape[0]
    code = np.zeros(n, np.uint32)
    order = np.zeros(n, np.int64)
    _lod_lib().orc_lod_morton(n, m.ctypes.data_as(C.POINTER(C.c_float)), code.ctypes.data_as(C.POINTER(C.c_uint32)),
                              order.ctypes.data_as(C.POINTER(C.c_int64)))
    return code, order


def _cov3(c6):
    c = np.asarray(c6)
    out = np.empty(c.shape[:-1] + (3, 3))
    out[..., 0, 0], out[..., 0, 1], out[..., 0, 2] = c[..., 0], c[..., 1], c[..., 2]
    out[..., 1, 0], out[..., 1, 1], out[..., 1, 2] = c[..., 1], c[..., 3], c[..., 4]
    out[..., 2, 0], out[..., 2, 1], out[..., 2, 2] = c[..., 2], c[..., 4], c[..., 5]
    return out


def lod_merge(means, log_scales, quats, opa_logits, sh):
    """Moment-matching merge of k children (natural layouts; sh [k, nsh])."""
    mu, ls, q, o = _f64(means), _f64(log_scales), _f64(quats), _f64(opa_logits).reshape(-1)
    s = _f64(sh).reshape(len(o), -1)
    k, nsh = s.shape
    mean, cov6, lso, qo, oo, sho = np.zeros(3), np.zeros(6), np.zeros(3), np.zeros(4), np.zeros(1), np.zeros(nsh)
    _lod_lib().orc_lod_merge(k, _p(mu), _p(ls), _p(q), _p(o), _p(s), nsh, _p(mean), _p(cov6), _p(lso), _p(qo),
                             _p(oo), _p(sho))
    return {"mean": mean, "cov": _cov3(cov6), "log_scales": lso, "quat": qo, "opa_logit": float(oo[0]), "sh": sho}


def lod_build(scene):
    """Three-level hierarchy over the scene's Gaussians (the leaves).  Node
    numbering: leaves [0, n), level 1 [n, n + n1), level 2 after.  Returns
    parent [N] (-1 for roots), n1, n2 and the coarse nodes' parameters."""
    n = scene.n
    nc = (scene.sh_degree + 1) ** 2
    nsh = 3 * nc
    m32 = np.ascontiguousarray(scene.means, np.float32)
    mu, ls, q, o = _f64(scene.means), _f64(scene.log_scales), _f64(scene.quats), _f64(scene.opa_logits)
    sh = _f64(scene.sh).reshape(n, nsh)
    n1 = (n + 7) // 8
    n2 = (n1 + 7) // 8
    k = n1 + n2
    parent = np.zeros(n + k, np.int64)
    n1o = np.zeros(1, np.int64)
    pm, pc, pl, pq, po, ps = (np.zeros((k, 3)), np.zeros((k, 6)), np.zeros((k, 3)), np.zeros((k, 4)), np.zeros(k),
                              np.zeros((k, nsh)))
    got = _lod_lib().orc_lod_build(n, nsh, m32.ctypes.data_as(C.POINTER(C.c_float)), _p(mu), _p(ls), _p(q), _p(o),
                                   _p(sh), parent.ctypes.data_as(C.POINTER(C.c_int64)),
                                   n1o.ctypes.data_as(C.POINTER(C.c_int64)), _p(pm), _p(pc), _p(pl), _p(pq), _p(po),
                                   _p(ps))
    assert got == k and n1o[0] == n1
    return {"parent": parent, "n1": n1, "n2": n2, "means": pm, "cov": _cov3(pc), "log_scales": pl, "quats": pq,
            "opa_logits": po, "sh": ps.reshape(k, 3, nc)}


def lod_cut(means, log_scales, parent, n_leaf, cam, tau=1.0, znear=0.2):
    """Screen size of every node and the cut for one camera: selected[i] = 1
    if node i is rendered; amb[i] = 1 where a decision sits within 1e-5 tau
    of the threshold."""
    mu, ls = _f64(means), _f64(log_scales)
    par = np.ascontiguousarray(parent, np.int64)
    N = mu.shape[0]
    pose = _f64(cam.pose12())
    screen = np.zeros(N)
    sel = np.zeros(N, np.uint8)
    amb = np.zeros(N, np.uint8)
    _lod_lib().orc_lod_cut(N, int(n_leaf), _p(mu), _p(ls), par.ctypes.data_as(C.POINTER(C.c_int64)), _p(pose),
                           float(cam.fx), float(znear), float(tau), _p(screen),
                           sel.ctypes.data_as(C.POINTER(C.c_uint8)), amb.ctypes.data_as(C.POINTER(C.c_uint8)))
    return {"screen": screen, "selected": sel.astype(bool), "amb": amb.astype(bool)}


# ---------------------------------------------------------------------------
# Loop-closure update of the Gaussians (Sec. 5.5 / 6)
# ---------------------------------------------------------------------------

def _qmul(a, b):
    """Hamilton product of quaternions (w, x, y, z), row-wise."""
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def _qrot(q):
    """Rotation matrices of unit quaternions (w, x, y, z)."""
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z); R[..., 0, 1] = 2 * (x * y - w * z); R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z); R[..., 1, 1] = 1 - 2 * (x * x + z * z); R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y); R[..., 2, 1] = 2 * (y * z + w * x); R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def sim3_update(means, log_scales, quats, kf, sim3):
    """Every Gaussian moves with the Sim(3) correction of the keyframe that
    spawned it (Sec. 5.5: the same transformation as its keyframe, scale and
    rotation updated accordingly): mean' = s R mean + t, rotation' = R * rotation
    (quaternion q_S q), log-scales' = log-scales + log s; a negative keyframe
    leaves the Gaussian unchanged.  sim3 [K, 8] = (qw, qx, qy, qz, tx, ty, tz, s)
    with the rotation as a unit quaternion.  FP64; returns new arrays."""
    mu, ls, q = _f64(means).copy(), _f64(log_scales).copy(), _f64(quats).copy()
    kf = np.asarray(kf, np.int64)
    S = _f64(sim3).reshape(-1, 8)
    sel = kf >= 0
    k = kf[sel]
    qs = S[k, :4] / np.linalg.norm(S[k, :4], axis=1, keepdims=True)
    R = _qrot(qs)
    s = S[k, 7]
    mu[sel] = s[:, None] * np.einsum("nij,nj->ni", R, mu[sel]) + S[k, 4:7]
    q[sel] = _qmul(qs, q[sel])
    ls[sel] = ls[sel] + np.log(s)[:, None]
    return mu, ls, q


# ---------------------------------------------------------------------------
# Keyframe selection for optimisation (Sec. 6.2)
# ---------------------------------------------------------------------------

def keyframe_weights(kf, num_kf, min_keep=50, frac=0.05):
    """Sampling probabilities of the keyframes (Sec. 6.2): keyframe k is drawn
    with probability proportional to the number of active leaf Gaussians it
    generated (c_k); keyframes whose count is below frac * max_j c_j are
    offloaded, except that the min_keep keyframes with the largest counts
    (ties: smaller id first) always stay.  Returns (counts, probabilities,
    kept mask)."""
    kf = np.asarray(kf, np.int64)
    kf = kf[(kf >= 0) & (kf < num_kf)]
    c = np.bincount(kf, minlength=num_kf).astype(np.int64)
    kept = c >= frac * c.max() if num_kf and c.max() > 0 else np.zeros(num_kf, bool)
    order = sorted(range(num_kf), key=lambda k: (-c[k], k))
    for k in order[:min_keep]:
        kept[k] = True
    w = np.where(kept, c, 0).astype(np.float64)
    p = w / w.sum() if w.sum() > 0 else w
    return c, p, kept


# ---------------------------------------------------------------------------
# Progressive hierarchy (gs_lod_oracle.cpp, orc_hier_*)
# ---------------------------------------------------------------------------

def _hier_lib():
    L = _lod_lib()
    if not hasattr(L, "_hier_ready"):
        d = C.POINTER(C.c_double)
        f = C.POINTER(C.c_float)
        i32 = C.POINTER(C.c_int32)
        u8 = C.POINTER(C.c_uint8)
        i64 = C.POINTER(C.c_int64)
        L.orc_hier_analyze.argtypes = [C.c_int64, C.c_int64, C.c_int, f, d, d, d, d, d, i32, i32, u8, d, d, i32,
                                       C.c_double, C.c_double, d, u8, i64]
        L.orc_hier_analyze.restype = C.c_int
        L.orc_hier_refine.argtypes = [C.c_int64, d, d, i32, u8, d, d, i32, C.c_double, C.c_double, u8]
        L.orc_hier_refine.restype = C.c_int64
        L.orc_hier_render_cut.argtypes = [C.c_int64, d, d, i32, i32, d, d, i32, C.c_double, C.c_double, u8, u8]
        L.orc_hier_render_cut.restype = C.c_int64
        L._hier_ready = True
    return L


class HierState:
    """Node state of the progressive hierarchy in natural layouts, capacity
    `cap` rows, the first n_nodes in use: means32 [cap,3] float32, means /
    log_scales [cap,3], quats [cap,4], opa_logits [cap], sh [cap,3,nc]
    (float64), parent [cap] int32 (-1: root), child [cap,4] int32 (-1: none),
    active [cap] uint8."""

    def __init__(self, scene, cap):
        n = scene.n
        self.nc = (scene.sh_degree + 1) ** 2
        self.cap, self.n_nodes = int(cap), n
        self.means32 = np.zeros((cap, 3), np.float32)
        self.means32[:n] = scene.means
        self.means = np.zeros((cap, 3))
        self.means[:n] = scene.means
        self.log_scales = np.zeros((cap, 3))
        self.log_scales[:n] = scene.log_scales
        self.quats = np.zeros((cap, 4))
        self.quats[:, 0] = 1.0
        self.quats[:n] = scene.quats
        self.opa_logits = np.zeros(cap)
        self.opa_logits[:n] = scene.opa_logits
        self.sh = np.zeros((cap, 3, self.nc))
        self.sh[:n] = scene.sh
        self.parent = np.full(cap, -1, np.int32)
        self.child = np.full((cap, 4), -1, np.int32)
        self.active = np.zeros(cap, np.uint8)
        self.active[:n] = 1

    @classmethod
    def from_arrays(cls, nat, parent, child, active, n_nodes):
        """A state from arrays of `cap` rows: nat = natural-layout parameters
        (means, log_scales, quats, opa_logits, sh), the links and flags."""
        st = cls.__new__(cls)
        cap = len(parent)
        st.nc = nat["sh"].shape[2]
        st.cap, st.n_nodes = cap, int(n_nodes)
        st.means = np.ascontiguousarray(nat["means"], np.float64)
        st.means32 = np.ascontiguousarray(nat["means"], np.float32)
        st.log_scales = np.ascontiguousarray(nat["log_scales"], np.float64)
        st.quats = np.ascontiguousarray(nat["quats"], np.float64)
        st.opa_logits = np.ascontiguousarray(nat["opa_logits"], np.float64)
        st.sh = np.ascontiguousarray(nat["sh"], np.float64)
        st.parent = np.ascontiguousarray(parent, np.int32)
        st.child = np.ascontiguousarray(np.asarray(child).reshape(cap, 4), np.int32)
        st.active = np.ascontiguousarray(active, np.uint8)
        return st

    def copy(self):
        c = HierState.__new__(HierState)
        c.__dict__ = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in self.__dict__.items()}
        return c


def _cam_args(cam):
    pose = _f64(cam.pose12())
    intr = _f64([cam.fx, cam.fy, cam.cx, cam.cy])
    wh = np.ascontiguousarray(np.array([cam.width, cam.height], np.int32))
    return pose, intr, wh


def hier_analyze(st: HierState, cam, znear=0.2, tau_l=0.5) -> Dict:
    """One analysis of the progressive hierarchy from `cam` (updates st in
    place).  Returns info (n_nodes, triggered, candidates, active, pulled,
    groups, grouped), the screen sizes S and the ambiguity flags."""
    L = _hier_lib()
    nsh = 3 * st.nc
    S = np.zeros(st.cap)
    amb = np.zeros(st.cap, np.uint8)
    info = np.zeros(8, np.int64)
    pose, intr, wh = _cam_args(cam)
    sh = np.ascontiguousarray(st.sh.reshape(st.cap, nsh))
    rc = L.orc_hier_analyze(st.n_nodes, st.cap, nsh, st.means32.ctypes.data_as(C.POINTER(C.c_float)),
                            _p(st.means), _p(st.log_scales), _p(st.quats), _p(st.opa_logits), _p(sh),
                            st.parent.ctypes.data_as(C.POINTER(C.c_int32)),
                            st.child.ctypes.data_as(C.POINTER(C.c_int32)),
                            st.active.ctypes.data_as(C.POINTER(C.c_uint8)), _p(pose), _p(intr),
                            wh.ctypes.data_as(C.POINTER(C.c_int32)), float(znear), float(tau_l), _p(S),
                            amb.ctypes.data_as(C.POINTER(C.c_uint8)), info.ctypes.data_as(C.POINTER(C.c_int64)))
    assert rc == 0, "hierarchy capacity exceeded"
    st.sh[:] = sh.reshape(st.cap, 3, st.nc)
    st.n_nodes = int(info[0])
    names = ("n_nodes", "triggered", "candidates", "active", "pulled", "groups", "grouped")
    return {"info": {k: int(v) for k, v in zip(names, info)}, "S": S, "amb": amb}


def hier_refine(st: HierState, cam, znear=0.2, tau_h=1.0):
    """Reload: refinement passes of st.active for `cam` (in place).  Returns
    the number of nodes replaced by their children and the ambiguity flags."""
    L = _hier_lib()
    amb = np.zeros(max(1, st.n_nodes), np.uint8)
    pose, intr, wh = _cam_args(cam)
    k = L.orc_hier_refine(st.n_nodes, _p(st.means), _p(st.log_scales), st.child.ctypes.data_as(C.POINTER(C.c_int32)),
                          st.active.ctypes.data_as(C.POINTER(C.c_uint8)), _p(pose), _p(intr),
                          wh.ctypes.data_as(C.POINTER(C.c_int32)), float(znear), float(tau_h),
                          amb.ctypes.data_as(C.POINTER(C.c_uint8)))
    return int(k), amb


def hier_render_cut(st: HierState, cam, znear=0.2, tau=1.0):
    """Rendering a stored hierarchy (Sec. 6.2): descend from the roots while a
    node is coarser than tau and has children.  Returns (selected [n_nodes]
    uint8, amb [n_nodes] uint8: a decision within 1e-5 of tau on the node's
    path); the state is not changed."""
    L = _hier_lib()
    n = st.n_nodes
    sel = np.zeros(max(1, n), np.uint8)
    amb = np.zeros(max(1, n), np.uint8)
    pose, intr, wh = _cam_args(cam)
    L.orc_hier_render_cut(n, _p(st.means), _p(st.log_scales), st.parent.ctypes.data_as(C.POINTER(C.c_int32)),
                          st.child.ctypes.data_as(C.POINTER(C.c_int32)), _p(pose), _p(intr),
                          wh.ctypes.data_as(C.POINTER(C.c_int32)), float(znear), float(tau),
                          sel.ctypes.data_as(C.POINTER(C.c_uint8)), amb.ctypes.data_as(C.POINTER(C.c_uint8)))
    return sel[:n].copy(), amb[:n].copy()


def hier_view_cut(st: HierState, cam, znear=0.2, tau_h=1.0) -> np.ndarray:
    """The nodes a render from `cam` uses: the refinement of a copy of the
    active set (the state is not changed)."""
    c = st.copy()
    hier_refine(c, cam, znear, tau_h)
    return c.active[:st.n_nodes].copy()
