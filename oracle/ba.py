"""FP64 CPU oracle of the local bundle adjustment (Sec. 5.1, "Local Bundle
Adjustment" and its supplementary "Fast Bundle Adjustment" paragraph).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this module; it shares nothing with
the CUDA path.

The paper fixes the problem's shape (N keyframes of which n_f are fixed, K
landmarks each observed by a fixed subset of the keyframes, intrinsics
optimised, GPU residual/Jacobian kernels, dense Schur complement) but not the
solver's details.  The readings taken here, in the order the solver uses them:

* Observation model: pinhole with one shared focal length f (fx = fy = f) and
  a fixed principal point; a keyframe's pose is world->camera (R, t), a
  landmark X is projected as u = f x/z + cx, v = f y/z + cy with
  (x, y, z) = R X + t.  Residual r = (u, v) - observation, in pixels; an
  observation with z <= Z_MIN contributes no residual.
* Cost: E = sum of r^2 over all valid observations (no robust kernel).
* Update (retraction): R <- Exp(dtheta) R, t <- t + dt for every free
  keyframe (Exp = Rodrigues), X <- X + dX, f <- f + df.  Fixed keyframes keep
  their pose exactly.
* Parameter order: free keyframes in index order (dtheta then dt, 6 each),
  then f (when optimised), then the landmarks (3 each).
* Levenberg-Marquardt (Marquardt's diagonal scaling): H = J^T J, g = J^T r,
  (H + lambda D) delta = -g with D = diag(H) clamped to [1e-6, 1e32]; the
  landmarks are eliminated with the dense Schur complement
  S = U_l - W V_l^-1 W^T, b = -g_c + W V_l^-1 g_p, S dc = b (Cholesky), then
  dp = V_l^-1 (-g_p - W^T dc).  A candidate whose cost is below the current
  one is accepted and lambda is divided by 10, otherwise the state is kept and
  lambda is multiplied by 10.  One iteration = one linearisation, one damped
  solve and one accept/reject decision; the count is fixed (no early stop).
"""
from __future__ import annotations

from typing import Dict

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

Z_MIN = 1e-6
D_MIN, D_MAX = 1e-6, 1e32


def rodrigues(w) -> np.ndarray:
    """Exp map of so(3): rotation by |w| about w/|w| (Rodrigues' formula)."""
    w = np.asarray(w, np.float64)
    th = np.linalg.norm(w)
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / (th * th) * (K @ K)


def split_poses(poses):
    P = np.asarray(poses, np.float64).reshape(-1, 3, 4)
    return P[:, :, :3].copy(), P[:, :, 3].copy()


def join_poses(R, t) -> np.ndarray:
    return np.concatenate([R, t[:, :, None]], axis=2).reshape(-1, 12)


def residuals(R, t, X, f, obs_cam, obs_uv, cx, cy):
    """r [P, M, 2] and validity [P, M] of every observation slot (slot with
    camera -1 or depth <= Z_MIN is invalid, r = 0 there)."""
    obs_cam = np.asarray(obs_cam)
    valid = obs_cam >= 0
    c = np.where(valid, obs_cam, 0)
    Xc = np.einsum("pmij,pj->pmi", R[c], X) + t[c]
    z = Xc[..., 2]
    valid &= z > Z_MIN
    zs = np.where(valid, z, 1.0)
    u = f * Xc[..., 0] / zs + cx
    v = f * Xc[..., 1] / zs + cy
    r = np.stack([u, v], axis=-1) - np.asarray(obs_uv, np.float64)
    r[~valid] = 0.0
    return r, valid


def cost(R, t, X, f, obs_cam, obs_uv, cx, cy) -> float:
    r, _ = residuals(R, t, X, f, obs_cam, obs_uv, cx, cy)
    return float(np.sum(r * r))


def layout(num_cams, fixed, opt_focal, num_points):
    """Column index of each free keyframe's 6-block (-1 if fixed), of f (-1 if
    not optimised), the first landmark column and the total column count."""
    fixed = np.asarray(fixed, bool)
    cam_col = -np.ones(num_cams, np.int64)
    nc = 0
    for k in range(num_cams):
        if not fixed[k]:
            cam_col[k] = nc
            nc += 6
    f_col = nc if opt_focal else -1
    nc += 1 if opt_focal else 0
    return cam_col, f_col, nc, nc + 3 * num_points


def jacobian(R, t, X, f, obs_cam, fixed, opt_focal):
    """Sparse J [2 * P * M, columns] of the residual vector (observation slots
    in [P][M] order, u then v) with respect to the update parameters; the
    blocks of one observation, with (x, y, z) = R X + t and
    dpi = d(u, v)/d(x, y, z) = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]]:
    dX -> dpi R, dtheta -> dpi (-[R X]x) (derivative of Exp(w) R X at w = 0),
    dt -> dpi, df -> (x/z, y/z)."""
    obs_cam = np.asarray(obs_cam)
    P, M = obs_cam.shape
    cam_col, f_col, n_cam_cols, ncol = layout(R.shape[0], fixed, opt_focal, P)
    _, valid = residuals(R, t, X, f, obs_cam, np.zeros((P, M, 2)), 0.0, 0.0)
    p_idx, m_idx = np.nonzero(valid)
    k = obs_cam[p_idx, m_idx]
    RX = np.einsum("nij,nj->ni", R[k], X[p_idx])
    x, y, z = (RX + t[k]).T
    zero = np.zeros_like(z)
    dpi = np.stack([np.stack([f / z, zero, -f * x / (z * z)], -1),
                    np.stack([zero, f / z, -f * y / (z * z)], -1)], 1)          # [n, 2, 3]
    skew = np.stack([np.stack([zero, -RX[:, 2], RX[:, 1]], -1),
                     np.stack([RX[:, 2], zero, -RX[:, 0]], -1),
                     np.stack([-RX[:, 1], RX[:, 0], zero], -1)], 1)           # [R X]x
    row0 = 2 * (p_idx * M + m_idx)
    rows, cols, vals = [], [], []

    def put(col0, B, sel=slice(None)):
        n, _, w = B.shape
        rr = row0[sel][:, None, None] + np.arange(2)[None, :, None] + np.zeros((1, 1, w), np.int64)
        cc = col0[:, None, None] + np.arange(w)[None, None, :] + np.zeros((1, 2, 1), np.int64)
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(B.ravel())

    put(n_cam_cols + 3 * p_idx, dpi @ R[k])
    free = cam_col[k] >= 0
    put(cam_col[k][free], -(dpi[free] @ skew[free]), free)
    put(cam_col[k][free] + 3, dpi[free], free)
    if f_col >= 0:
        put(np.full(len(z), f_col), np.stack([x / z, y / z], -1)[:, :, None])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(2 * P * M, ncol))


def damped_system(J, r, lam):
    """H + lambda D (sparse) and g = J^T r with D = diag(H) clamped to
    [D_MIN, D_MAX]."""
    H = (J.T @ J).tocsr()
    g = J.T @ r.reshape(-1)
    D = np.clip(H.diagonal(), D_MIN, D_MAX)
    return (H + sp.diags(lam * D)).tocsr(), g


def schur_step(Hd, g, n_cam_cols, num_points):
    """Solve Hd delta = -g by eliminating the landmark blocks (block-diagonal
    3x3 V_l) with the dense Schur complement; returns (delta, S, b) or None if
    S is not positive definite."""
    U = Hd[:n_cam_cols, :n_cam_cols].toarray()
    W = Hd[:n_cam_cols, n_cam_cols:]
    V = Hd[n_cam_cols:, n_cam_cols:]
    gc, gp = g[:n_cam_cols], g[n_cam_cols:]
    Vblocks = np.stack([V[3 * p:3 * p + 3, 3 * p:3 * p + 3].toarray() for p in range(num_points)])
    ii, jj = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    base = 3 * np.arange(num_points)[:, None, None]
    Vinv = sp.csr_matrix((np.linalg.inv(Vblocks).ravel(), ((base + ii).ravel(), (base + jj).ravel())),
                         shape=(3 * num_points, 3 * num_points))
    S = U - (W @ Vinv @ W.T).toarray()
    b = -gc + W @ (Vinv @ gp)
    try:
        cf = sla.cho_factor(S, lower=True)
    except np.linalg.LinAlgError:
        return None
    dc = sla.cho_solve(cf, b)
    dp = Vinv @ (-gp - W.T @ dc)
    return np.concatenate([dc, dp]), S, b


def retract(R, t, X, f, delta, cam_col, f_col, n_cam_cols):
    """Apply an update (Exp on the left of R, additive on t, X, f)."""
    R, t, X = R.copy(), t.copy(), X.copy()
    for k in range(R.shape[0]):
        c = cam_col[k]
        if c >= 0:
            R[k] = rodrigues(delta[c:c + 3]) @ R[k]
            t[k] = t[k] + delta[c + 3:c + 6]
    if f_col >= 0:
        f = f + delta[f_col]
    X = X + delta[n_cam_cols:].reshape(-1, 3)
    return R, t, X, f


def solve(poses, points, f, obs_cam, obs_uv, cx, cy, fixed, opt_focal=True, iters=10,
          lambda0=1e-3) -> Dict[str, np.ndarray]:
    """Run `iters` Levenberg-Marquardt iterations; returns the final poses
    [N][12], points [P][3], f, and per iteration the cost at the current state,
    the candidate's cost, lambda used and the accept flag."""
    R, t = split_poses(poses)
    X = np.asarray(points, np.float64).copy()
    f = float(f)
    obs_cam = np.asarray(obs_cam)
    P = X.shape[0]
    cam_col, f_col, n_cam_cols, _ = layout(R.shape[0], fixed, opt_focal, P)
    lam = float(lambda0)
    trace = np.zeros((iters, 4))
    for it in range(iters):
        r, _ = residuals(R, t, X, f, obs_cam, obs_uv, cx, cy)
        E = float(np.sum(r * r))
        J = jacobian(R, t, X, f, obs_cam, fixed, opt_focal)
        Hd, g = damped_system(J, r, lam)
        out = schur_step(Hd, g, n_cam_cols, P)
        Ec, acc = np.inf, False
        if out is not None:
            Rn, tn, Xn, fn = retract(R, t, X, f, out[0], cam_col, f_col, n_cam_cols)
            Ec = cost(Rn, tn, Xn, fn, obs_cam, obs_uv, cx, cy)
            acc = Ec < E
        trace[it] = (E, Ec, lam, float(acc))
        if acc:
            R, t, X, f = Rn, tn, Xn, fn
            lam = lam * 0.1
        else:
            lam = lam * 10.0
    return {"poses": join_poses(R, t), "points": X, "f": f, "trace": trace,
            "cost": cost(R, t, X, f, obs_cam, obs_uv, cx, cy)}
