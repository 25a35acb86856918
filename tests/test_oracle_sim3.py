"""Pins of the oracle of the loop-closure update (every Gaussian moves with
the Sim(3) correction of its spawning keyframe): a closed form, scipy's
rotation algebra, and the invariance of the rendered image when the scene and
the camera move together."""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import synth


def _sim3(g):
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([q, g.normal(size=3), [np.exp(g.normal(0, 0.3))]])


def test_closed_form_quarter_turn():
    S = [np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4), 1, 2, 3, 2.0]
    mu, ls, q = oracle.sim3_update([[1.0, 0, 0], [0, 0, 5.0]], np.zeros((2, 3)), [[1.0, 0, 0, 0]] * 2, [0, -1], [S])
    assert np.allclose(mu, [[1, 4, 3], [0, 0, 5]], atol=1e-14)
    assert np.allclose(ls, [[np.log(2)] * 3, [0, 0, 0]], atol=1e-15)
    assert np.allclose(q, [[np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)], [1, 0, 0, 0]], atol=1e-15)


def test_against_scipy_per_keyframe():
    g = np.random.default_rng(1)
    n, K = 500, 4
    mu = g.normal(size=(n, 3))
    ls = g.normal(-3, 0.5, size=(n, 3))
    q = g.normal(size=(n, 4))
    kf = g.integers(-1, K, n)
    S = np.stack([_sim3(g) for _ in range(K)])
    mu2, ls2, q2 = oracle.sim3_update(mu, ls, q, kf, S)
    for i in range(n):
        if kf[i] < 0:
            assert np.array_equal(mu2[i], mu[i]) and np.array_equal(q2[i], q[i]) and np.array_equal(ls2[i], ls[i])
            continue
        s = S[kf[i]]
        Rs = Rotation.from_quat([s[1], s[2], s[3], s[0]])
        assert np.allclose(mu2[i], s[7] * Rs.apply(mu[i]) + s[4:7], atol=1e-12)
        assert np.allclose(ls2[i], ls[i] + np.log(s[7]), atol=1e-14)
        Rg = Rotation.from_quat([q[i, 1], q[i, 2], q[i, 3], q[i, 0]])
        ref = (Rs * Rg).as_matrix()
        got = Rotation.from_quat([q2[i, 1], q2[i, 2], q2[i, 3], q2[i, 0]]).as_matrix()
        assert np.allclose(got, ref, atol=1e-12)
        # the quaternion keeps the input's norm (the renderer normalises)
        assert abs(np.linalg.norm(q2[i]) - np.linalg.norm(q[i])) < 1e-12


def test_render_invariant_when_scene_and_camera_move_together():
    """x' = s R x + t for every Gaussian and the camera pose R_c' = R_c R^T,
    t_c' = s t_c - R_c R^T t: camera-space points scale by s, which the
    pinhole projection, the 2D covariance and the depth order absorb (SH
    degree 0: the colour does not depend on the view direction)."""
    sc, cams, _ = synth.plain_small()
    g = np.random.default_rng(2)
    S = _sim3(g)
    S[7] = 1.7  # >= 1 keeps every Gaussian on the same side of the near plane
    mu, ls, q = oracle.sim3_update(sc.means, sc.log_scales, sc.quats, np.zeros(sc.n, np.int64), S[None])
    moved = synth.Scene(mu, ls, q, np.asarray(sc.opa_logits, np.float64), np.asarray(sc.sh, np.float64))
    R = Rotation.from_quat([S[1], S[2], S[3], S[0]]).as_matrix()
    c = cams[0]
    Rc = np.asarray(c.R, np.float64)
    tc = np.asarray(c.t, np.float64)
    cam2 = synth.Camera(Rc @ R.T, S[7] * tc - Rc @ R.T @ S[4:7], c.fx, c.fy, c.cx, c.cy, c.width, c.height)
    a = oracle.render(sc, [c])
    b = oracle.render(moved, [cam2])
    ok = ((a["flags"][0] | b["flags"][0]) & 1) == 0
    assert np.abs(a["image"][0] - b["image"][0])[:, ok].max() < 1e-9
    assert np.abs(a["alpha"][0] - b["alpha"][0])[ok].max() < 1e-9
