"""Pins of the FP64 level-of-detail oracle (coarse nodes merge up to 8
children by moment matching; the cut descends from the roots until a node's
screen size is below tau or a leaf is reached), against closed forms, Monte
Carlo moments of the mixture, a pure-Python bit interleave and a recursive
descent written independently of the oracle."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import synth


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def _cov(log_scales, quat):
    R = Rotation.from_quat([quat[1], quat[2], quat[3], quat[0]]).as_matrix()
    return R @ np.diag(np.exp(2 * np.asarray(log_scales))) @ R.T


# ---------------------------------------------------------------------------
# merge
# ---------------------------------------------------------------------------
def test_merge_cube_corners_closed_form():
    a, s, o = 0.7, 0.05, 0.3
    mu = np.array([[x, y, z] for x in (-a, a) for y in (-a, a) for z in (-a, a)])
    sh = np.random.default_rng(1).normal(size=(8, 12))
    r = oracle.lod_merge(mu, np.full((8, 3), np.log(s)), np.tile([1.0, 0, 0, 0], (8, 1)), np.full(8, o), sh)
    assert np.allclose(r["mean"], 0.0, atol=1e-15)
    assert np.allclose(r["cov"], (s * s + a * a) * np.eye(3), rtol=1e-13, atol=1e-15)
    assert np.allclose(r["sh"], sh.mean(axis=0), rtol=1e-13)
    assert abs(_sig(r["opa_logit"]) - _sig(o)) < 1e-13


def test_merge_identical_children_identity():
    g = np.random.default_rng(2)
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    ls = np.array([-2.0, -2.7, -3.1])
    mu = np.array([0.3, -1.2, 2.5])
    sh = g.normal(size=48)
    for k in (1, 3, 8):
        r = oracle.lod_merge(np.tile(mu, (k, 1)), np.tile(ls, (k, 1)), np.tile(q, (k, 1)), np.full(k, 0.4),
                             np.tile(sh, (k, 1)))
        assert np.allclose(r["mean"], mu, rtol=1e-14)
        assert np.allclose(r["cov"], _cov(ls, q), rtol=1e-12, atol=1e-16)
        assert np.allclose(r["sh"], sh, rtol=1e-13)
        assert abs(r["opa_logit"] - 0.4) < 1e-12


def test_merge_weighted_two_children_closed_form():
    mu = np.array([[0.0, 0.0, 0.0], [2.0, -1.0, 0.5]])
    o = np.array([-1.0, 1.5])
    w = _sig(o)
    r = oracle.lod_merge(mu, np.full((2, 3), -3.0), np.tile([1.0, 0, 0, 0], (2, 1)), o, np.array([[1.0], [3.0]]))
    assert np.allclose(r["mean"], (w[0] * mu[0] + w[1] * mu[1]) / w.sum(), rtol=1e-14)
    assert abs(_sig(r["opa_logit"]) - (w * w).sum() / w.sum()) < 1e-13
    assert abs(r["sh"][0] - (w[0] * 1.0 + w[1] * 3.0) / w.sum()) < 1e-13
    d = mu[1] - mu[0]
    spread = w[0] * w[1] / w.sum() ** 2 * np.outer(d, d)
    assert np.allclose(r["cov"], np.exp(-6.0) * np.eye(3) + spread, rtol=1e-12)


def test_merge_matches_mixture_moments_monte_carlo():
    """The parent's mean and covariance are the first two moments of the
    children's mixture with weights proportional to opacity (sampled)."""
    g = np.random.default_rng(3)
    k = 8
    mu = g.normal(size=(k, 3))
    ls = g.normal(-1.5, 0.4, size=(k, 3))
    q = g.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = g.normal(0.0, 1.5, size=k)
    r = oracle.lod_merge(mu, ls, q, o, np.zeros((k, 3)))
    w = _sig(o) / _sig(o).sum()
    N = 2_000_000
    comp = g.choice(k, size=N, p=w)
    pts = np.empty((N, 3))
    for i in range(k):
        sel = comp == i
        L = np.linalg.cholesky(_cov(ls[i], q[i]))
        pts[sel] = mu[i] + g.normal(size=(sel.sum(), 3)) @ L.T
    m = pts.mean(axis=0)
    C = np.cov(pts.T)
    scale = np.abs(r["cov"]).max()
    assert np.abs(m - r["mean"]).max() < 5 * np.sqrt(scale / N) * 3
    assert np.abs(C - r["cov"]).max() < 6e-3 * scale
    # uniform weights would be far off (pins w = opacity)
    mu_uniform = mu.mean(axis=0)
    assert np.abs(mu_uniform - r["mean"]).max() > 20 * np.sqrt(scale / N)


def test_merge_factors_reconstruct_covariance():
    g = np.random.default_rng(4)
    for _ in range(20):
        k = int(g.integers(1, 9))
        q = g.normal(size=(k, 4))
        r = oracle.lod_merge(g.normal(size=(k, 3)), g.normal(-2, 0.5, size=(k, 3)), q, g.normal(size=k),
                             np.zeros((k, 3)))
        assert abs(np.linalg.norm(r["quat"]) - 1) < 1e-14 and r["quat"][0] >= 0
        assert np.allclose(_cov(r["log_scales"], r["quat"]), r["cov"], rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------------------
# grouping
# ---------------------------------------------------------------------------
def _py_morton(m32):
    lo = m32.min(axis=0)
    hi = m32.max(axis=0)
    codes = []
    for p in m32:
        qs = []
        for a in range(3):
            ext = np.float32(hi[a] - lo[a])
            scale = np.float32(1024.0) / ext if ext > 0 else np.float32(0.0)
            t = np.float32(np.float32(p[a] - lo[a]) * scale)
            qs.append(int(min(1023, max(0, np.floor(t)))))
        c = 0
        for bit in range(10):
            for a in range(3):
                c |= ((qs[a] >> bit) & 1) << (3 * bit + a)
        codes.append(c)
    return np.array(codes, np.uint32)


def test_morton_codes_and_order_against_bit_interleave():
    g = np.random.default_rng(5)
    m32 = g.uniform(-3, 5, size=(500, 3)).astype(np.float32)
    m32[:40] = m32[40:80]  # duplicates: equal codes keep index order
    code, order = oracle.lod_morton(m32)
    ref = _py_morton(m32)
    assert np.array_equal(code, ref)
    assert np.array_equal(order, np.array(sorted(range(500), key=lambda i: (int(ref[i]), i))))


def test_build_structure_and_parent_parameters():
    sc = synth.random_scene(300, 6, 1, (-1, -1, -1), (1, 1, 1), -3.0, 0.4)
    b = oracle.lod_build(sc)
    n, n1, n2 = sc.n, b["n1"], b["n2"]
    assert (n1, n2) == (38, 5)
    par = b["parent"]
    assert np.all(par[:n] >= n) and np.all(par[:n] < n + n1)
    assert np.all(par[n:n + n1] >= n + n1) and np.all(par[n + n1:] == -1)
    _, order = oracle.lod_morton(np.asarray(sc.means, np.float32))
    for g in range(n1):
        kids = order[8 * g:8 * g + 8]
        assert np.all(par[kids] == n + g)
        r = oracle.lod_merge(sc.means[kids], sc.log_scales[kids], sc.quats[kids], sc.opa_logits[kids],
                             np.asarray(sc.sh[kids], np.float64).reshape(len(kids), -1))
        assert np.allclose(b["means"][g], r["mean"], rtol=1e-13, atol=1e-15)
        assert np.allclose(b["cov"][g], r["cov"], rtol=1e-12, atol=1e-16)
        assert np.allclose(b["sh"][g].reshape(-1), r["sh"], rtol=1e-12, atol=1e-15)
    for g in range(n2):
        kids = np.arange(8 * g, min(n1, 8 * g + 8))
        assert np.all(par[n + kids] == n + n1 + g)
        r = oracle.lod_merge(b["means"][kids], b["log_scales"][kids], b["quats"][kids], b["opa_logits"][kids],
                             b["sh"][kids].reshape(len(kids), -1))
        assert np.allclose(b["cov"][n1 + g], r["cov"], rtol=1e-10, atol=1e-16)


# ---------------------------------------------------------------------------
# the cut
# ---------------------------------------------------------------------------
def _nodes(sc, b):
    means = np.concatenate([np.asarray(sc.means, np.float64), b["means"]])
    ls = np.concatenate([np.asarray(sc.log_scales, np.float64), b["log_scales"]])
    return means, ls


def _descent(means, ls, parent, n_leaf, cam, tau, znear=0.2):
    """Recursive descent from the roots (independent of the oracle)."""
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    children = {}
    for i, p in enumerate(parent):
        children.setdefault(int(p), []).append(i)
    out = set()

    def S(i):
        tz = R[2] @ means[i] + t[2]
        return np.inf if tz <= znear else cam.fx * 3.0 * np.exp(ls[i].max()) / tz

    def visit(i):
        if i < n_leaf or S(i) < tau:
            out.add(i)
        else:
            for c in children.get(i, []):
                visit(c)

    for r in children[-1]:
        visit(r)
    return out


@pytest.mark.parametrize("dist,tau", [(7.0, 1.0), (20.0, 16.0), (40.0, 16.0), (40.0, 40.0)])
def test_cut_matches_recursive_descent(dist, tau):
    sc = synth.random_scene(3000, 7, 0, (-4, -1, -4), (4, 1, 4), -2.5, 0.5)
    b = oracle.lod_build(sc)
    means, ls = _nodes(sc, b)
    cam = synth.look_at((0.0, -0.5, -dist), (0, 0, 0), 300.0, 300.0, 160, 120, 320, 240)
    r = oracle.lod_cut(means, ls, b["parent"], sc.n, cam, tau=tau)
    ref = _descent(means, ls, b["parent"], sc.n, cam, tau)
    assert set(np.flatnonzero(r["selected"]).tolist()) == ref
    # a partition of the leaves: each leaf has exactly one selected node among
    # itself and its ancestors
    par = b["parent"]
    for i in range(sc.n):
        chain = [i]
        while par[chain[-1]] >= 0:
            chain.append(int(par[chain[-1]]))
        assert r["selected"][chain].sum() == 1
    if dist > 10:
        assert 0 < (r["selected"][sc.n:]).sum()  # far away, coarse nodes are used


def test_cut_extremes_and_screen_size_closed_form():
    sc = synth.random_scene(500, 8, 0, (-1, -1, -1), (1, 1, 1), -3.0, 0.3)
    b = oracle.lod_build(sc)
    means, ls = _nodes(sc, b)
    cam = synth.look_at((0.0, 0.0, -6.0), (0, 0, 0), 200.0, 200.0, 100, 100, 200, 200)
    r0 = oracle.lod_cut(means, ls, b["parent"], sc.n, cam, tau=0.0)
    assert np.array_equal(np.flatnonzero(r0["selected"]), np.arange(sc.n))
    rinf = oracle.lod_cut(means, ls, b["parent"], sc.n, cam, tau=1e30)
    roots = np.flatnonzero(b["parent"] == -1)
    assert np.array_equal(np.flatnonzero(rinf["selected"]), roots)
    # S = 3 f sigma_max / z for a node straight ahead
    one = np.array([[0.0, 0.0, 0.0]])
    cam2 = synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 4.0], np.float32), 250.0, 250.0, 50, 50,
                        100, 100)
    r = oracle.lod_cut(one, np.log([[0.02, 0.05, 0.01]]), np.array([-1]), 1, cam2, tau=1.0)
    assert abs(r["screen"][0] - 3 * 250.0 * 0.05 / 4.0) < 1e-12
    # behind the near plane: infinitely large, never coarse enough
    cam3 = synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 0.1], np.float32), 250.0, 250.0, 50, 50,
                        100, 100)
    r = oracle.lod_cut(one, np.log([[0.02, 0.05, 0.01]]), np.array([-1]), 0, cam3, tau=1.0)
    assert np.isinf(r["screen"][0]) and not r["selected"][0]
