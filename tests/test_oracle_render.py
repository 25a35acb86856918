"""Pins of the oracle's forward renderer (the splat renderer of Sec. 5.2).

Each test checks the oracle against something other than itself: closed forms
of one and two isotropic Gaussians, the transmittance invariant, permutation
invariance, independence of the tile shape, the early-stop worked example in
tests/golden/, and the projected covariance against a finite-difference
Jacobian of the pinhole map with a library quaternion rotation.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Y00 = 0.5 / np.sqrt(np.pi)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.float64(x)))


def _scene(means, sigmas, opa_logits, dc, quats=None):
    n = len(means)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    sh = np.zeros((n, 3, 1), np.float32)
    sh[:, :, 0] = np.asarray(dc, np.float32)
    ls = np.log(np.asarray(sigmas, np.float64))[:, None].repeat(3, 1).astype(np.float32)
    return synth.Scene(np.asarray(means, np.float32), ls, q, np.asarray(opa_logits, np.float32), sh)


def _cam(z0, f=100.0, cx=32.0, cy=32.0, W=64, H=64):
    return synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, z0], np.float32), f, f, cx, cy, W, H)


def _closed_form_alpha(cam, m, s2, o, W, H):
    """alpha of an isotropic screen Gaussian (variance s2) at every pixel,
    with the support box [m - r, m + r]^2, r = ceil(3 sqrt(s2)), the 0.99 clamp
    and the 1/255 skip."""
    r = np.ceil(3 * np.sqrt(s2))
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5
    U, Vv = np.meshgrid(u, v)
    d2 = (U - m[0]) ** 2 + (Vv - m[1]) ** 2
    a = np.minimum(0.99, o * np.exp(-0.5 * d2 / s2))
    inside = (np.abs(U - m[0]) <= r) & (np.abs(Vv - m[1]) <= r)
    return np.where(inside & (a >= 1 / 255), a, 0.0)


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 1.0)])
def test_single_isotropic_gaussian_closed_form(bg):
    # On the optical axis with an isotropic sigma: J R Sigma R^T J^T = (f sigma / z)^2 I,
    # so the splat is isotropic with variance (f sigma / z)^2 + 0.3.
    sigma, z0, f = 0.05, 3.0, 100.0
    sc = _scene([[0, 0, 0]], [sigma], [0.7], [[0.2, 0.6, 0.9]],
                quats=[[0.3, -0.5, 0.7, 0.1]])  # isotropic: rotation is irrelevant
    cam = _cam(z0, f)
    out = oracle.render(sc, [cam], bg=bg)
    s2 = (f * np.exp(np.float64(sc.log_scales[0, 0])) / z0) ** 2 + 0.3
    a = _closed_form_alpha(cam, (32.0, 32.0), s2, _sigmoid(sc.opa_logits[0]), 64, 64)
    rgb = 0.5 + Y00 * sc.sh[0, :, 0].astype(np.float64)
    for ch in range(3):
        ref = rgb[ch] * a + (1 - a) * bg[ch]
        assert np.abs(out["image"][0][ch] - ref).max() < 1e-12
    assert np.abs(out["alpha"][0] - a).max() < 1e-12


def test_two_gaussians_closed_form():
    # Two isotropic Gaussians on the axis at depths 2 and 3: front-to-back
    # C = c1 a1 + c2 a2 (1 - a1), alpha = 1 - (1 - a1)(1 - a2).
    f = 100.0
    sc = _scene([[0, 0, -1.0], [0, 0, 0.0]], [0.04, 0.06], [1.5, 0.3],
                [[0.9, 0.1, 0.4], [0.2, 0.8, 0.3]])
    cam = _cam(3.0, f)
    out = oracle.render(sc, [cam])
    a = []
    for i, z in enumerate((2.0, 3.0)):
        s2 = (f * np.exp(np.float64(sc.log_scales[i, 0])) / z) ** 2 + 0.3
        a.append(_closed_form_alpha(cam, (32.0, 32.0), s2, _sigmoid(sc.opa_logits[i]), 64, 64))
    c = [0.5 + Y00 * sc.sh[i, :, 0].astype(np.float64) for i in range(2)]
    for ch in range(3):
        ref = c[0][ch] * a[0] + c[1][ch] * a[1] * (1 - a[0])
        assert np.abs(out["image"][0][ch] - ref).max() < 1e-12
    assert np.abs(out["alpha"][0] - (1 - (1 - a[0]) * (1 - a[1]))).max() < 1e-12


def test_early_stop_golden():
    # Worked example in tests/golden/early_stop_stack.json: centred splats
    # with alpha = 0.95 at the centre pixel; transmittance 0.05, 2.5e-3,
    # 1.25e-4, then 6.25e-6 < 1e-4, so exactly three are blended.
    with open(os.path.join(GOLDEN, "early_stop_stack.json")) as fh:
        gold = json.load(fh)
    k = gold["splats"]
    o = gold["alpha_at_centre"]
    logit = np.float32(np.log(o / (1 - o)))
    ofl = _sigmoid(logit)
    sc = _scene([[0, 0, 0.1 * i] for i in range(k)], [0.05] * k, [logit] * k,
                [[0.0, 0.0, 0.0]] * k)
    # principal point at a pixel centre so that the splat centre is exact
    cam = _cam(3.0, 100.0, cx=32.5, cy=32.5)
    out = oracle.render(sc, [cam])
    T = [1.0]
    for _ in range(k):
        T.append(T[-1] * (1 - ofl))
    nb = gold["blended"]
    assert T[nb] >= 1e-4 > T[nb + 1]
    assert abs(out["alpha"][0][32, 32] - (1 - T[nb])) < 1e-14
    for want, got in zip(gold["transmittance"], T[1:]):
        assert abs(got - want) <= 0.2 * want  # alpha is sigmoid(float32 logit), ~0.95
    # rgb = 0.5 for DC 0: colour = 0.5 (1 - T_nb)
    assert abs(out["image"][0][0, 32, 32] - 0.5 * (1 - T[nb])) < 1e-14


def test_transmittance_invariant_black_splats():
    # With every splat's colour exactly 0 and background 1, the image is the
    # final transmittance: image_c = T_final = 1 - alpha for every channel.
    sc, cams, _ = synth.plain_small(11)
    sc.sh[:, :, 0] = np.float32(-0.5 / Y00)
    out = oracle.render(sc, cams, bg=(1.0, 1.0, 1.0))
    rgb0 = 0.5 + Y00 * np.float64(sc.sh[0, 0, 0])
    assert abs(rgb0) < 1e-7 or rgb0 <= 0
    T = 1.0 - out["alpha"][0]
    assert T.min() < 0.5  # non-trivial coverage
    for ch in range(3):
        assert np.abs(out["image"][0][ch] - T).max() < 1e-6


def test_permutation_invariance_distinct_depths():
    sc, cams, _ = synth.plain_small(7)
    proj = oracle.render(sc, cams, want_proj=True)["proj"][0]
    d32 = proj[:, 10].astype(np.float32)
    # keep Gaussians whose single-precision depths are distinct
    _, first = np.unique(d32, return_index=True)
    keep = np.sort(first)
    sc = sc.subset(keep)
    ref = oracle.render(sc, cams)
    perm = np.random.default_rng(1).permutation(sc.n)
    out = oracle.render(sc.subset(perm), cams)
    assert np.abs(out["image"][0] - ref["image"][0]).max() < 1e-12
    assert np.abs(out["alpha"][0] - ref["alpha"][0]).max() < 1e-12


def test_image_independent_of_tile_shape():
    sc, cams, _ = synth.plain_small(9)
    ref = oracle.render(sc, cams, tile=(16, 16))
    for tile in ((8, 8), (32, 8), (16, 32)):
        out = oracle.render(sc, cams, tile=tile)
        assert np.array_equal(out["image"][0], ref["image"][0])
        assert np.array_equal(out["alpha"][0], ref["alpha"][0])


def _pinhole(t, cam):
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def test_projected_covariance_against_fd_jacobian():
    # Anisotropic, rotated Gaussians off the axis: the oracle's conic must be
    # the inverse of J_fd R Sigma R^T J_fd^T + 0.3 I with J_fd the central
    # finite-difference Jacobian of the pinhole map and Sigma built with scipy's
    # quaternion rotation.
    g = np.random.default_rng(2)
    n = 20
    means = g.uniform(-0.6, 0.6, (n, 3)).astype(np.float32)
    ls = g.normal(-2.5, 0.4, (n, 3)).astype(np.float32)
    q = g.normal(size=(n, 4)).astype(np.float32)
    sc = synth.Scene(means, ls, q, np.zeros(n, np.float32), np.zeros((n, 3, 1), np.float32))
    cam = synth.look_at((0.7, -0.4, -2.8), (0.1, 0.0, 0.0), 90.0, 95.0, 40.0, 30.0, 80, 64)
    proj = oracle.render(sc, [cam], want_proj=True)["proj"][0]
    R = cam.R.astype(np.float64)
    tt = cam.t.astype(np.float64)
    for i in range(n):
        assert proj[i, 0] == 1
        t = R @ means[i].astype(np.float64) + tt
        h = 1e-5
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (_pinhole(t + e, cam) - _pinhole(t - e, cam)) / (2 * h)
        qq = q[i].astype(np.float64)
        Rq = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        S = np.diag(np.exp(2 * ls[i].astype(np.float64)))
        Sig = Rq @ S @ Rq.T
        S2 = J @ R @ Sig @ R.T @ J.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S2)
        A, B, Cc = proj[i, 3], proj[i, 4], proj[i, 5]
        assert np.allclose([A, B, Cc], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-7, atol=1e-9)
        m = _pinhole(t, cam)
        assert np.allclose(proj[i, 1:3], m, rtol=0, atol=1e-9)
        # radius: ceil(3 sqrt(largest eigenvalue))
        assert proj[i, 11] == np.ceil(3 * np.sqrt(np.linalg.eigvalsh(S2).max()))


def test_window_equals_crop_of_full_render():
    # a pixel window composites exactly the same pixels as the full render
    sc, cams, _ = synth.plain_small(13)
    full = oracle.render(sc, cams)
    win = [(37, 21, 50, 30)]
    part = oracle.render(sc, cams, windows=win)
    x0, y0, w, h = win[0]
    assert np.array_equal(part["image"][0], full["image"][0][:, y0:y0 + h, x0:x0 + w])
    assert np.array_equal(part["alpha"][0], full["alpha"][0][y0:y0 + h, x0:x0 + w])
    # and the backward of a loss living in the window equals the full
    # backward with the loss gradient zero outside it
    g = np.random.default_rng(0).normal(size=(3, h, w))
    gfull = np.zeros((3, 128, 128))
    gfull[:, y0:y0 + h, x0:x0 + w] = g
    a = oracle.backward(sc, cams, [g], windows=win)
    b = oracle.backward(sc, cams, [gfull])
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(1.0, np.abs(b[k]).max())


def test_tile_rect_holds_every_pixel_that_can_blend():
    """The tile rect (tiles of [m-h, m+h], h from the alpha >= 1/255 ellipse)
    must contain every pixel whose centre lies in the support box and whose
    alpha reaches 1/255 (brute force over pixels in FP64, from the oracle's
    own conic and opacity); splats culled for low opacity reach it nowhere.
    A rect computed from the 3-sigma square alone would also pass; the check
    is that the tighter one never drops a contributing pixel."""
    sc = synth.box_scene(3000, seed=77)
    sc.opa_logits[:] = np.random.default_rng(5).normal(-1.0, 2.5, sc.n).astype(np.float32)  # many faint splats
    cams = synth.forward_trajectory(3, seed=78)[1:2]
    P = oracle.render(sc, cams, want_proj=True)["proj"][0]
    F = {k: i for i, k in enumerate(oracle.PROJ_FIELDS)}
    W, H = cams[0].width, cams[0].height
    checked = tighter = 0
    for i in range(sc.n):
        r = P[i, F["radius"]]
        if r <= 0:
            continue
        mx, my, A, B, C, o = (P[i, F[k]] for k in ("mx", "my", "A", "B", "C", "opacity"))
        x0, x1 = int(max(0, np.floor(mx - r))), int(min(W - 1, np.ceil(mx + r)))
        y0, y1 = int(max(0, np.floor(my - r))), int(min(H - 1, np.ceil(my + r)))
        if x0 > x1 or y0 > y1:
            continue
        px, py = np.meshgrid(np.arange(x0, x1 + 1) + 0.5, np.arange(y0, y1 + 1) + 0.5)
        dx, dy = mx - px, my - py
        inbox = (np.abs(dx) <= r) & (np.abs(dy) <= r)
        power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
        hit = inbox & (power <= 0) & (o * np.exp(power) >= 1.0 / 255.0)
        if P[i, F["bin_amb"]]:
            continue
        if not P[i, F["vis"]]:
            assert not hit.any(), i
            continue
        tx, ty = np.floor(px[hit] / 16).astype(int), np.floor(py[hit] / 16).astype(int)
        assert np.all(tx >= P[i, F["xlo"]]) and np.all(tx <= P[i, F["xhi"]]), i
        assert np.all(ty >= P[i, F["ylo"]]) and np.all(ty <= P[i, F["yhi"]]), i
        checked += int(hit.any())
        full = (int(np.floor(max(0, mx - r) / 16)), int(min(W // 16 - 1, np.floor((mx + r) / 16))))
        tighter += int(P[i, F["xhi"]] - P[i, F["xlo"]] < full[1] - full[0])
    assert checked > 200 and tighter > 0.2 * checked, (checked, tighter)
