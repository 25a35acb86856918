"""Pins of the oracle's hand-derived analytic backward (the renderer's gradient
to means, log-scales, quaternions, opacity logits, SH and the camera pose).

  * forward-mode dual numbers through the same forward give exact directional
    derivatives; the analytic gradient must agree to rounding (1e-10 relative),
    per parameter group and for the 6-DoF pose of every view;
  * central finite differences (h = 1e-4) of the FP64 forward, pose moved by
    Exp(+-h e_k) T, must agree to 1e-6 relative.  Pixels whose decisions sit
    near a threshold (support edge, 1/255 skip, stop, clamps) are masked out of
    the loss so that +-h crosses no discrete decision (including a swap of
    the blend order of two splats at nearly equal depth).
"""
import numpy as np
import pytest

import oracle
from paper_2607_14481_b300 import synth

GROUPS = ("means", "log_scales", "quats", "opa_logits", "sh")


def _scene_arrays(sc):
    return {"means": sc.means, "log_scales": sc.log_scales, "quats": sc.quats,
            "opa_logits": sc.opa_logits, "sh": sc.sh}


@pytest.fixture(scope="module")
def diff_case():
    sc, cams, targets = synth.diffcheck()
    base = oracle.render(sc, cams)
    # MSE loss (the smooth reading of the differentiation-check loss)
    loss, dimg = oracle.mse_loss(base["image"], targets)
    return sc, cams, targets, dimg


def _dot_image(w, imgs):
    return float(sum((np.asarray(a) * b).sum() for a, b in zip(w, imgs)))


def test_analytic_matches_dual_numbers_per_group(diff_case):
    sc, cams, _, dimg = diff_case
    g = oracle.backward(sc, cams, dimg)
    rng = np.random.default_rng(0)
    arrays = _scene_arrays(sc)
    V = len(cams)
    for group in GROUPS + ("pose",):
        for trial in range(2):
            tan = {k: np.zeros(v.shape) for k, v in arrays.items()}
            tp = np.zeros((V, 6))
            if group == "pose":
                tp = rng.normal(size=(V, 6))
                pred = float((g["pose"] * tp).sum())
            else:
                tan[group] = rng.normal(size=arrays[group].shape)
                pred = float((g[group] * tan[group]).sum())
            d = oracle.render_dual(sc, tan, tp, cams)
            exact = _dot_image(dimg, d["image_tan"])
            scale = max(abs(exact), 1e-30)
            assert abs(pred - exact) <= 1e-10 * scale + 1e-18, (group, pred, exact)


def test_dual_numbers_with_alpha_output(diff_case):
    sc, cams, _, dimg = diff_case
    rng = np.random.default_rng(4)
    dal = [rng.normal(size=(c.height, c.width)) for c in cams]
    g = oracle.backward(sc, cams, dimg, dalpha=dal, bg=(0.3, 0.6, 0.9))
    arrays = _scene_arrays(sc)
    tan = {k: rng.normal(size=v.shape) for k, v in arrays.items()}
    tp = rng.normal(size=(len(cams), 6))
    d = oracle.render_dual(sc, tan, tp, cams, bg=(0.3, 0.6, 0.9))
    exact = _dot_image(dimg, d["image_tan"]) + _dot_image(dal, d["alpha_tan"])
    pred = sum(float((g[k] * tan[k]).sum()) for k in GROUPS) + float((g["pose"] * tp).sum())
    assert abs(pred - exact) <= 1e-10 * abs(exact)


def _masked_weights(sc, cams, dimg):
    # generous margins: +-h = 1e-4 must not reach any decision
    wide = oracle.render(sc, cams, margins=[0.05, 0.02, 0.02, 1e-3, 0.02, 0.02, 1e-4])
    return [np.where(f[None] != 0, 0.0, w) for f, w in zip(wide["flags"], dimg)], wide


def test_finite_differences(diff_case):
    sc, cams, _, dimg = diff_case
    w, wide = _masked_weights(sc, cams, dimg)
    assert sum(int((f != 0).sum()) for f in wide["flags"]) < 0.2 * sum(f.size for f in wide["flags"])
    g = oracle.backward(sc, cams, w)
    h = 1e-4
    rng = np.random.default_rng(1)

    def L(scn, cs):
        return _dot_image(w, oracle.render(scn, cs)["image"])

    for group in GROUPS:
        arr = _scene_arrays(sc)[group]
        flat_idx = rng.choice(arr.size, size=min(10, arr.size), replace=False)
        gmax = np.abs(g[group]).max()
        for fi in flat_idx:
            idx = np.unravel_index(fi, arr.shape)
            vals = []
            for s in (+1, -1):
                sp = sc.copy()
                a = _scene_arrays(sp)[group].astype(np.float64)
                a[idx] += s * h
                # the oracle consumes float64 values directly
                setattr(sp, group, a)
                vals.append(L(sp, cams))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[group][idx]) <= 1e-6 * gmax + 1e-12, (group, idx, fd, g[group][idx])

    gmax = np.abs(g["pose"]).max()
    for v in range(len(cams)):
        for k in range(6):
            vals = []
            for s in (+1, -1):
                xi = np.zeros(6)
                xi[k] = s * h
                Re, te = oracle.se3_exp(xi)
                cs = list(cams)
                c = cams[v]
                R = Re @ c.R.astype(np.float64)
                t = Re @ c.t.astype(np.float64) + te
                cs[v] = synth.Camera(R, t, c.fx, c.fy, c.cx, c.cy, c.width, c.height)
                vals.append(L(sc, cs))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g["pose"][v, k]) <= 1e-6 * gmax + 1e-12, (v, k, fd, g["pose"][v, k])


def test_l1_gradient_plain_small():
    # L1 loss on the 4k-Gaussian single view: analytic against dual numbers
    sc, cams, targets = synth.plain_small()
    base = oracle.render(sc, cams)
    _, dimg = oracle.l1_loss(base["image"], targets)
    g = oracle.backward(sc, cams, dimg)
    rng = np.random.default_rng(3)
    tan = {k: rng.normal(size=v.shape) for k, v in _scene_arrays(sc).items()}
    tp = rng.normal(size=(1, 6))
    d = oracle.render_dual(sc, tan, tp, cams)
    exact = _dot_image(dimg, d["image_tan"])
    pred = sum(float((g[k] * tan[k]).sum()) for k in GROUPS) + float((g["pose"] * tp).sum())
    assert abs(pred - exact) <= 1e-10 * abs(exact)
