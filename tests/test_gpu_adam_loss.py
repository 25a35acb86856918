"""GPU parity of the fused Adam step (with per-group and per-lane learning
rates and the pose step T <- Exp(xi) T) against the FP64 oracle, of the
device step counters against host steps, and of the image loss against its
definition."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import raster, synth
from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


def _lr_per_element(arena, groups):
    lr = np.zeros(arena.padded)
    inside = np.zeros(arena.padded, bool)
    for G in groups:  # first matching group wins, as in the kernel
        for e in range(G.begin, G.end):
            if not inside[e]:
                lr[e] = G.lr[(e - G.begin) & 3]
                inside[e] = True
    return lr, inside


def test_adam_matches_oracle(cuda_device):
    ensure_built()
    sc = synth.random_scene(1001, 3, 2, (-1, -1, -1), (1, 1, 1), -3.0, 0.5)  # odd n: ragged tail
    p = raster.Arena.from_scene(sc, cuda_device)
    g, m, v = p.like(), p.like(), p.like()
    groups = p.adam_groups(lr_means=1e-2, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3, lr_sh_dc=2.5e-3,
                           lr_sh_rest=1.25e-4)
    lr, inside = _lr_per_element(p, groups)
    P = p.buf.cpu().numpy().astype(np.float64)
    M = np.zeros_like(P)
    Vv = np.zeros_like(P)
    rng = np.random.default_rng(0)
    for step in range(1, 5):
        grad = (rng.normal(size=p.padded) * 10.0 ** rng.uniform(-4, 0, p.padded)).astype(np.float32)
        g.buf.copy_(torch.from_numpy(grad))
        raster.adam_step(p, g, m, v, step, groups)
        oracle.adam(P, grad.astype(np.float64) * inside, M, Vv, lr, step)
    torch.cuda.synchronize()
    Pg = p.buf.cpu().numpy().astype(np.float64)
    # each step moves a parameter by at most ~lr; FP32 rounding of p and of the update
    err = np.abs(Pg - P)
    assert np.all(err <= 1e-6 * np.abs(P) + 4 * 1e-4 * lr + 1e-7), err.max()
    # elements outside every group (the means4 padding lane has lr 0) do not move
    assert np.all(Pg[~inside] == p.buf.cpu().numpy()[~inside])


def test_pose_step_matches_oracle(cuda_device):
    ensure_built()
    cams = synth.loop_views(4, seed=3)
    poses = raster.poses_tensor(cams, cuda_device)
    P = np.stack([c.pose12() for c in cams]).astype(np.float64)
    arena = raster.Arena(4, 0, cuda_device)
    dummy = arena.like()
    m, v = arena.like(), arena.like()
    pm = torch.zeros((4, 6), dtype=torch.float32, device=cuda_device)
    pv = torch.zeros_like(pm)
    M = np.zeros((4, 6))
    Vv = np.zeros((4, 6))
    rng = np.random.default_rng(1)
    for step in range(1, 4):
        gp = rng.normal(size=(4, 6)).astype(np.float32)
        dpose = torch.from_numpy(gp).to(cuda_device)
        raster.adam_step(arena, dummy, m, v, step, arena.adam_groups(), pose=poses, dpose=dpose, pose_m=pm,
                         pose_v=pv, pose_lr=1e-2)
        oracle.pose_adam(P, gp.astype(np.float64), M, Vv, 1e-2, step)
    torch.cuda.synchronize()
    assert np.abs(poses.cpu().numpy() - P).max() < 2e-5


def test_device_step_counter_equals_host_steps(cuda_device):
    ensure_built()
    sc = synth.random_scene(512, 9, 1, (-1, -1, -1), (1, 1, 1), -3.0, 0.5)
    a = raster.Arena.from_scene(sc, cuda_device)
    b = raster.Arena.from_scene(sc, cuda_device)
    ga = a.like()
    ma, va, mb, vb = a.like(), a.like(), b.like(), b.like()
    step = torch.zeros(1, dtype=torch.int32, device=cuda_device)
    groups = a.adam_groups()
    rng = np.random.default_rng(2)
    for s in range(1, 4):
        ga.buf.copy_(torch.from_numpy(rng.normal(size=a.padded).astype(np.float32)))
        raster.adam_step(a, ga, ma, va, s, groups)
        raster.adam_step(b, ga, mb, vb, 0, groups, step_dev=step)
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    assert torch.equal(a.buf, b.buf)


@pytest.mark.parametrize("kind", [0, 1])
def test_image_loss(cuda_device, kind):
    ensure_built()
    rng = np.random.default_rng(kind)
    n = 3 * 130 * 70 + 5
    img = rng.random(n).astype(np.float32)
    tgt = rng.random(n).astype(np.float32)
    tgt[:7] = img[:7]  # exact ties: zero L1 gradient
    li = raster.ImageLoss(cuda_device)
    it = torch.from_numpy(img).to(cuda_device)
    tt = torch.from_numpy(tgt).to(cuda_device)
    grad = torch.empty_like(it)
    loss = float(li(it, tt, grad, kind).item())
    d = img.astype(np.float64) - tgt
    if kind == 0:
        ref, gref = np.abs(d).mean(), np.sign(d) / n
    else:
        ref, gref = (d * d).mean(), 2 * d / n
    assert abs(loss - ref) <= 1e-6 * ref
    assert np.abs(grad.cpu().numpy() - gref).max() <= 1e-6 * np.abs(gref).max()
    # deterministic
    loss2 = float(li(it, tt, grad, kind).item())
    assert loss2 == loss
