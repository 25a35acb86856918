"""The training step exactly as the benchmark runs it, against the FP64 oracle
on outputs the oracle can compute one by one.  The step is 1M Gaussians, SH3,
one 1280x720 view of the forward trajectory, L1 loss and the pose step, with
the fused composite + loss + backward pass and the tile shape and schedule
its autotuner picks, replayed from a captured CUDA graph.  Checked:

- image windows of the replayed step, among them the ragged corner;
- the replayed step's Adam update of sampled Gaussians' parameters and of
  random arena elements, given its gradient;
- the gradients of 40 sampled Gaussians and of the pose.  Each sampled Gaussian
  has a window covering its whole tile rect, and the windows are disjoint.
  The replayed step's parameters, pose and tile lists are kept, and its
  backward kernels run once more, with the step's own dL/dimage restricted
  to the windows.  Pixels whose value or derivative the oracle flags as
  decided within rounding reach of a threshold are zeroed on both sides, as
  in the other full-size tests.  Each sampled Gaussian's gradient is then
  its whole gradient from its window; the pose gradient is the sum over the
  windows."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import raster, synth, train
from gpu_util import GRAD_TOL, IMG_TOL, ensure_built, rel_err

pytestmark = pytest.mark.gpu

W, H = 1280, 720


def _lr_per_element(arena, groups):
    lr = np.zeros(arena.padded)
    for G in groups:
        e = np.arange(G.begin, G.end)
        lr[e] = np.asarray(list(G.lr), np.float64)[(e - G.begin) & 3]
    return lr


def _disjoint_small_splats(rec, rng, want, tw, th):
    """Gaussians whose rect is at most 2x2 tiles (of tw x th pixels), with
    pairwise disjoint rects (their pixel windows then never overlap)."""
    touched = rec["touched"][0].astype(np.int64)
    cand = np.flatnonzero((touched >= 1) & (touched <= 4))
    rng.shuffle(cand)
    used = np.zeros((H // th + 2, W // tw + 2), bool)
    out = []
    for i in cand:
        r0, r1 = int(rec["rect"][0][i, 0]), int(rec["rect"][0][i, 1])
        x0, y0, x1, y1 = r0 & 0xFFFF, r0 >> 16, r1 & 0xFFFF, r1 >> 16
        if used[y0:y1 + 1, x0:x1 + 1].any():
            continue
        used[max(0, y0 - 1):y1 + 2, max(0, x0 - 1):x1 + 2] = True
        out.append((int(i), (tw * x0, th * y0, min(tw * (x1 + 1), W) - tw * x0, min(th * (y1 + 1), H) - th * y0)))
        if len(out) == want:
            break
    return out


def test_graph_replayed_step_1m_720p(cuda_device):
    ensure_built()
    dev = cuda_device
    sc_init = synth.box_scene(1_000_000, seed=1007)
    cam = synth.forward_trajectory(100, seed=1008)[10]
    arena = raster.Arena.from_scene(sc_init, dev)
    grads, m, v = arena.like(), arena.like(), arena.like()
    groups = arena.adam_groups(lr_means=1.6e-3)
    poses = raster.poses_tensor([cam], dev)
    pm = torch.zeros((1, 6), dtype=torch.float32, device=dev)
    pv = torch.zeros_like(pm)
    psteps = torch.zeros(1, dtype=torch.int32, device=dev)
    step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rast = raster.Rasterizer(arena.n, 3, [cam], device=dev)
    img, dimg = rast.new_image(), rast.new_image()
    rast.forward(arena, poses, img, None, check=True)
    rast.set_capacity(int(rast.read_counts()[1] * 1.3) + 4096)
    gen = torch.Generator(device="cpu").manual_seed(1009)
    target = torch.rand(3 * W * H, generator=gen).to(dev)
    loss = raster.ImageLoss(dev)
    rast.autotune_fused(arena, poses, target, 0, img, loss.loss, reps=1)
    rast.forward(arena, poses, img, None, check=True)  # pair capacity at the chosen tile shape
    rast.set_capacity(int(rast.read_counts()[1] * 1.3) + 4096)
    st = train.TrainStep(arena, grads, m, v, groups, rast, poses, target, step_dev, pose_m=pm, pose_v=pv,
                         pose_steps=psteps, pose_lr=1e-4, loss_kind=0, status=status, image=img, dimage=dimg,
                         loss=loss, cams=[cam])
    st.run()  # step 1, eager (also the capture's warm-up)
    st.capture()
    torch.cuda.synchronize()
    P0 = arena.buf.cpu().numpy().astype(np.float64)
    M0 = m.buf.cpu().numpy().astype(np.float64)
    V0 = v.buf.cpu().numpy().astype(np.float64)
    nat0 = arena.to_natural()
    pose0 = poses.cpu().numpy().reshape(3, 4)
    st.run()  # step 2: graph replay, the step under test
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and rast.read_counts()[2] == 0 and int(step_dev.item()) == 2

    sc = synth.Scene(nat0["means"].astype(np.float32), nat0["log_scales"].astype(np.float32),
                     nat0["quats"].astype(np.float32), nat0["opa_logits"].astype(np.float32),
                     nat0["sh"].astype(np.float32))
    cam0 = synth.Camera(pose0[:, :3].astype(np.float32), pose0[:, 3].astype(np.float32), cam.fx, cam.fy, cam.cx,
                        cam.cy, W, H)
    rng = np.random.default_rng(11)
    rec = rast.splat_arrays()
    # 40 samples: many small splats are hidden (zero gradient on both sides)
    # and a few barely visible ones have near-cancelling gradients, so the
    # per-group normalisation needs a broad sample
    samples = _disjoint_small_splats(rec, rng, 40, *rast.tile)
    assert len(samples) >= 30
    wins = [w for _, w in samples] + [(W - 40, H - 24, 40, 24)] + \
        [(int(rng.integers(0, W - 48)), int(rng.integers(0, H - 48)), 48, 48) for _ in range(2)]
    ref = oracle.render(sc, [cam0] * len(wins), windows=wins, tile=rast.tile)
    full = rast.split(img.cpu(), 3)[0].numpy().astype(np.float64)
    flagged = total = 0
    for k, (x0, y0, w, h) in enumerate(wins):
        ok = (ref["flags"][k] & 1) == 0
        flagged += int((~ok).sum())
        total += ok.size
        d = np.abs(full[:, y0:y0 + h, x0:x0 + w] - ref["image"][k])
        assert d[:, ok].max(initial=0.0) <= IMG_TOL, k
    assert flagged <= 0.03 * total

    # the Adam update (step 2) of the sampled Gaussians' parameters and of random elements
    ids_all = np.array([i for i, _ in samples])
    n, nc = arena.n, arena.nc
    elems = [np.concatenate([4 * ids_all + c for c in range(3)]),          # means
             np.concatenate([4 * n + 4 * ids_all + c for c in range(4)]),  # log-scales, opacity logit
             np.concatenate([8 * n + 4 * ids_all + c for c in range(4)]),  # quaternion
             np.concatenate([12 * n + q * n + ids_all for q in range(3 * nc)]),
             rng.integers(0, arena.size, 20000)]
    e = np.unique(np.concatenate(elems))
    lr = _lr_per_element(arena, groups)[e]
    G = grads.buf.cpu().numpy().astype(np.float64)[e]
    p, mm, vv = P0[e].copy(), M0[e].copy(), V0[e].copy()
    oracle.adam(p, G, mm, vv, lr, 2)
    P1 = arena.buf.cpu().numpy().astype(np.float64)[e]
    assert np.all(np.abs(P1 - p) <= 1e-6 * np.abs(p) + 4e-4 * lr + 1e-7)
    M1 = m.buf.cpu().numpy().astype(np.float64)[e]
    # m = b1 m0 + (1 - b1) g in float32: rounding relative to the terms
    assert np.all(np.abs(M1 - mm) <= 1e-6 * (0.9 * np.abs(M0[e]) + 0.1 * np.abs(G)) + 1e-30)

    # gradients: the step's backward kernels on its own tile lists, with the
    # pre-step parameters and pose and the windowed, masked dL/dimage (the L1
    # gradient of the step's image, which the fused pass formed internally)
    loss(img, target, dimg, 0)
    arena.buf.copy_(torch.from_numpy(P0.astype(np.float32)))
    poses.copy_(torch.from_numpy(pose0.reshape(1, 12).astype(np.float32)))
    gwins = [w for _, w in samples]
    dfull = rast.split(dimg.cpu(), 3)[0].numpy().astype(np.float64)
    dmask = np.zeros((3, H, W))
    dwin = []
    for k, (x0, y0, w, h) in enumerate(gwins):
        gk = np.where(ref["flags"][k][None] != 0, 0.0, dfull[:, y0:y0 + h, x0:x0 + w])
        dwin.append(gk)
        dmask[:, y0:y0 + h, x0:x0 + w] = gk
    dmask_dev = torch.from_numpy(dmask.reshape(-1).astype(np.float32)).to(dev)
    dpose = torch.full((1, 6), float("nan"), dtype=torch.float32, device=dev)
    rast.backward_pixels(dmask_dev, None, img)
    rast.backward_gaussians(arena, poses, grads, dpose)
    torch.cuda.synchronize()
    g_ref = oracle.backward(sc, [cam0] * len(gwins), dwin, windows=gwins, tile=rast.tile)
    g_gpu = grads.to_natural()
    for name in ("means", "log_scales", "quats", "opa_logits", "sh"):
        assert rel_err(g_gpu[name][ids_all], g_ref[name][ids_all]) <= GRAD_TOL, name
    assert np.abs(g_gpu["means"][ids_all]).max() > 0
    assert rel_err(dpose.cpu().numpy().astype(np.float64)[0], g_ref["pose"].sum(axis=0)) <= GRAD_TOL
