"""The fused persistent training pass (gs_render_fused: composite + image loss
+ single front-to-back backward per (view, tile) item, items taken from a
device counter) against the separate kernels and the FP64 oracle, for every
tile shape (16x16, 32x8, 8x32), splats per batch, work order and both losses.

Targets are the image plus a random offset of at least 0.02 in magnitude,
and equal to the image on pixels the oracle flags (a decision within
single-precision reach of its threshold): there the loss gradient is exactly
zero on both sides, and elsewhere its sign (L1) cannot differ between them.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import _lib, raster, synth
from gpu_util import IMG_TOL, compare_grads, ensure_built, fused_step, gpu_backward, gpu_forward, loss_grad, \
    target_near

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (32, 8), (8, 32)]


def _setup(case, tile):
    if case == "plain_small":
        sc, cams, _ = synth.plain_small()
    elif case == "diffcheck":
        sc, cams, _ = synth.diffcheck()
    else:  # ragged views of different sizes, background, SH1
        sc = synth.random_scene(3000, 77, 1, (-1, -1, -1), (1, 1, 1), -3.2, 0.4)
        eye = [(0.0, 0.0, -3.0), (0.4, -0.2, -2.8)]
        cams = [synth.look_at(e, (0, 0, 0), 90.0, 90.0, w / 2, h / 2, w, h) for e, (w, h) in
                zip(eye, [(100, 70), (77, 91)])]
    return sc, cams


def _target(r, img, ref, rng):
    tv = target_near([x.numpy() for x in r.split(img.cpu(), 3)], ref["flags"], rng)
    return tv, torch.from_numpy(np.concatenate([t.reshape(-1) for t in tv])).to(img.device)


@pytest.mark.parametrize("tile", SHAPES)
@pytest.mark.parametrize("case", ["plain_small", "diffcheck", "ragged"])
@pytest.mark.parametrize("kind", [0, 1])
def test_fused_pass_matches_separate_kernels_and_oracle(cuda_device, tile, case, kind):
    sc, cams = _setup(case, tile)
    bg = (0.2, 0.1, 0.3) if case == "ragged" else (0.0, 0.0, 0.0)
    r, arena, poses, img, alpha = gpu_forward(sc, cams, bg=bg, tile=tile)
    ref = oracle.render(sc, cams, tile=tile, bg=bg)
    rng = np.random.default_rng(11 + kind)
    tv, tgt = _target(r, img, ref, rng)
    count = 3 * r.pixels
    img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, kind)
    # the composite is the same code as gs_render_fwd: identical bits
    assert torch.equal(img_f, img)
    # the loss: the mean over all views' pixels and channels
    iv = [x.numpy().astype(np.float64) for x in r.split(img.cpu(), 3)]
    d = np.concatenate([(a - t).reshape(-1) for a, t in zip(iv, tv)])
    want = np.abs(d).mean() if kind == 0 else (d * d).mean()
    assert abs(loss_f - want) <= 1e-5 * want
    # the separate kernels with the same loss gradient
    dimg = loss_grad(iv, tv, kind, count)
    g_sep = gpu_backward(r, arena, poses, dimg, image=img)
    for k in g_sep:
        if k == "means_pad":
            continue
        scale = max(np.abs(g_sep[k]).max(), 1e-30)
        assert np.abs(g_f[k] - g_sep[k]).max() <= 1e-5 * scale, k
    # the oracle with the same upstream gradient
    g_ref = oracle.backward(sc, cams, dimg, tile=tile, bg=bg)
    compare_grads(g_f, g_ref)


@pytest.mark.parametrize("tile", SHAPES)
def test_fused_schedules_change_no_result(cuda_device, tile):
    """Splats per batch (128, 64, 32) and work order (view-major, longest
    lists first) change no bit of the image, loss or gradients; repeated runs
    are bit-identical."""
    sc, cams, _ = synth.diffcheck()
    r, arena, poses, img, alpha = gpu_forward(sc, cams, tile=tile)
    ref = oracle.render(sc, cams, tile=tile)
    _, tgt = _target(r, img, ref, np.random.default_rng(5))
    base = None
    for order in (0, 1):
        for b in (0, 1, 2):
            r.cfg.schedule = (_lib.GS_SCHED_FUSED_LONGEST_FIRST if order else 0) | _lib.GS_SCHED_FUSED_BATCH(b)
            r.bin_sort()  # the longest-first order is written by the binning
            for _ in range(2):
                got = fused_step(r, arena, poses, tgt, 0)
                if base is None:
                    base = got
                    continue
                assert torch.equal(base[0], got[0]) and base[1] == got[1], (order, b)
                for k in base[2]:
                    assert np.array_equal(base[2][k], got[2][k]), (order, b, k)


def test_fused_many_items_per_cta_three_720p_views(cuda_device):
    """Three 1280x720 views (10,800 tiles, several items per resident CTA):
    image identical to gs_render_fwd, gradients equal to the separate kernels
    and to the oracle on sampled windows."""
    sc = synth.box_scene(40_000, seed=1007)
    cams = synth.forward_trajectory(100, seed=1008)[20:23]
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    rng = np.random.default_rng(8)
    wins = [(int(rng.integers(0, 1280 - 40)), int(rng.integers(0, 720 - 40)), 40, 40) for _ in cams]
    ref = oracle.render(sc, cams, windows=wins)
    # target = image outside the windows (zero gradient there)
    iv = [x.numpy() for x in r.split(img.cpu(), 3)]
    tv = [im.copy() for im in iv]
    for t, im, f, (x0, y0, w, h) in zip(tv, iv, ref["flags"], wins):
        off = rng.uniform(0.02, 0.2, size=(3, h, w)) * rng.choice([-1.0, 1.0], size=(3, h, w))
        patch = (im[:, y0:y0 + h, x0:x0 + w].astype(np.float64) + off).astype(np.float32)
        t[:, y0:y0 + h, x0:x0 + w] = np.where((f != 0)[None], im[:, y0:y0 + h, x0:x0 + w], patch)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in tv])).to(cuda_device)
    r.cfg.schedule = _lib.GS_SCHED_FUSED_LONGEST_FIRST
    r.bin_sort()
    img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, 0)
    assert torch.equal(img_f, img)
    count = 3 * r.pixels
    dimg = loss_grad([x.astype(np.float64) for x in iv], tv, 0, count)
    g_sep = gpu_backward(r, arena, poses, dimg, image=img)
    for k in g_sep:
        if k != "means_pad":
            assert np.abs(g_f[k] - g_sep[k]).max() <= 1e-5 * max(np.abs(g_sep[k]).max(), 1e-30), k
    dwin = [d[:, y0:y0 + h, x0:x0 + w] for d, (x0, y0, w, h) in zip(dimg, wins)]
    g_ref = oracle.backward(sc, cams, dwin, windows=wins)
    compare_grads(g_f, g_ref)


def test_fused_empty_scene_and_all_culled(cuda_device):
    """No splat on screen: the image is the background, the loss that of the
    background, every gradient zero."""
    sc = synth.random_scene(64, 3, 0, (-1, -1, 5), (1, 1, 6), -3.0, 0.3)  # behind the camera at z = -3 ... +z
    cams = [synth.look_at((0, 0, 0), (0, 0, -1), 60.0, 60.0, 24.0, 20.0, 48, 40)]
    r, arena, poses, img, alpha = gpu_forward(sc, cams, bg=(0.25, 0.5, 0.75))
    assert int(r.read_counts()[1]) == 0
    tgt = torch.zeros_like(img)
    img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, 1)
    bgv = torch.tensor([0.25, 0.5, 0.75], device=cuda_device).repeat_interleave(48 * 40)
    assert torch.equal(img_f, bgv)
    assert abs(loss_f - (0.25 ** 2 + 0.5 ** 2 + 0.75 ** 2) / 3) < 1e-6
    for k in ("means", "log_scales", "quats", "opa_logits", "sh", "pose"):
        assert np.all(g_f[k] == 0.0), k


def _occluded_scene():
    """Six large, nearly opaque Gaussians in front of 2,000 small ones: every
    pixel stops within the first few list entries while each tile's list runs
    on for several batches of staged splats."""
    back = synth.random_scene(2000, 41, 1, (-0.5, -0.4, 1.5), (0.5, 0.4, 3.0), -3.5, 0.3)
    front = synth.random_scene(6, 42, 1, (-0.05, -0.05, 0.5), (0.05, 0.05, 0.8), 0.5, 0.1)
    front.opa_logits[:] = 3.0  # opacity 0.953: below the alpha clamp, no decision near a threshold
    return synth.Scene(*(np.concatenate([getattr(front, f), getattr(back, f)])
                         for f in ("means", "log_scales", "quats", "opa_logits", "sh")))


@pytest.mark.parametrize("tile", SHAPES)
def test_fused_every_pixel_stops_in_the_first_batch(cuda_device, tile):
    """Lists several batches long where every pixel stops in the first: the
    pairs past the stop get zero gradients and the result matches the
    separate kernels and the oracle at every splats-per-batch setting."""
    sc = _occluded_scene()
    cams = [synth.look_at((0, 0, 0), (0, 0, 1), 60.0, 60.0, 24.0, 20.0, 48, 40)]
    r, arena, poses, img, alpha = gpu_forward(sc, cams, tile=tile)
    ref = oracle.render(sc, cams, tile=tile)
    pairs = int(r.read_counts()[1])
    assert pairs > 2 * 128 * r.num_tiles // 3  # long lists: a few batches per tile on average
    assert not np.any(np.asarray(ref["flags"][0]))  # no decision within single-precision reach
    assert np.all(alpha.cpu().numpy() > 1.0 - 1e-3)  # every pixel saturated by the front splats
    # (the oracle's image without the back splats is the same image)
    assert np.array_equal(np.asarray(oracle.render(sc.subset(np.arange(6)), cams, tile=tile)["image"][0]),
                          np.asarray(ref["image"][0]))
    _, tgt = _target(r, img, ref, np.random.default_rng(9))
    iv = [x.numpy().astype(np.float64) for x in r.split(img.cpu(), 3)]
    tv = [x.numpy().astype(np.float64) for x in r.split(tgt.cpu(), 3)]
    dimg = loss_grad(iv, tv, 0, 3 * r.pixels)
    g_ref = oracle.backward(sc, cams, dimg, tile=tile)
    g_sep = gpu_backward(r, arena, poses, dimg, image=img)
    for b in (0, 1, 2):
        r.cfg.schedule = _lib.GS_SCHED_FUSED_BATCH(b)
        img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, 0)
        assert torch.equal(img_f, img)
        for k in g_sep:
            if k == "means_pad":
                continue
            scale = max(np.abs(g_sep[k]).max(), 1e-30)
            assert np.abs(g_f[k] - g_sep[k]).max() <= 1e-5 * scale, (b, k)
        compare_grads(g_f, g_ref)
        # the hidden splats receive nothing
        assert np.all(g_f["opa_logits"][6:] == 0.0) and np.all(g_f["sh"][6:] == 0.0), b


def test_autotune_fused_picks_a_shape_and_leaves_its_results(cuda_device):
    ensure_built()
    sc, cams, _ = synth.diffcheck()
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    ref = oracle.render(sc, cams)
    tv, tgt = _target(r, img, ref, np.random.default_rng(2))
    loss = torch.zeros(1, device=cuda_device)
    res = r.autotune_fused(arena, poses, tgt, 0, img, loss, reps=2)
    assert tuple(res["tile"]) in SHAPES and r.tile == tuple(res["tile"])
    assert (r.cfg.tile_w, r.cfg.tile_h) == r.tile
    times = [v for v in res["ms"].values() if np.isfinite(v)]
    assert len(times) >= 6 and all(t > 0 for t in times)
    # the buffers hold the chosen configuration's results: a fused step on them
    # matches the oracle at that tile shape
    img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, 0)
    ref_t = oracle.render(sc, cams, tile=r.tile)
    for a, o, f in zip(r.split(img_f.cpu(), 3), ref_t["image"], ref_t["flags"]):
        ok = (f & 1) == 0
        assert np.abs(a.numpy().astype(np.float64) - o)[:, ok].max() <= IMG_TOL
    dimg = loss_grad([x.numpy() for x in r.split(img_f.cpu(), 3)], tv, 0, 3 * r.pixels)
    compare_grads(g_f, oracle.backward(sc, cams, dimg, tile=r.tile))


def test_full_size_batched_2m_16_views_fused_every_tile_shape(cuda_device):
    """The batched workload at full size (2M Gaussians, SH3, 16 views of
    uneven resolution) through the fused pass at every tile shape the
    autotuner may pick, longest lists first: images and gradients on sampled
    windows against the oracle."""
    sc = synth.box_scene(2_000_000, seed=1007)
    cams = synth.loop_views(16, 1009)
    rng = np.random.default_rng(3)
    wins = [(int(rng.integers(0, c.width - 32)), int(rng.integers(0, c.height - 32)), 32, 32) for c in cams[:-1]]
    wins.append((cams[-1].width - 24, cams[-1].height - 20, 24, 20))  # a ragged corner
    ref = oracle.render(sc, cams, windows=wins)
    offs = [rng.uniform(0.02, 0.2, size=(3, w[3], w[2])) * rng.choice([-1.0, 1.0], size=(3, w[3], w[2]))
            for w in wins]
    g_ref = None
    for tile in SHAPES:
        r, arena, poses, img, alpha = gpu_forward(sc, cams, tile=tile)
        iv = [x.numpy() for x in r.split(img.cpu(), 3)]
        tv = [im.copy() for im in iv]
        for t, im, f, o, (x0, y0, w, h) in zip(tv, iv, ref["flags"], offs, wins):
            patch = (im[:, y0:y0 + h, x0:x0 + w].astype(np.float64) + o).astype(np.float32)
            t[:, y0:y0 + h, x0:x0 + w] = np.where((f != 0)[None], im[:, y0:y0 + h, x0:x0 + w], patch)
        tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in tv])).to(cuda_device)
        r.cfg.schedule = _lib.GS_SCHED_FUSED_LONGEST_FIRST
        r.bin_sort()
        img_f, loss_f, g_f = fused_step(r, arena, poses, tgt, 0)
        assert torch.equal(img_f, img), tile
        flagged = total = 0
        for v, (x0, y0, w, h) in enumerate(wins):
            ok = (ref["flags"][v] & 1) == 0
            flagged += int((~ok).sum())
            total += ok.size
            d = np.abs(iv[v].astype(np.float64)[:, y0:y0 + h, x0:x0 + w] - ref["image"][v])
            assert d[:, ok].max(initial=0.0) <= IMG_TOL, (tile, v)
        assert flagged <= 0.03 * total
        dimg = loss_grad([x.astype(np.float64) for x in iv], tv, 0, 3 * r.pixels)
        dwin = [d[:, y0:y0 + h, x0:x0 + w] for d, (x0, y0, w, h) in zip(dimg, wins)]
        if g_ref is None:
            g_ref = oracle.backward(sc, cams, dwin, windows=wins)
        compare_grads(g_f, g_ref)
        del r, arena, img, alpha
        torch.cuda.empty_cache()


@pytest.mark.parametrize("deg,nviews", [(0, 1), (1, 2), (2, 1), (3, 3), (3, 40)])
def test_adam_fused_into_the_gaussian_backward_equals_separate_step(cuda_device, deg, nviews):
    """gs_render_bwd_gaussians_adam (the Adam update applied by the SH kernel)
    leaves parameters and moments bit-identical to gs_render_bwd_gaussians +
    gs_adam_step with the matching groups, over two steps with the device step
    counter; a set skip word leaves everything unchanged; parameters left out
    of update_mask keep their values and moments."""
    from paper_2607_14481_b300 import train
    dev = torch.device("cuda:0")
    sc = synth.random_scene(4000, 31 + deg, deg, (-1, -1, -1), (1, 1, 1), -3.2, 0.4)
    if nviews <= 3:
        eyes = [(0.0, 0.0, -3.0), (0.5, -0.2, -2.7), (-0.4, 0.3, -3.2)][:nviews]
        sizes = [(96, 64), (80, 88), (70, 50)][:nviews]
    else:  # a circle of small views: more than 32 views per launch
        eyes = [(3.0 * np.sin(2 * np.pi * k / nviews), 0.2, -3.0 * np.cos(2 * np.pi * k / nviews))
                for k in range(nviews)]
        sizes = [(40 + 8 * (k % 3), 32) for k in range(nviews)]
    cams = [synth.look_at(e, (0, 0, 0), 80.0, 80.0, w / 2, h / 2, w, h) for e, (w, h) in zip(eyes, sizes)]
    lrs = dict(lr_means=1e-2, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3, lr_sh_dc=2.5e-3, lr_sh_rest=1.25e-4)
    runs = []
    for fused_adam in (False, True):
        arena = raster.Arena.from_scene(sc, dev)
        grads, m, v = arena.like(), arena.like(), arena.like()
        r = raster.Rasterizer(sc.n, deg, cams, device=dev)
        poses = raster.poses_tensor(cams, dev)
        tgt = torch.rand(3 * r.pixels, generator=torch.Generator().manual_seed(5)).to(dev)
        step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        ap = raster.adam_params(deg, step_dev=step_dev, status=status, **lrs) if fused_adam else None
        st = train.TrainStep(arena, grads, m, v, arena.adam_groups(**lrs), r, poses, tgt, step_dev, status=status,
                             adam=ap)
        r.forward(arena, poses, r.new_image(), None, check=True)  # pair capacity for these views
        for _ in range(2):
            st.run()
        torch.cuda.synchronize()
        assert int(status.item()) == 0 and int(step_dev.item()) == 2
        runs.append((arena.buf.clone(), m.buf.clone(), v.buf.clone()))
    for a, b in zip(runs[0], runs[1]):
        assert torch.equal(a, b)
    # skip word and update mask, straight through the entry point
    arena = raster.Arena.from_scene(sc, dev)
    grads, m, v = arena.like(), arena.like(), arena.like()
    m.buf.fill_(0.5)
    v.buf.fill_(0.25)
    r = raster.Rasterizer(sc.n, deg, cams, device=dev)
    poses = raster.poses_tensor(cams, dev)
    img = r.new_image()
    r.forward(arena, poses, img, None, check=True)
    dimg = torch.full_like(img, 1e-3)
    r.backward_pixels(dimg, None, img)
    skip = torch.ones(1, dtype=torch.int32, device=dev)
    before = (arena.buf.clone(), m.buf.clone(), v.buf.clone())
    r.backward_gaussians_adam(arena, poses, grads, m, v, raster.adam_params(deg, step=1, skip_dev=skip, **lrs), None)
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(before, (arena.buf, m.buf, v.buf)))
    ap = raster.adam_params(deg, step=1, **lrs)
    ap.update_mask = 1 | 8  # means and SH only
    r.backward_gaussians_adam(arena, poses, grads, m, v, ap, None)
    torch.cuda.synchronize()
    n = sc.n
    for lo, hi in ((4 * n, 8 * n), (8 * n, 12 * n)):  # scale_opa, quat untouched
        assert torch.equal(arena.buf[lo:hi], before[0][lo:hi])
        assert torch.equal(m.buf[lo:hi], before[1][lo:hi]) and torch.equal(v.buf[lo:hi], before[2][lo:hi])
    assert not torch.equal(arena.buf[0:4 * n], before[0][0:4 * n])
    assert not torch.equal(m.buf[12 * n:], before[1][12 * n:])
