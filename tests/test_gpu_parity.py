"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: images 1e-5 max-abs per pixel channel; gradients 1e-3 relative
per parameter group (||g_gpu - g_ref||_inf / max(||g_ref||_inf, 1e-8)); tile
keys, ranges and sort order bit-exact.  Pixels whose value hangs on a decision
within single-precision reach of its threshold (the oracle's flags) are
excluded from the element-wise image check and their loss gradient is set to
zero on both sides; their count is bounded.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import synth
from gpu_util import IMG_TOL, compare_grads, gpu_backward, gpu_forward

pytestmark = pytest.mark.gpu


def _check_images(r, img, alpha, ref, max_flag_frac=0.02):
    imgs = r.split(img.cpu(), 3)
    als = r.split(alpha.cpu(), 1)
    flagged = 0
    total = 0
    for g_img, g_al, o_img, o_al, fl in zip(imgs, als, ref["image"], ref["alpha"], ref["flags"]):
        ok = (fl & 1) == 0
        flagged += int((~ok).sum())
        total += ok.size
        d = np.abs(g_img.numpy().astype(np.float64) - o_img)
        assert d[:, ok].max(initial=0.0) <= IMG_TOL, d[:, ok].max()
        da = np.abs(g_al.numpy().astype(np.float64) - o_al)
        assert da[ok].max(initial=0.0) <= IMG_TOL, da[ok].max()
        # decisions near a threshold still give a valid, bounded value
        assert d.max() < 0.1
    assert flagged <= max_flag_frac * total, (flagged, total)


def _masked(ws, flags):
    return [np.where(f[None] != 0, 0.0, w) if w.ndim == 3 else np.where(f != 0, 0.0, w)
            for w, f in zip(ws, flags)]


# ---------------------------------------------------------------------------
# projection records
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["plain_small", "diffcheck", "box720"])
def test_projection_records(cuda_device, case):
    if case == "plain_small":
        sc, cams, _ = synth.plain_small()
    elif case == "diffcheck":
        sc, cams, _ = synth.diffcheck()
    else:
        sc = synth.box_scene(20000, seed=1007)
        cams = synth.forward_trajectory(3, seed=1008)[1:2]
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    rec = r.splat_arrays()
    proj = oracle.render(sc, cams, want_proj=True, windows=[(0, 0, 16, 16)] * len(cams))["proj"]
    F = {k: i for i, k in enumerate(oracle.PROJ_FIELDS)}
    for v in range(len(cams)):
        P = proj[v]
        vis_o = P[:, F["vis"]] == 1
        vis_g = rec["touched"][v] > 0
        amb = P[:, F["bin_amb"]] == 1
        assert np.array_equal(vis_o[~amb], vis_g[~amb])
        both = vis_o & vis_g
        assert both.sum() > 0
        m_g = rec["xy"][v][:, :2].astype(np.float64) + rec["xy"][v][:, 2:].astype(np.float64)
        m_o = P[:, [F["mx"], F["my"]]]
        assert np.abs(m_g[both] - m_o[both]).max() < 2e-5
        assert np.all(rec["xy"][v][both][:, 2:] >= 0) and np.all(rec["xy"][v][both][:, 2:] < 1)
        for j, name in enumerate(("A", "B", "C")):
            o = P[both, F[name]]
            g = rec["conic"][v][both, j].astype(np.float64)
            scale = np.maximum(np.abs(P[both, F["A"]]), np.abs(P[both, F["C"]]))
            assert np.all(np.abs(g - o) <= 2e-5 * scale), name
        assert np.abs(rec["conic"][v][both, 3] - P[both, F["opacity"]]).max() < 1e-6
        for j, name in enumerate(("r", "g", "b")):
            assert np.abs(rec["rgb"][v][both, j] - P[both, F[name]]).max() < 1e-5
        # depth key: the correctly rounded single-precision depth
        assert np.array_equal(rec["depth"][v][both], P[both, F["depth"]].astype(np.float32))
        ramb = amb
        assert np.array_equal(rec["rgb"][v][both & ~ramb, 3], P[both & ~ramb, F["radius"]])
        rect = rec["rect"][v]
        xlo, ylo = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16
        xhi, yhi = rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
        sel = both & ~amb
        assert np.array_equal(xlo[sel], P[sel, F["xlo"]]) and np.array_equal(yhi[sel], P[sel, F["yhi"]])
        assert np.array_equal(xhi[sel], P[sel, F["xhi"]]) and np.array_equal(ylo[sel], P[sel, F["ylo"]])
        touched = (xhi - xlo + 1) * (yhi - ylo + 1)
        assert np.array_equal(rec["touched"][v][vis_g], touched[vis_g])
        clamp = rec["aux"][v][both] & 7
        assert np.array_equal(clamp[~ramb[both]], P[both, F["clamp"]][~ramb[both]].astype(np.uint32))


# ---------------------------------------------------------------------------
# binning: bit-exact on given records
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [("tiny", [(5, 3), (2, 4)], 40, 0), ("ties", [(5, 3), (2, 4)], 300, 3),
                                   ("720p", [(80, 45)], 200_000, 0), ("multi", [(60, 34), (120, 68), (80, 45)],
                                                                     50_000, 7)])
def test_bins_bit_exact_on_records(cuda_device, shape):
    name, tiles, n, ties = shape
    depth, rect = synth.random_records(tiles, n, seed=31 + n, tie_levels=ties)
    cams = [synth.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 100.0, 100.0, 0.0, 0.0,
                         16 * tx, 16 * ty) for tx, ty in tiles]
    keys_o, vals_o, ranges_o = oracle.bin_records(depth, rect, tiles)
    from paper_2607_14481_b300 import raster
    from gpu_util import ensure_built
    ensure_built()
    r = raster.Rasterizer(n, 0, cams, capacity=len(keys_o) + 17, device=cuda_device, keep_keys=True)
    sv = r.splat_views()
    sv["depth"].copy_(torch.from_numpy(depth))
    packed = np.zeros((len(tiles), n, 2), np.uint32)
    packed[..., 0] = rect[..., 0].astype(np.uint32) | (rect[..., 1].astype(np.uint32) << 16)
    packed[..., 1] = rect[..., 2].astype(np.uint32) | (rect[..., 3].astype(np.uint32) << 16)
    sv["rect"].copy_(torch.from_numpy(packed.view(np.int32)))
    ok = (rect[..., 0] <= rect[..., 2]) & (rect[..., 1] <= rect[..., 3])
    touched = np.where(ok, (rect[..., 2] - rect[..., 0] + 1) * (rect[..., 3] - rect[..., 1] + 1), 0)
    sv["touched"].copy_(torch.from_numpy(touched.astype(np.int32)))
    r.bin_sort()
    torch.cuda.synchronize()
    cnt = r.read_counts()
    K = len(keys_o)
    assert cnt[1] == K and cnt[2] == 0 and cnt[3] == K and cnt[0] == int(ok.sum())
    keys_g = r.keys[:K].cpu().numpy().view(np.uint64)
    vals_g = r.vals[:K].cpu().numpy().view(np.uint32)
    ranges_g = r.ranges[:2 * r.num_tiles].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(keys_g, keys_o)
    assert np.array_equal(vals_g, vals_o)
    # empty tiles: both ends 0 on the GPU; the oracle leaves them 0 too
    assert np.array_equal(ranges_g, ranges_o)
    # pair offsets partition [0, K) into each visible item's contiguous block
    po = r.pair_off.cpu().numpy().view(np.uint32).reshape(len(tiles), n)
    starts = po[ok]
    lens = touched[ok]
    order = np.argsort(starts)
    assert starts[order][0] == 0
    assert np.array_equal(starts[order][1:], np.cumsum(lens[order])[:-1])


def test_bins_bit_exact_long_tile_lists(cuda_device):
    """Tile lists longer than the shared-memory sort (4096 pairs) take the
    CTA-wide radix sort: every record covers the whole 4x3-tile view, with
    three depth levels so that the id order of equal depths is exercised."""
    tiles = [(4, 3)]
    n = 9000
    g = np.random.default_rng(77)
    depth = np.zeros((1, n), np.float32)
    depth[0] = np.float32([0.5, 2.0, 7.25])[g.integers(0, 3, n)]
    rect = np.zeros((1, n, 4), np.int32)
    rect[0, :, 2], rect[0, :, 3] = 3, 2
    culled = g.random(n) < 0.2
    rect[0, culled] = (1, 1, 0, 0)
    rect[0, :50] = (1, 0, 2, 1)  # a few smaller footprints
    keys_o, vals_o, ranges_o = oracle.bin_records(depth, rect, tiles)
    lens = ranges_o[:, 1] - ranges_o[:, 0]
    assert lens.max() > 4096
    cams = [synth.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 100.0, 100.0, 0.0, 0.0, 64, 48)]
    from paper_2607_14481_b300 import raster
    from gpu_util import ensure_built
    ensure_built()
    r = raster.Rasterizer(n, 0, cams, capacity=len(keys_o) + 5, device=cuda_device, keep_keys=True)
    sv = r.splat_views()
    sv["depth"].copy_(torch.from_numpy(depth))
    packed = np.zeros((1, n, 2), np.uint32)
    packed[..., 0] = rect[..., 0].astype(np.uint32) | (rect[..., 1].astype(np.uint32) << 16)
    packed[..., 1] = rect[..., 2].astype(np.uint32) | (rect[..., 3].astype(np.uint32) << 16)
    sv["rect"].copy_(torch.from_numpy(packed.view(np.int32)))
    ok = (rect[..., 0] <= rect[..., 2]) & (rect[..., 1] <= rect[..., 3])
    touched = np.where(ok, (rect[..., 2] - rect[..., 0] + 1) * (rect[..., 3] - rect[..., 1] + 1), 0)
    sv["touched"].copy_(torch.from_numpy(touched.astype(np.int32)))
    for _ in range(2):
        r.bin_sort()
        torch.cuda.synchronize()
        K = len(keys_o)
        cnt = r.read_counts()
        assert cnt[1] == K and cnt[2] == 0 and cnt[3] == K
        assert np.array_equal(r.keys[:K].cpu().numpy().view(np.uint64), keys_o)
        assert np.array_equal(r.vals[:K].cpu().numpy().view(np.uint32), vals_o)
        assert np.array_equal(r.ranges[:2 * r.num_tiles].cpu().numpy().view(np.uint32).reshape(-1, 2), ranges_o)


def test_bins_bit_exact_at_every_sort_size_boundary(cuda_device):
    """One list per tile at the lengths where the per-tile sort changes form
    or shape (warp networks of 32..256 keys, merged warp runs of 256 up to
    2048, the CTA network up to 4096, radix passes beyond, and the padding
    of each), single-tile footprints with a few depth levels so that equal
    depths must come out in id order: keys, ids and ranges equal the oracle's
    bit for bit."""
    lens = [0, 1, 31, 32, 33, 255, 256, 257, 383, 511, 512, 513, 767, 768, 1024, 1025, 1500, 2047, 2048, 2049,
            3000, 4096, 4097, 5000]
    tiles = [(6, 4)]
    n = int(sum(lens))
    g = np.random.default_rng(91)
    depth = np.zeros((1, n), np.float32)
    rect = np.zeros((1, n, 4), np.int32)
    tile_of = np.repeat(np.arange(len(lens)), lens)
    g.shuffle(tile_of)  # the lists' members interleaved in id order
    depth[0] = np.where(g.random(n) < 0.3, np.float32(3.5), (0.2 + 20.0 * g.random(n)).astype(np.float32))
    rect[0, :, 0] = rect[0, :, 2] = tile_of % 6
    rect[0, :, 1] = rect[0, :, 3] = tile_of // 6
    keys_o, vals_o, ranges_o = oracle.bin_records(depth, rect, tiles)
    assert np.array_equal(ranges_o[:, 1] - ranges_o[:, 0], lens)
    cams = [synth.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 100.0, 100.0, 0.0, 0.0, 96, 64)]
    from paper_2607_14481_b300 import raster
    from gpu_util import ensure_built
    ensure_built()
    r = raster.Rasterizer(n, 0, cams, capacity=len(keys_o) + 9, device=cuda_device, keep_keys=True)
    sv = r.splat_views()
    sv["depth"].copy_(torch.from_numpy(depth))
    packed = np.zeros((1, n, 2), np.uint32)
    packed[..., 0] = rect[..., 0].astype(np.uint32) | (rect[..., 1].astype(np.uint32) << 16)
    packed[..., 1] = rect[..., 2].astype(np.uint32) | (rect[..., 3].astype(np.uint32) << 16)
    sv["rect"].copy_(torch.from_numpy(packed.view(np.int32)))
    sv["touched"].copy_(torch.ones((1, n), dtype=torch.int32))
    r.bin_sort()
    torch.cuda.synchronize()
    K = len(keys_o)
    cnt = r.read_counts()
    assert cnt[1] == K and cnt[2] == 0 and cnt[3] == K
    assert np.array_equal(r.keys[:K].cpu().numpy().view(np.uint64), keys_o)
    assert np.array_equal(r.vals[:K].cpu().numpy().view(np.uint32), vals_o)
    assert np.array_equal(r.ranges[:2 * r.num_tiles].cpu().numpy().view(np.uint32).reshape(-1, 2), ranges_o)


def test_bins_capacity_overflow_is_flagged_and_recovered(cuda_device):
    sc, cams, _ = synth.plain_small()
    r, arena, poses, img, alpha = gpu_forward(sc, cams, capacity=64)
    # forward(check=True) grew the capacity after the device flagged overflow
    assert r.capacity > 64 and r.read_counts()[2] == 0
    ref = oracle.render(sc, cams)
    _check_images(r, img, alpha, ref)
    r.set_capacity(16)
    r.bin_sort()
    torch.cuda.synchronize()
    c = r.read_counts()
    assert c[2] == 1 and c[3] == 16 and c[1] > 16


# ---------------------------------------------------------------------------
# images
# ---------------------------------------------------------------------------
def test_image_plain_small(cuda_device):
    sc, cams, _ = synth.plain_small()
    r, _, _, img, alpha = gpu_forward(sc, cams)
    _check_images(r, img, alpha, oracle.render(sc, cams))


def test_image_diffcheck_three_views(cuda_device):
    sc, cams, _ = synth.diffcheck()
    r, _, _, img, alpha = gpu_forward(sc, cams)
    _check_images(r, img, alpha, oracle.render(sc, cams))


def test_image_ragged_tiles_background_sh1(cuda_device):
    # 130x70: partial tiles on both edges; degree-1 SH; coloured background
    sc = synth.random_scene(3000, 77, 1, (-1, -1, -1), (1, 1, 1), -3.2, 0.5)
    cams = [synth.look_at((0.3, -0.2, -3.0), (0, 0, 0), 110.0, 105.0, 61.3, 37.9, 130, 70)]
    bg = (0.25, 0.5, 0.75)
    r, _, _, img, alpha = gpu_forward(sc, cams, bg=bg)
    _check_images(r, img, alpha, oracle.render(sc, cams, bg=bg))


def test_image_permutation_bit_exact(cuda_device):
    sc, cams, _ = synth.plain_small(7)
    proj = oracle.render(sc, cams, want_proj=True, windows=[(0, 0, 1, 1)])["proj"][0]
    _, first = np.unique(proj[:, 10].astype(np.float32), return_index=True)
    sc = sc.subset(np.sort(first))
    _, _, _, a, _ = gpu_forward(sc, cams)
    perm = np.random.default_rng(3).permutation(sc.n)
    _, _, _, b, _ = gpu_forward(sc.subset(perm), cams)
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("single_pass", [False, True])
def test_gradients_plain_small_l1(cuda_device, single_pass):
    sc, cams, targets = synth.plain_small()
    ref = oracle.render(sc, cams)
    _, dimg = oracle.l1_loss(ref["image"], targets)
    dimg = _masked(dimg, ref["flags"])
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    g_gpu = gpu_backward(r, arena, poses, dimg, image=img if single_pass else None)
    g_ref = oracle.backward(sc, cams, dimg)
    compare_grads(g_gpu, g_ref)


def test_single_pass_backward_mse_background_multiview(cuda_device):
    """The front-to-back form (colour behind = forward image minus composited
    prefix) against the oracle, with a background (the remainder ends at
    T_final * bg) and several views of different sizes in one launch."""
    sc, cams, targets = synth.diffcheck()
    bg = (0.1, 0.2, 0.3)
    ref = oracle.render(sc, cams, bg=bg)
    _, dimg = oracle.mse_loss(ref["image"], targets)
    dimg = _masked(dimg, ref["flags"])
    r, arena, poses, img, alpha = gpu_forward(sc, cams, bg=bg)
    g_one = gpu_backward(r, arena, poses, dimg, image=img)
    g_ref = oracle.backward(sc, cams, dimg, bg=bg)
    compare_grads(g_one, g_ref)
    g_two = gpu_backward(r, arena, poses, dimg)
    compare_grads(g_one, g_two)


def test_gradients_diffcheck_mse_with_alpha_and_background(cuda_device):
    sc, cams, targets = synth.diffcheck()
    bg = (0.1, 0.2, 0.3)
    ref = oracle.render(sc, cams, bg=bg)
    _, dimg = oracle.mse_loss(ref["image"], targets)
    dimg = _masked(dimg, ref["flags"])
    rng = np.random.default_rng(5)
    dal = _masked([rng.normal(size=(c.height, c.width)) * 1e-3 for c in cams], ref["flags"])
    r, arena, poses, img, alpha = gpu_forward(sc, cams, bg=bg)
    g_gpu = gpu_backward(r, arena, poses, dimg, dal)
    g_ref = oracle.backward(sc, cams, dimg, dal, bg=bg)
    compare_grads(g_gpu, g_ref)


def test_gradients_forty_views_in_one_launch(cuda_device):
    """40 views of the diffcheck scene on a full circle in one launch (more
    than 32, so the per-Gaussian backward's bit set of the views that see a
    Gaussian uses both of its words; views from behind see the scene's other
    side): gradients, the 40 pose gradients included, against the oracle."""
    sc, _, _ = synth.diffcheck()
    cams = []
    for k in range(40):
        a = 2.0 * np.pi * k / 40
        eye = (2.5 * np.sin(a), 0.4 * np.sin(3.0 * a), -2.5 * np.cos(a))
        cams.append(synth.look_at(eye, (0, 0, 0), 40.0, 40.0, 16.0, 12.0, 32, 24))
    g = np.random.default_rng(11)
    targets = [g.random((3, 24, 32)).astype(np.float32) for _ in cams]
    ref = oracle.render(sc, cams)
    _, dimg = oracle.l1_loss(ref["image"], targets)
    dimg = _masked(dimg, ref["flags"])
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    g_gpu = gpu_backward(r, arena, poses, dimg, image=img)
    g_ref = oracle.backward(sc, cams, dimg)
    compare_grads(g_gpu, g_ref)


@pytest.mark.parametrize("single_pass", [False, True])
def test_backward_deterministic(cuda_device, single_pass):
    sc, cams, targets = synth.diffcheck()
    ref = oracle.render(sc, cams)
    _, dimg = oracle.mse_loss(ref["image"], targets)
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    image = img if single_pass else None
    a = gpu_backward(r, arena, poses, dimg, image=image)
    b = gpu_backward(r, arena, poses, dimg, image=image)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_empty_and_all_culled(cuda_device):
    sc, cams, _ = synth.plain_small()
    bg = (0.3, 0.2, 0.1)
    # every Gaussian behind the camera
    behind = [synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, -5], np.float32), 120.0, 120.0,
                           64.0, 64.0, 128, 128)]
    r, arena, poses, img, alpha = gpu_forward(sc, behind, bg=bg)
    im = r.split(img.cpu(), 3)[0].numpy()
    for ch in range(3):
        assert np.all(im[ch] == np.float32(bg[ch]))
    assert torch.all(alpha == 0)
    for image in (None, img):
        g = gpu_backward(r, arena, poses, [np.ones((3, 128, 128))], image=image)
        for k in ("means", "log_scales", "quats", "opa_logits", "sh", "pose"):
            assert np.all(g[k] == 0), k
    # a single Gaussian (n = 1) far outside the view
    one = sc.subset([0])
    one.means[0] = (50.0, 0.0, 0.0)
    r, arena, poses, img, alpha = gpu_forward(one, cams, bg=bg)
    assert r.read_counts()[1] == 0
    im = r.split(img.cpu(), 3)[0].numpy()
    assert np.all(im[1] == np.float32(bg[1]))


def test_single_huge_gaussian_covering_every_tile(cuda_device):
    sc = synth.random_scene(1, 5, 0, (0, 0, 0), (0, 0, 0), np.log(0.8), 0.0)
    sc.opa_logits[:] = 2.0
    cams = [synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 3], np.float32), 120.0, 120.0,
                         64.0, 64.0, 128, 128)]
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    assert r.read_counts()[1] == 64
    ref = oracle.render(sc, cams)
    _check_images(r, img, alpha, ref)


# ---------------------------------------------------------------------------
# full size: 500k Gaussians, SH3, 1280x720, on a forward-moving trajectory
# ---------------------------------------------------------------------------
def test_full_size_500k_720p_sampled_windows(cuda_device):
    sc = synth.box_scene(500_000, seed=1007)
    cams = synth.forward_trajectory(100, seed=1008)[10:11]
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    full = r.split(img.cpu(), 3)[0].numpy().astype(np.float64)
    full_a = r.split(alpha.cpu(), 1)[0].numpy().astype(np.float64)
    rng = np.random.default_rng(9)
    wins = [(int(rng.integers(0, 1280 - 48)), int(rng.integers(0, 720 - 48)), 48, 48) for _ in range(3)]
    wins.append((1280 - 40, 720 - 24, 40, 24))  # the ragged corner
    flagged = total = 0
    for win in wins:
        x0, y0, w, h = win
        ref = oracle.render(sc, cams, windows=[win])
        ok = (ref["flags"][0] & 1) == 0
        flagged += int((~ok).sum())
        total += ok.size
        d = np.abs(full[:, y0:y0 + h, x0:x0 + w] - ref["image"][0])
        assert d[:, ok].max(initial=0.0) <= IMG_TOL
        da = np.abs(full_a[y0:y0 + h, x0:x0 + w] - ref["alpha"][0])
        assert da[ok].max(initial=0.0) <= IMG_TOL
    assert flagged <= 0.03 * total
    # gradients of a loss living in one window (zero elsewhere), all groups
    x0, y0, w, h = wins[0]
    ref = oracle.render(sc, cams, windows=[wins[0]])
    gw = rng.normal(size=(3, h, w)) / (3 * h * w)
    gw = np.where(ref["flags"][0][None] != 0, 0.0, gw)
    dfull = np.zeros((3, 720, 1280))
    dfull[:, y0:y0 + h, x0:x0 + w] = gw
    g_ref = oracle.backward(sc, cams, [gw], windows=[wins[0]])
    for image in (None, img):  # replay + reverse walk, and the single front-to-back pass
        g_gpu = gpu_backward(r, arena, poses, [dfull], image=image)
        compare_grads(g_gpu, g_ref)


# ---------------------------------------------------------------------------
# full size, batched: 2M Gaussians, SH3, 16 views of uneven resolution
# (540p-1080p) on the inward loop, all in one launch per stage, with the blend
# schedule the autotuner picks (the bench's batched launch configuration)
# ---------------------------------------------------------------------------
def test_full_size_batched_2m_16_views_sampled_windows(cuda_device):
    sc = synth.box_scene(2_000_000, seed=1007)
    cams = synth.loop_views(16, 1009)
    rng = np.random.default_rng(3)
    wins = [(int(rng.integers(0, c.width - 32)), int(rng.integers(0, c.height - 32)), 32, 32) for c in cams[:-1]]
    wins.append((cams[-1].width - 24, cams[-1].height - 20, 24, 20))  # a ragged corner
    ref = oracle.render(sc, cams, windows=wins)
    # a loss gradient living in the windows, zero on pixels whose decisions
    # the oracle flags as too close to a threshold to be compared
    gw = [np.where(f[None] != 0, 0.0, rng.normal(size=(3, w[3], w[2])) / (3 * w[2] * w[3] * 16))
          for f, w in zip(ref["flags"], wins)]
    dfull = [np.zeros((3, c.height, c.width)) for c in cams]
    for d, g, (x0, y0, w, h) in zip(dfull, gw, wins):
        d[:, y0:y0 + h, x0:x0 + w] = g
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    dimg = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dfull]).astype(np.float32)).to(cuda_device)
    r.autotune(img, dimg, reps=1)
    r.forward(arena, poses, img, alpha)
    imgs, alphas = r.split(img.cpu(), 3), r.split(alpha.cpu(), 1)
    flagged = total = 0
    for v, (x0, y0, w, h) in enumerate(wins):
        ok = (ref["flags"][v] & 1) == 0
        flagged += int((~ok).sum())
        total += ok.size
        d = np.abs(imgs[v].numpy().astype(np.float64)[:, y0:y0 + h, x0:x0 + w] - ref["image"][v])
        assert d[:, ok].max(initial=0.0) <= IMG_TOL, v
        da = np.abs(alphas[v].numpy().astype(np.float64)[y0:y0 + h, x0:x0 + w] - ref["alpha"][v])
        assert da[ok].max(initial=0.0) <= IMG_TOL, v
    assert flagged <= 0.03 * total
    g_ref = oracle.backward(sc, cams, gw, windows=wins)
    g_gpu = gpu_backward(r, arena, poses, dfull, image=img)
    compare_grads(g_gpu, g_ref)


def test_tile_order_is_a_bucketed_permutation_and_changes_nothing(cuda_device):
    """Longest-lists-first scheduling: the order is a permutation of the
    tiles with non-increasing power-of-two length buckets (empty tiles last),
    and images and gradients are bit-identical to the natural order."""
    sc, cams, _ = synth.diffcheck()
    ref = oracle.render(sc, cams)
    _, dimg = oracle.mse_loss(ref["image"], synth.diffcheck()[2])
    out = []
    for lf in (False, True):
        from paper_2607_14481_b300 import _lib
        r, arena, poses, img, alpha = gpu_forward(sc, cams)
        r.cfg.schedule = (_lib.GS_SCHED_FWD_LONGEST_FIRST | _lib.GS_SCHED_BWD_LONGEST_FIRST) if lf else 0
        r.forward(arena, poses, img, alpha)
        g = gpu_backward(r, arena, poses, dimg, image=img)
        torch.cuda.synchronize()
        out.append((img.clone(), alpha.clone(), g))
        if lf:
            order = r.tile_order[:r.num_tiles].cpu().numpy().astype(np.int64)
            assert np.array_equal(np.sort(order), np.arange(r.num_tiles))
            rg = r.ranges[:2 * r.num_tiles].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
            L = (rg[:, 1] - rg[:, 0])[order]
            b = np.where(L == 0, 16, 15 - np.minimum(15, np.floor(np.log2(np.maximum(L, 1))).astype(np.int64)))
            assert np.all(np.diff(b) >= 0)
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    for k in out[0][2]:
        assert np.array_equal(out[0][2][k], out[1][2][k]), k


def test_schedules_change_no_result_and_autotune_picks_one(cuda_device):
    """Every blend schedule (tile order x splats per batch) gives bit-identical
    images and gradients; the autotuner times them and keeps one."""
    from paper_2607_14481_b300 import _lib
    sc, cams, targets = synth.diffcheck()
    ref = oracle.render(sc, cams)
    _, dimg = oracle.mse_loss(ref["image"], targets)
    base = None
    for order in (0, 1):
        for fb in (0, 1, 2):
            for bb in (0, 1):
                sched = (order * (_lib.GS_SCHED_FWD_LONGEST_FIRST | _lib.GS_SCHED_BWD_LONGEST_FIRST)) | (fb << 4) | \
                        (bb << 8)
                r, arena, poses, img, alpha = gpu_forward(sc, cams)
                r.cfg.schedule = sched
                r.forward(arena, poses, img, alpha)
                g = gpu_backward(r, arena, poses, dimg, image=img)
                torch.cuda.synchronize()
                got = (img.clone(), alpha.clone(), g)
                if base is None:
                    base = got
                    continue
                assert torch.equal(base[0], got[0]) and torch.equal(base[1], got[1]), hex(sched)
                for k in base[2]:
                    assert np.array_equal(base[2][k], got[2][k]), (hex(sched), k)
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    d = torch.from_numpy(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in dimg])).cuda()
    res = r.autotune(img, d, reps=2)
    assert r.cfg.schedule == res["schedule"]
    assert all(np.isfinite(v) and v > 0 for v in res["ms"].values())
    # the image the autotuner leaves behind is the composite
    assert torch.equal(img, base[0])
