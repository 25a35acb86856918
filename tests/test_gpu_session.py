"""The streaming session (continuous batching, admission by HBM budget):

  * a render request gives the same image alone and in a batch mixed with
    other requests of other resolutions (bit-identical), equal to the direct
    rasterizer and within tolerance of the FP64 oracle;
  * training requests give the same parameters alone and with render
    requests mixed into their batches, and the same as the direct API's
    training steps (bit-identical: render views never enter the update);
  * save / load resumes bit-identically;
  * a batch that overflows its pair capacity grows it and runs again.
"""
import ctypes as C
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import _lib, raster, session, synth
from gpu_util import IMG_TOL, ensure_built

pytestmark = pytest.mark.gpu

RENDER, TRAIN = _lib.GS_REQUEST_RENDER, _lib.GS_REQUEST_TRAIN


def _scene(n=20000, seed=5, deg=3):
    return synth.random_scene(n, seed, deg, (-2, -1, -2), (2, 1, 2), -3.5, 0.5)


def _cams(k, seed=8):
    g = np.random.default_rng(seed)
    sizes = [(320, 180), (480, 270), (400, 224), (256, 144)]
    out = []
    for i in range(k):
        a = 2 * np.pi * i / k
        w, h = sizes[int(g.integers(0, len(sizes)))]
        out.append(synth.look_at((5 * np.sin(a), -0.5, -5 * np.cos(a)), (0, 0, 0), 0.8 * w, 0.8 * w, w / 2, h / 2, w, h))
    return out


def _cfg(n, **kw):
    kw.setdefault("max_batch_views", 8)
    kw.setdefault("max_width", 480)
    kw.setdefault("max_height", 272)
    kw.setdefault("hbm_budget_gb", 8.0)
    return session.default_config(n, **kw)


def _direct_render(sc, cam):
    dev = torch.device("cuda:0")
    a = raster.Arena.from_scene(sc, dev)
    r = raster.Rasterizer(sc.n, sc.sh_degree, [cam], device=dev)
    img, _ = r.forward(a, raster.poses_tensor([cam], dev), r.new_image(), None)
    torch.cuda.synchronize()
    return r.split(img.cpu(), 3)[0].numpy()


def test_render_alone_equals_in_mix(cuda_device):
    ensure_built()
    sc = _scene()
    cams = _cams(8)
    with session.Session(_cfg(sc.n)) as s:
        s.add(sc)
        rid = s.submit(RENDER, cams[0], want_image=True)
        alone = s.wait(rid)
        s.hold(True)  # the next eight requests arrive as one group
        ids = [s.submit(RENDER, c, want_image=True) for c in cams[1:4]]
        rid2 = s.submit(RENDER, cams[0], want_image=True)
        ids += [s.submit(RENDER, c, want_image=True) for c in cams[4:]]
        s.hold(False)
        mixed = s.wait(rid2)
        for i in ids:
            s.wait(i)
        st = s.stats()
    assert st["completed"] == 9 and st["failed"] == 0
    # the held group went out as one batch; a retry after a pair-capacity
    # overflow (the pair buffers grow on first use) counts as a batch too
    assert st["batches"] - st["retries"] == 2
    assert np.array_equal(alone, mixed)
    assert np.array_equal(alone, _direct_render(sc, cams[0]))
    ref = oracle.render(sc, cams[:1])
    ok = (ref["flags"][0] & 1) == 0
    assert np.abs(alone.astype(np.float64) - ref["image"][0])[:, ok].max() <= IMG_TOL


def _targets(cams, seed=3):
    g = np.random.default_rng(seed)
    return [g.random((3, c.height, c.width)).astype(np.float32) for c in cams]


def _direct_train(sc, cams, targets, lrs):
    """The same training steps through the direct API (one view per step)."""
    dev = torch.device("cuda:0")
    a = raster.Arena.from_scene(sc, dev)
    g, m, v = a.like(), a.like(), a.like()
    groups = a.adam_groups(**lrs)
    loss = raster.ImageLoss(dev)
    for k, (c, t) in enumerate(zip(cams, targets)):
        r = raster.Rasterizer(sc.n, sc.sh_degree, [c], device=dev)
        img, _ = r.forward(a, raster.poses_tensor([c], dev), r.new_image(), None)
        dimg = r.new_image()
        loss(img, torch.from_numpy(t.reshape(-1)).to(dev), dimg, 0)
        r.backward(a, raster.poses_tensor([c], dev), dimg, None, g, None, img)
        raster.adam_step(a, g, m, v, k + 1, groups)
    torch.cuda.synchronize()
    return a


def test_train_alone_equals_with_renders_mixed_and_direct(cuda_device):
    ensure_built()
    sc = _scene(n=15000, seed=6)
    cams = _cams(4, seed=9)
    targets = _targets(cams)
    lrs = dict(lr_means=1e-3, lr_scale=5e-3, lr_opacity=5e-2, lr_quat=1e-3, lr_sh_dc=2.5e-3, lr_sh_rest=1.25e-4)
    extra = _cams(6, seed=10)
    results = []
    for mixed in (False, True):
        with session.Session(_cfg(sc.n + 1000, **lrs)) as s:
            s.add(sc)
            for c, t in zip(cams, targets):
                rid = s.submit(TRAIN, c, target=t)
                others = [s.submit(RENDER, e, want_image=True) for e in extra[:3]] if mixed else []
                s.wait(rid)
                for o in others:
                    s.wait(o)
            st = s.stats()
            assert st["iterations"] == len(cams) and st["failed"] == 0
            results.append(s.params())
    for k in results[0]:
        assert np.array_equal(results[0][k], results[1][k]), k
    d = _direct_train(sc, cams, targets, lrs)
    nat = d.buf.cpu().numpy()
    n = sc.n
    assert np.array_equal(results[0]["means4"], nat[0:4 * n].reshape(n, 4))
    assert np.array_equal(results[0]["scale_opa"], nat[4 * n:8 * n].reshape(n, 4))
    assert np.array_equal(results[0]["quat"], nat[8 * n:12 * n].reshape(n, 4))
    assert np.array_equal(results[0]["sh"], nat[12 * n:12 * n + 48 * n].reshape(48, n))


def test_borrowed_pinned_targets_train_like_copied_ones(cuda_device):
    """GS_REQUEST_BORROW_TARGET: train requests whose targets stay in the
    caller's pinned memory (several in flight at once, two sharing one
    buffer) leave the parameters bit-identical to the same requests with
    targets copied during submit; a pageable array is refused as a borrowed
    target and unknown flags are rejected by the library."""
    ensure_built()
    sc = _scene(n=12000, seed=12)
    cams = _cams(5, seed=13)
    targets = _targets(cams, seed=5)
    pinned = [torch.from_numpy(np.ascontiguousarray(t, np.float32)).pin_memory() for t in targets]
    results = []
    for borrow in (False, True):
        with session.Session(_cfg(sc.n)) as s:
            s.add(sc)
            s.hold(True)
            ids = [s.submit(TRAIN, c, target=(p if borrow else t), borrow_target=borrow)
                   for c, t, p in zip(cams, targets, pinned)]
            ids.append(s.submit(TRAIN, cams[0], target=(pinned[0] if borrow else targets[0]), borrow_target=borrow))
            s.hold(False)
            for rid in ids:
                s.wait(rid)
            assert s.stats()["failed"] == 0
            results.append(s.params())
    for k in results[0]:
        assert np.array_equal(results[0][k], results[1][k]), k
    with session.Session(_cfg(sc.n)) as s:
        s.add(sc)
        with pytest.raises(ValueError):
            s.submit(TRAIN, cams[0], target=targets[0], borrow_target=True)
        req = _lib.GsRequest()
        req.kind = TRAIN
        req.cam = _lib.GsCamera(cams[0].fx, cams[0].fy, cams[0].cx, cams[0].cy, cams[0].width, cams[0].height)
        req.target = pinned[0].data_ptr()
        req.flags = 2
        rid = C.c_int64()
        assert s.L.gs_session_submit(s.h, C.byref(req), C.byref(rid)) == _lib.GS_ERR_INVALID


def test_save_load_resumes_bit_identically(cuda_device, tmp_path):
    ensure_built()
    sc = _scene(n=8000, seed=7, deg=1)
    cams = _cams(4, seed=11)
    targets = _targets(cams, seed=4)
    path = str(tmp_path / "ckpt.bin")
    with session.Session(_cfg(sc.n, sh_degree=1)) as s:
        s.add(sc)
        for c, t in zip(cams[:2], targets[:2]):
            s.wait(s.submit(TRAIN, c, target=t))
        s.save(path)
        for c, t in zip(cams[2:], targets[2:]):
            s.wait(s.submit(TRAIN, c, target=t))
        full = s.params()
    with session.Session(_cfg(sc.n, sh_degree=1)) as s2:
        s2.load(path)
        for c, t in zip(cams[2:], targets[2:]):
            s2.wait(s2.submit(TRAIN, c, target=t))
        resumed = s2.params()
    assert np.all(np.isfinite(full["means4"]))
    for k in full:
        assert np.array_equal(full[k], resumed[k]), k


def test_pair_capacity_overflow_retries(cuda_device):
    ensure_built()
    sc = _scene(n=20000, seed=12)
    cams = _cams(2, seed=13)
    # initial pair capacity 4096 (the floor) is far below this scene's pairs
    with session.Session(_cfg(sc.n, pair_factor=1e-6)) as s:
        s.add(sc)
        rid = s.submit(RENDER, cams[0], want_image=True)
        img = s.wait(rid)
        st = s.stats()
    assert st["completed"] == 1 and st["failed"] == 0
    assert st["batches"] >= 2  # the first attempt overflowed and was issued again
    assert np.array_equal(img, _direct_render(sc, cams[0]))


def test_empty_scene_renders_background(cuda_device):
    ensure_built()
    cam = _cams(1)[0]
    with session.Session(_cfg(1000, bg=(0.25, 0.5, 0.75))) as s:
        img = s.wait(s.submit(RENDER, cam, want_image=True))
    for ch, b in enumerate((0.25, 0.5, 0.75)):
        assert np.all(img[ch] == np.float32(b))


def _clustered_scene(clusters, per, seed):
    """Tight clusters of `per` tiny Gaussians (a fraction of a pixel from a
    camera at the origin looking down +z, focal 300): a merged cluster stays
    below a pixel, so it stays in the active set after the reload."""
    g = np.random.default_rng(seed)
    z = g.uniform(10, 30, clusters)
    centres = np.column_stack([g.uniform(-0.4, 0.4, clusters) * z, g.uniform(-0.3, 0.3, clusters) * z, z])
    means = np.repeat(centres, per, axis=0) + g.normal(0, 0.002, (clusters * per, 3)) * np.repeat(z, per)[:, None] / 20
    zz = means[:, 2]
    S = g.uniform(0.05, 0.3, len(zz))
    ls = np.log(S * zz / 900.0)[:, None] - np.abs(g.normal(0, 0.2, (len(zz), 3)))
    base = synth.random_scene(len(zz), seed + 1, 1, (0, 0, 0), (1, 1, 1), 0.0, 1.0)
    return synth.Scene(means.astype(np.float32), ls.astype(np.float32), base.quats, base.opa_logits, base.sh)


def test_progressive_hierarchy_in_the_session(cuda_device):
    """The session's progressive hierarchy (lod = 1).  Before any analysis
    every added leaf is active and a render equals the plain render.  An
    analysis from a keyframe's camera (merge below tau / 2, then reload above
    tau) gives the node rows, links, active flags and merged parameters of
    the direct gs_hier_analyze + gs_hier_refine, and renders through the
    render cut (descent from the roots) equal the direct
    gs_project_hier_render path while blending fewer splats.  A training request then updates merged nodes of the cut and
    leaves the merged-away leaves alone; keyframe counts cover the active
    nodes (merged nodes take their children's keyframe)."""
    ensure_built()
    n = 4000
    sc = _clustered_scene(n // 4, 4, seed=3)
    far = synth.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 300.0, 300.0, 320.0, 240.0, 640, 480)
    dev = torch.device("cuda:0")
    cfg = _cfg(n, sh_degree=1, lod=True, lod_tau=1.0, max_width=640, max_height=480, max_batch_views=2,
               lr_means=1e-2, lr_sh_dc=1e-2)
    with session.Session(cfg) as s:
        s.set_keyframe(0)
        s.add(sc)
        img0 = s.wait(s.submit(RENDER, far, want_image=True))
        assert s.analyze(far)
        s.drain()
        st = s.stats()
        h = s.hierarchy()
        img1 = s.wait(s.submit(RENDER, far, want_image=True))
        kw = s.keyframe_weights(1, min_keep=0)
        s.wait(s.submit(TRAIN, far, target=_targets([far], seed=5)[0]))
        h2 = s.hierarchy()
        st2 = s.stats()
    assert np.array_equal(img0, _direct_render(sc, far))
    assert st["lod_builds"] == 1 and st2["iterations"] == 1 and st2["failed"] == 0
    # the direct path on an arena of the same rows
    arena = raster.Arena.from_scene(sc, dev, capacity=2 * n)
    hier = raster.Hierarchy(arena, n)
    hier.analyze(far, tau_l=0.5)
    hier.refine(far, tau_h=1.0, passes=16)
    d = hier.state()
    rows = d["n_nodes"]
    assert rows > n and len(h["active"]) == rows
    assert np.array_equal(h["parent"], d["parent"][:rows])
    assert np.array_equal(h["child"], d["child"][:rows])
    assert np.array_equal(h["active"], d["active"][:rows])
    buf = arena.buf.cpu().numpy()
    cap = 2 * n
    assert np.array_equal(h["means4"], buf[0:4 * cap].reshape(cap, 4)[:rows])
    assert np.array_equal(h["scale_opa"], buf[4 * cap:8 * cap].reshape(cap, 4)[:rows])
    assert np.array_equal(h["quat"], buf[8 * cap:12 * cap].reshape(cap, 4)[:rows])
    assert np.array_equal(h["sh"], buf[12 * cap:12 * cap + 12 * cap].reshape(12, cap)[:, :rows])
    r = raster.Rasterizer(rows, 1, [far], device=dev)
    r.project_hier(hier, raster.poses_tensor([far], dev), tau_h=1.0, from_roots=True)
    r.bin_sort()
    img = r.new_image()
    r.render_fwd(img, None)
    torch.cuda.synchronize()
    assert np.array_equal(img1, r.split(img.cpu(), 3)[0].numpy())
    cut = int((r.splat_arrays()["touched"][0] > 0).sum())
    plain = raster.Rasterizer(n, 1, [far], device=dev)
    plain.project(raster.Arena.from_scene(sc, dev), raster.poses_tensor([far], dev))
    assert cut < int((plain.splat_arrays()["touched"][0] > 0).sum())
    # keyframe weights count the leaves still in the active set (Sec. 6.2)
    assert int(kw["counts"][0]) == int(h["active"][:n].sum()) < n
    # training: merged nodes of the cut move, merged-away leaves do not
    merged = np.flatnonzero(h["active"][n:] == 1) + n
    away = np.flatnonzero(h["active"][:n] == 0)
    assert len(merged) > 0 and len(away) > 0
    assert np.any(h2["means4"][merged] != h["means4"][merged])
    assert np.array_equal(h2["means4"][away], h["means4"][away])
    assert np.array_equal(h2["sh"][:, away], h["sh"][:, away])


def test_loop_closure_moves_gaussians_with_their_keyframe(cuda_device):
    """Gaussians added under keyframes 0 and 1 (and untagged ones) move with
    their keyframe's Sim(3) correction at a loop closure (FP64 oracle), and a
    render after it equals the direct render of the moved scene."""
    ensure_built()
    g = np.random.default_rng(21)
    parts = [synth.random_scene(3000, 30 + i, 1, (-2, -1, -2), (2, 1, 2), -3.0, 0.4) for i in range(3)]
    tags = [0, 1, -1]

    def sim3():
        q = g.normal(size=4)
        q /= np.linalg.norm(q)
        return np.concatenate([q, 0.2 * g.normal(size=3), [np.exp(0.2 * g.normal())]])

    S = np.stack([sim3(), sim3()]).astype(np.float32)
    cam = _cams(1, seed=22)[0]
    n = sum(p.n for p in parts)
    with session.Session(_cfg(n, sh_degree=1)) as s:
        for p, k in zip(parts, tags):
            s.set_keyframe(k)
            s.add(p)
        s.loop_closure(S)
        img = s.wait(s.submit(RENDER, cam, want_image=True))
        got = s.params()
    before = synth.Scene(*(np.concatenate([getattr(p, f) for p in parts]) for f in
                           ("means", "log_scales", "quats", "opa_logits", "sh")))
    kf = np.concatenate([np.full(p.n, k) for p, k in zip(parts, tags)])
    mu, ls, q = oracle.sim3_update(before.means, before.log_scales, before.quats, kf, S.astype(np.float64))
    scale = np.maximum(1.0, np.abs(mu))
    assert np.all(np.abs(got["means4"][:, :3] - mu) <= 4e-6 * scale)
    assert np.abs(got["scale_opa"][:, :3] - ls).max() <= 2e-6
    assert np.abs(got["quat"] - q).max() <= 2e-6 * max(1.0, np.abs(q).max())
    moved = synth.Scene(got["means4"][:, :3].copy(), got["scale_opa"][:, :3].copy(), got["quat"].copy(),
                        got["scale_opa"][:, 3].copy(), got["sh"].T.reshape(n, 3, 4).copy())
    assert np.array_equal(img, _direct_render(moved, cam))


def test_keyframe_weights_match_oracle(cuda_device):
    """Leaf counts per keyframe on the device and the Sec. 6.2 sampling rule
    (5% offload, at least min_keep kept) against the oracle."""
    ensure_built()
    g = np.random.default_rng(31)
    K = 120
    sizes = (g.pareto(1.2, K) * 40).astype(int)[:K]
    sizes = np.minimum(sizes, 3000)
    tags = []
    with session.Session(_cfg(int(sizes.sum()) + 200, sh_degree=0)) as s:
        for k in range(K):
            if sizes[k] == 0:
                continue
            s.set_keyframe(k)
            s.add(synth.random_scene(int(sizes[k]), 40 + k, 0, (-1, -1, -1), (1, 1, 1), -3.0, 0.3))
            tags.append(np.full(sizes[k], k))
        s.set_keyframe(-1)
        s.add(synth.random_scene(200, 7, 0, (-1, -1, -1), (1, 1, 1), -3.0, 0.3))  # untagged
        tags.append(np.full(200, -1))
        for min_keep in (0, 50, 200):
            got = s.keyframe_weights(K, min_keep=min_keep)
            c, p, kept = oracle.keyframe_weights(np.concatenate(tags), K, min_keep=min_keep)
            assert np.array_equal(got["counts"], c)
            assert np.array_equal(got["kept"], kept)
            assert np.allclose(got["p"], p, rtol=1e-12, atol=0)
        picks = s.sample_keyframes(K, 1000, np.random.default_rng(0))
        assert np.all(kept[picks])


def test_render_beside_train_sees_exactly_the_updates_issued_before_it(cuda_device):
    """Render parts run on their own batch contexts' streams.  A render issued
    before a train batch runs beside that batch's forward and backward and
    shows the parameters before its update; a render submitted while a train
    batch is executing waits for its update on the device.  Each equals the
    same render alone, bit for bit."""
    ensure_built()
    sc = _scene(n=20000, seed=12)
    view = _cams(1, seed=13)[0]
    tcam = synth.look_at((0.5, -0.4, -4.5), (0, 0, 0), 380.0, 380.0, 240.0, 136.0, 480, 272)
    tgt = _targets([tcam], seed=14)[0]
    cfg = _cfg(sc.n, max_batch_views=1, max_inflight=3, pair_factor=16.0, lr_means=1e-2, lr_opacity=0.2)
    with session.Session(cfg) as s:
        s.add(sc)
        assert s.stats()["contexts"] >= 2
        before = s.wait(s.submit(RENDER, view, want_image=True))  # alone, no update yet
        # render, then train, released together as two batches
        s.hold(True)
        ra = s.submit(RENDER, view, want_image=True)
        t1 = s.submit(TRAIN, tcam, target=tgt)
        s.hold(False)
        img_a = s.wait(ra)
        s.wait(t1)
        # train, then a render submitted while it executes
        t2 = s.submit(TRAIN, tcam, target=tgt)
        rb = s.submit(RENDER, view, want_image=True)
        img_b = s.wait(rb)
        s.wait(t2)
        after = s.wait(s.submit(RENDER, view, want_image=True))  # alone, after both updates
        st = s.stats()
    assert st["failed"] == 0 and st["iterations"] == 2 and st["retries"] == 0
    assert st["train_beside_render"] >= 1
    assert np.array_equal(img_a, before)
    assert np.array_equal(img_b, after)
    assert not np.array_equal(after, before)  # the two updates changed what the view shows


def test_allocation_failure_is_reported_and_the_session_keeps_serving(cuda_device):
    """Host-side fault injection: the pair buffers of a batch that overflowed
    cannot grow (the allocation fails as if the device were out of memory),
    so its request finishes with GS_ERR_OOM; the context keeps its old
    buffers and the session serves the next request (which grows them)."""
    ensure_built()
    sc = _scene(n=20000, seed=15)
    big = _cams(1, seed=16)[0]
    with session.Session(_cfg(sc.n, max_batch_views=1, max_inflight=1, pair_factor=0.01)) as s:
        s.add(sc)
        assert session.plan(_cfg(sc.n, max_batch_views=1, max_inflight=1, pair_factor=0.01))[
            "initial_pair_capacity"] == 4096
        s.inject_alloc_failures(1)
        rid = s.submit(RENDER, big, want_image=True)
        with pytest.raises(_lib.GsError) as ei:
            s.wait(rid)
        assert ei.value.status == _lib.GS_ERR_OOM
        img = s.wait(s.submit(RENDER, big, want_image=True))
        st = s.stats()
    assert st["failed"] == 1 and st["completed"] == 1 and st["retries"] >= 1
    assert np.array_equal(img, _direct_render(sc, big))


@pytest.mark.parametrize("tile", [(32, 8), (8, 32)])
def test_session_with_other_tile_shapes(cuda_device, tile):
    """Sessions take any supported tile shape: renders equal the direct
    rasterizer at that shape and the oracle; training runs."""
    ensure_built()
    sc = _scene(n=8000, seed=17)
    cams = _cams(2, seed=18)
    with session.Session(_cfg(sc.n, tile=tile)) as s:
        s.add(sc)
        img = s.wait(s.submit(RENDER, cams[0], want_image=True))
        s.wait(s.submit(TRAIN, cams[1], target=_targets(cams[1:], seed=19)[0]))
        st = s.stats()
    assert st["failed"] == 0 and st["iterations"] == 1
    dev = torch.device("cuda:0")
    a = raster.Arena.from_scene(sc, dev)
    r = raster.Rasterizer(sc.n, sc.sh_degree, cams[:1], device=dev, tile=tile)
    d, _ = r.forward(a, raster.poses_tensor(cams[:1], dev), r.new_image(), None)
    assert np.array_equal(img, r.split(d.cpu(), 3)[0].numpy())
    ref = oracle.render(sc, cams[:1], tile=tile)
    ok = (ref["flags"][0] & 1) == 0
    assert np.abs(img.astype(np.float64) - ref["image"][0])[:, ok].max() <= IMG_TOL


def test_hierarchy_session_never_draws_unused_slots(cuda_device):
    """With a hierarchy, leaf slots not yet filled (rows past the added
    Gaussians) hold no node: renders and trains skip them, so a render equals
    the direct render of the Gaussians added (a zeroed slot would be a unit
    Gaussian at the origin, in front of this camera)."""
    ensure_built()
    sc = _clustered_scene(500, 4, seed=9)
    cam = synth.Camera(np.eye(3, dtype=np.float32), np.array([0.0, 0.0, 5.0], np.float32), 300.0, 300.0, 160.0,
                       120.0, 320, 240)  # the world origin 5 m ahead
    cfg = _cfg(sc.n + 1000, sh_degree=1, lod=True, lod_tau=1.0, max_width=320, max_height=240)
    with session.Session(cfg) as s:
        s.add(sc)
        img = s.wait(s.submit(RENDER, cam, want_image=True))
        s.wait(s.submit(TRAIN, cam, target=_targets([cam], seed=2)[0]))
        st = s.stats()
    assert st["failed"] == 0 and st["iterations"] == 1
    assert np.array_equal(img, _direct_render(sc, cam))
