"""The progressive hierarchy on the GPU (gs_hier_analyze, gs_hier_refine,
gs_project_hier) against the FP64 oracle, step by step: each step starts the
oracle from the GPU's state before it, and compares bit-exactly the integer
outcome (counts, parent and child links, active flags, node count) and, for
merged nodes, the parameters within single-precision rounding.  A sequence of
analyses from a far camera, a reload from a near one and a second analysis
exercises grouping, reload and the parent pull.  The view cut of the
projection equals the oracle's refinement of a copy of the active set, and the
image rendered through it equals the oracle's render of those nodes."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import raster, synth
from gpu_util import IMG_TOL, ensure_built

pytestmark = pytest.mark.gpu

F = 300.0
PARAM_TOL = 2e-5
COV_TOL = 2e-5


def _cam(z=0.0, W=640, H=480):
    return synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, -z], np.float32), F, F, W / 2, H / 2, W, H)


def _scene(n, seed, deg=1, small=0.7):
    """Means in a box in front of the camera; screen sizes (from z = 0)
    either in [0.05, 0.3] px or in [1.5, 4] px, away from both thresholds."""
    g = np.random.default_rng(seed)
    z = g.uniform(8, 40, n)
    means = np.column_stack([g.uniform(-0.4, 0.4, n) * z, g.uniform(-0.3, 0.3, n) * z, z])
    S = np.where(g.random(n) < small, g.uniform(0.05, 0.3, n), g.uniform(1.5, 4.0, n))
    base = np.log(S * z / (3 * F))
    ls = base[:, None] - np.abs(g.normal(0, 0.3, (n, 3)))
    ls[np.arange(n), g.integers(0, 3, n)] = base  # the largest axis sets S
    sc = synth.random_scene(n, seed + 1, deg, (0, 0, 0), (1, 1, 1), 0.0, 1.0)
    return synth.Scene(means.astype(np.float32), ls.astype(np.float32), sc.quats, sc.opa_logits, sc.sh)


def _cov(ls, q):
    q = np.asarray(q, np.float64)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    return R @ (np.exp(2 * np.asarray(ls, np.float64))[:, :, None] * np.transpose(R, (0, 2, 1)))


def _gpu_state(arena, hier):
    torch.cuda.synchronize()
    s = hier.state()
    nat = arena.to_natural()
    st = oracle.HierState.from_arrays(nat, s["parent"], s["child"], s["active"], s["n_nodes"])
    return st, s


def _compare(st_ref, st_gpu, n0):
    """Integer state exactly; parameters of the nodes created after n0."""
    n = st_ref.n_nodes
    assert st_gpu.n_nodes == n
    assert np.array_equal(st_gpu.parent[:n], st_ref.parent[:n])
    assert np.array_equal(st_gpu.child[:n], st_ref.child[:n])
    assert np.array_equal(st_gpu.active[:n], st_ref.active[:n])
    if n > n0:
        c = slice(n0, n)
        assert np.abs(st_gpu.means[c] - st_ref.means[c]).max() <= PARAM_TOL * max(1.0, np.abs(st_ref.means).max())
        cg, cr = _cov(st_gpu.log_scales[c], st_gpu.quats[c]), _cov(st_ref.log_scales[c], st_ref.quats[c])
        for k in range(n - n0):
            assert np.abs(cg[k] - cr[k]).max() <= COV_TOL * np.abs(cr[k]).max(), k
        assert np.abs(st_gpu.sh[c] - st_ref.sh[c]).max() <= PARAM_TOL
        sig = lambda x: 1 / (1 + np.exp(-x))
        assert np.abs(sig(st_gpu.opa_logits[c]) - sig(st_ref.opa_logits[c])).max() <= PARAM_TOL


def _is_cut(st):
    n = st.n_nodes
    for i in range(n):
        if st.child[i, 0] >= 0:
            continue
        k, c = 0, i
        while c >= 0:
            k += int(st.active[c])
            c = st.parent[c]
        if k != 1:
            return False
    return True


def _setup(n=4000, seed=3, deg=1):
    ensure_built()
    dev = torch.device("cuda:0")
    sc = _scene(n, seed, deg)
    arena = raster.Arena.from_scene(sc, dev, capacity=3 * n)
    hier = raster.Hierarchy(arena, n)
    return sc, arena, hier


def test_analyze_reload_pull_sequence_matches_oracle(cuda_device):
    sc, arena, hier = _setup()
    n0 = sc.n
    far, near = _cam(0.0), _cam(7.0)
    seen = {"groups": 0, "pulled": 0, "reloaded": 0}
    steps = [("analyze", far), ("refine", near), ("analyze", far), ("analyze", _cam(-10.0)), ("refine", _cam(4.0)),
             ("analyze", _cam(-20.0))]
    for kind, cam in steps:
        st_in, _ = _gpu_state(arena, hier)
        n_before = st_in.n_nodes
        ref = st_in.copy()
        if kind == "analyze":
            out = oracle.hier_analyze(ref, cam)
            assert not out["amb"][:n_before].any(), "a screen size within rounding of tau_l: pick another seed"
            hier.analyze(cam)
            st_gpu, s = _gpu_state(arena, hier)
            want = [out["info"][k] for k in ("n_nodes", "triggered", "candidates", "active", "pulled", "groups",
                                             "grouped")]
            assert list(s["info"][:7]) == want and s["info"][7] == 0
            seen["groups"] += out["info"]["groups"]
            seen["pulled"] += out["info"]["pulled"]
        else:
            k, amb = oracle.hier_refine(ref, cam)
            assert not amb.any(), "a reload decision within rounding: pick another seed"
            hier.refine(cam)
            st_gpu, s = _gpu_state(arena, hier)
            assert int(s["info"][0]) == k
            seen["reloaded"] += k
        _compare(ref, st_gpu, n_before)
        assert _is_cut(st_gpu)
    assert seen["groups"] > 0 and seen["pulled"] > 0 and seen["reloaded"] > 0, seen


def test_view_cut_and_render_match_oracle(cuda_device):
    sc, arena, hier = _setup(seed=5)
    hier.analyze(_cam(0.0))
    hier.analyze(_cam(-12.0))
    st, s = _gpu_state(arena, hier)
    assert st.n_nodes > sc.n
    for cam in (_cam(6.0), _cam(0.0), _cam(-25.0)):
        want = oracle.hier_view_cut(st, cam)
        c = st.copy()
        _, amb = oracle.hier_refine(c, cam)
        assert not amb.any()
        dev = torch.device("cuda:0")
        r = raster.Rasterizer(st.n_nodes, sc.sh_degree, [cam], device=dev)
        poses = raster.poses_tensor([cam], dev)
        r.project_hier(hier, poses, tau_h=1.0)
        got = (r.splat_arrays()["touched"][0] > 0).astype(np.uint8)
        # culled by the projection itself (off screen, behind the near plane)
        # are a subset of the cut's nodes
        assert np.all(got <= want)
        ref_img = oracle.render(synth.Scene(st.means32[:st.n_nodes][want == 1],
                                            st.log_scales[:st.n_nodes][want == 1].astype(np.float32),
                                            st.quats[:st.n_nodes][want == 1].astype(np.float32),
                                            st.opa_logits[:st.n_nodes][want == 1].astype(np.float32),
                                            st.sh[:st.n_nodes][want == 1].astype(np.float32)), [cam])
        r.bin_sort()
        img = r.new_image()
        r.render_fwd(img, None)
        g_img = r.split(img.cpu(), 3)[0].numpy().astype(np.float64)
        ok = (ref_img["flags"][0] & 1) == 0
        assert np.abs(g_img - ref_img["image"][0])[:, ok].max(initial=0.0) <= IMG_TOL
        assert (~ok).mean() < 0.02
        # every node of the cut that the projection keeps is visible on screen
        missing = np.flatnonzero((want == 1) & (got == 0))
        proj = oracle.render(synth.Scene(st.means32[missing], st.log_scales[missing].astype(np.float32),
                                         st.quats[missing].astype(np.float32),
                                         st.opa_logits[missing].astype(np.float32),
                                         st.sh[missing].astype(np.float32)), [cam], want_proj=True,
                             windows=[(0, 0, 8, 8)])["proj"] if len(missing) else None
        if proj is not None:
            vis_col = oracle.PROJ_FIELDS.index("vis")
            amb_col = oracle.PROJ_FIELDS.index("bin_amb")
            assert np.all((proj[0][:, vis_col] == 0) | (proj[0][:, amb_col] == 1))


def test_moments_of_changed_nodes_are_zeroed(cuda_device):
    sc, arena, hier = _setup(n=2000, seed=9, deg=0)
    m, v = arena.like(), arena.like()
    m.buf.fill_(1.0)
    v.buf.fill_(2.0)
    before = hier.state()
    hier.analyze(_cam(0.0), m=m, v=v)
    after = hier.state()
    n = after["n_nodes"]
    changed = np.flatnonzero(before["active"][:n] != after["active"][:n])
    assert len(changed) > 0
    mm = m.to_natural()
    for key in ("means", "log_scales", "quats", "sh"):
        assert np.all(mm[key][changed] == 0.0), key
    same = np.setdiff1d(np.arange(sc.n), changed)
    assert np.all(mm["means"][same] == 1.0) and np.all(v.to_natural()["log_scales"][same] == 2.0)


def test_no_merge_below_the_trigger_and_capacity_guard(cuda_device):
    # 10% candidates: nothing changes
    sc, arena, hier = _setup(n=3000, seed=11)
    small = _scene(3000, 11, small=0.1)
    arena2 = raster.Arena.from_scene(small, torch.device("cuda:0"), capacity=6000)
    h2 = raster.Hierarchy(arena2, 3000)
    h2.analyze(_cam(0.0))
    s = h2.state()
    assert s["info"][1] == 0 and s["n_nodes"] == 3000 and s["active"][:3000].all()
    # capacity too small for the new nodes: nothing merged, status bit set
    arena3 = raster.Arena.from_scene(sc, torch.device("cuda:0"), capacity=sc.n + 5)
    h3 = raster.Hierarchy(arena3, sc.n)
    h3.analyze(_cam(0.0))
    s3 = h3.state()
    assert s3["info"][1] == 1 and s3["info"][7] & 1 and s3["n_nodes"] == sc.n
    st3, _ = _gpu_state(arena3, h3)
    assert _is_cut(st3)


def test_render_cut_from_the_roots_matches_oracle(cuda_device):
    """gs_project_hier_render: the nodes the projection keeps are the oracle's
    render cut (Sec. 6.2, descent from the roots while coarser than tau) up to
    the projection's own culling and decisions within rounding of tau; the
    image equals the oracle's render of the cut, and far views draw merged
    nodes whatever the active set holds."""
    sc, arena, hier = _setup(seed=5)
    hier.analyze(_cam(0.0))
    hier.analyze(_cam(-12.0))
    hier.refine(_cam(8.0))  # the active set back to fine nodes near that camera
    st, s = _gpu_state(arena, hier)
    assert st.n_nodes > sc.n
    merged_drawn = 0
    dev = torch.device("cuda:0")
    for cam, tau in ((_cam(6.0), 1.0), (_cam(0.0), 1.0), (_cam(-25.0), 1.0), (_cam(-25.0), 4.0)):
        want, amb = oracle.hier_render_cut(st, cam, tau=tau)
        r = raster.Rasterizer(st.n_nodes, sc.sh_degree, [cam], device=dev)
        r.project_hier(hier, raster.poses_tensor([cam], dev), tau_h=tau, from_roots=True)
        got = (r.splat_arrays()["touched"][0] > 0).astype(np.uint8)
        ok = amb == 0
        assert np.all(got[ok] <= want[ok])
        missing = np.flatnonzero(ok & (want == 1) & (got == 0))
        if len(missing):
            proj = oracle.render(synth.Scene(st.means32[missing], st.log_scales[missing].astype(np.float32),
                                             st.quats[missing].astype(np.float32),
                                             st.opa_logits[missing].astype(np.float32),
                                             st.sh[missing].astype(np.float32)), [cam], want_proj=True,
                                 windows=[(0, 0, 8, 8)])["proj"][0]
            vis_col = oracle.PROJ_FIELDS.index("vis")
            amb_col = oracle.PROJ_FIELDS.index("bin_amb")
            assert np.all((proj[:, vis_col] == 0) | (proj[:, amb_col] == 1))
        merged_drawn += int(got[sc.n:].sum())
        if amb.any():
            continue
        ref_img = oracle.render(synth.Scene(st.means32[:st.n_nodes][want == 1],
                                            st.log_scales[:st.n_nodes][want == 1].astype(np.float32),
                                            st.quats[:st.n_nodes][want == 1].astype(np.float32),
                                            st.opa_logits[:st.n_nodes][want == 1].astype(np.float32),
                                            st.sh[:st.n_nodes][want == 1].astype(np.float32)), [cam])
        r.bin_sort()
        img = r.new_image()
        r.render_fwd(img, None)
        g_img = r.split(img.cpu(), 3)[0].numpy().astype(np.float64)
        okp = (ref_img["flags"][0] & 1) == 0
        assert np.abs(g_img - ref_img["image"][0])[:, okp].max(initial=0.0) <= IMG_TOL
    assert merged_drawn > 0
