"""The level-of-detail hierarchy on the GPU against the FP64 oracle:
grouping (parent of every node) bit-exact, coarse-node parameters within
single-precision rounding (covariances compared through their factors, which
are unique only up to the eigenvector choice), the cut per view, and images
rendered through the cut against the oracle's render of its own cut."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import _lib, raster, synth
from gpu_util import IMG_TOL, ensure_built

pytestmark = pytest.mark.gpu

COV_TOL = 2e-5     # per node: max |Sigma_gpu - Sigma_ref| / max |Sigma_ref| (FP32 merge + Jacobi)
PARAM_TOL = 2e-5   # means (scene units ~1), SH coefficients, opacity


def _cov(ls, q):
    q = np.asarray(q, np.float64)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    return R @ (np.exp(2 * np.asarray(ls, np.float64))[:, :, None] * np.transpose(R, (0, 2, 1)))


def _gpu_build(sc):
    ensure_built()
    dev = torch.device("cuda:0")
    cap = int(_lib.load().gs_lod_nodes(sc.n))
    arena = raster.Arena.from_scene(sc, dev, capacity=cap)
    lod = raster.LodHierarchy(arena, sc.n)
    lod.build()
    torch.cuda.synchronize()
    return arena, lod


@pytest.mark.parametrize("n,deg", [(20000, 3), (1, 0), (8, 1), (9, 1), (65, 2), (4097, 0)])
def test_lod_build_matches_oracle(cuda_device, n, deg):
    sc = synth.random_scene(n, 11 + n, deg, (-4, -1, -4), (4, 1, 4), -2.5, 0.5)
    ref = oracle.lod_build(sc)
    arena, lod = _gpu_build(sc)
    N = lod.n_nodes
    assert N == n + ref["n1"] + ref["n2"]
    assert np.array_equal(lod.parent[:N].cpu().numpy(), ref["parent"].astype(np.int32))
    nat = arena.to_natural()
    # leaves untouched
    assert np.array_equal(nat["means"][:n].astype(np.float32), np.asarray(sc.means, np.float32))
    c = slice(n, N)
    assert np.abs(nat["means"][c] - ref["means"]).max() <= PARAM_TOL * max(1.0, np.abs(ref["means"]).max())
    cg = _cov(nat["log_scales"][c], nat["quats"][c])
    for k in range(N - n):
        assert np.abs(cg[k] - ref["cov"][k]).max() <= COV_TOL * np.abs(ref["cov"][k]).max(), k
    assert np.abs(nat["sh"][c] - ref["sh"]).max() <= PARAM_TOL
    sig = lambda x: 1 / (1 + np.exp(-x))
    assert np.abs(sig(nat["opa_logits"][c]) - sig(ref["opa_logits"])).max() <= PARAM_TOL
    assert np.all(np.abs(np.linalg.norm(nat["quats"][c], axis=1) - 1) < 1e-5)


def test_lod_identical_children_identity(cuda_device):
    base = synth.random_scene(1, 3, 1, (0, 0, 0), (0, 0, 0), -2.0, 0.3)
    sc = base.subset(np.zeros(8, np.int64))
    arena, lod = _gpu_build(sc)
    nat = arena.to_natural()
    leaf = _cov(nat["log_scales"][:1], nat["quats"][:1])[0]
    for node in (8, 9):  # the level-1 node and the root
        assert np.abs(nat["means"][node] - nat["means"][0]).max() < 1e-6
        assert np.abs(_cov(nat["log_scales"][node:node + 1], nat["quats"][node:node + 1])[0] - leaf).max() \
            <= COV_TOL * np.abs(leaf).max()
        assert np.abs(nat["sh"][node] - nat["sh"][0]).max() < 1e-6


@pytest.mark.parametrize("dist,tau", [(40.0, 16.0), (20.0, 16.0), (40.0, 1.0)])
def test_lod_cut_and_render_match_oracle(cuda_device, dist, tau):
    sc = synth.random_scene(6000, 12, 1, (-4, -1, -4), (4, 1, 4), -2.5, 0.5)
    ref = oracle.lod_build(sc)
    n = sc.n
    nodes = synth.Scene(np.concatenate([np.asarray(sc.means, np.float64), ref["means"]]),
                        np.concatenate([np.asarray(sc.log_scales, np.float64), ref["log_scales"]]),
                        np.concatenate([np.asarray(sc.quats, np.float64), ref["quats"]]),
                        np.concatenate([np.asarray(sc.opa_logits, np.float64), ref["opa_logits"]]),
                        np.concatenate([np.asarray(sc.sh, np.float64), ref["sh"]]))
    cam = synth.look_at((0.0, -0.5, -dist), (0, 0, 0), 300.0, 300.0, 160, 120, 320, 240)
    cut = oracle.lod_cut(nodes.means, nodes.log_scales, ref["parent"], n, cam, tau=tau)
    assert not cut["amb"].any()
    sel = np.flatnonzero(cut["selected"])
    ref_img = oracle.render(nodes.subset(sel), [cam])

    arena, lod = _gpu_build(sc)
    dev = torch.device("cuda:0")
    r = raster.Rasterizer(lod.n_nodes, sc.sh_degree, [cam], device=dev)
    img, alpha = r.forward(arena, raster.poses_tensor([cam], dev), r.new_image(), r.new_alpha(), lod=lod, tau=tau)
    torch.cuda.synchronize()
    touched = r.splat_views()["touched"][0].cpu().numpy()
    vis = np.flatnonzero(touched > 0)
    assert set(vis.tolist()) <= set(sel.tolist())  # only nodes of the cut are projected
    if dist > 30 and tau > 8:
        assert (vis >= n).sum() > 0  # coarse nodes are rendered
    ok = (ref_img["flags"][0] & 1) == 0
    im = r.split(img.cpu(), 3)[0].numpy().astype(np.float64)
    assert np.abs(im - ref_img["image"][0])[:, ok].max() <= IMG_TOL
    assert (~ok).mean() < 0.02
