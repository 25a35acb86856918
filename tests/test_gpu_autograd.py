"""The torch.autograd adjoint (differentiation check): 256 Gaussians, SH
degree 3, three 64x64 views, mean-squared-error loss written in torch on the
rendered image; the adjoint keeps no per-pixel state and takes the replay
backward (transmittance recomputed in reverse).  autograd gradients of every parameter group and of the camera
poses must match the FP64 oracle's analytic gradient (itself pinned to dual
numbers and central finite differences) within 1e-3 relative, and a sample of
coordinates is checked directly against central differences (step 1e-4) of the
FP64 oracle forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_14481_b300 import autograd, raster, synth
from gpu_util import compare_grads, ensure_built

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_and_finite_differences(cuda_device):
    ensure_built()
    sc, cams, targets = synth.diffcheck()
    # weight 0 on pixels whose value hangs on a near-threshold decision; the
    # margins are wide enough that the finite-difference steps below (1e-4)
    # cross no decision either (including a swap of nearly equal depths)
    ref = oracle.render(sc, cams, margins=[0.05, 0.02, 0.02, 1e-3, 0.02, 0.02, 1e-4])
    mask = [torch.from_numpy((f == 0).astype(np.float32)).to(cuda_device) for f in ref["flags"]]
    arena = raster.Arena.from_scene(sc, cuda_device)
    arena.buf.requires_grad_(True)
    poses = raster.poses_tensor(cams, cuda_device)
    twist = torch.zeros((len(cams), 6), dtype=torch.float32, device=cuda_device, requires_grad=True)
    rast = raster.Rasterizer(sc.n, sc.sh_degree, cams, device=cuda_device)
    img, _ = autograd.render(arena, rast, poses, twist)
    # nothing per pixel is kept for the backward (it replays the tile lists)
    assert len(img.grad_fn.saved_tensors) == 0
    views = rast.split(img, 3)
    n = sum(t.size for t in targets)
    loss = 0.0
    for v, t, mk in zip(views, targets, mask):
        d = v - torch.from_numpy(t).to(cuda_device)
        loss = loss + (mk[None] * d * d).sum()
    loss = loss / n
    loss.backward()
    torch.cuda.synchronize()

    gbuf = raster.Arena(sc.n, sc.sh_degree, cuda_device, buf=arena.buf.grad.detach().clone())
    g_gpu = gbuf.to_natural()
    g_gpu["pose"] = twist.grad.cpu().numpy().astype(np.float64)
    # the oracle's gradient of the same masked loss (upstream gradient from its own image)
    dimg = [2.0 * (f == 0)[None] * (im - t) / n for im, t, f in zip(ref["image"], targets, ref["flags"])]
    g_ref = oracle.backward(sc, cams, dimg)
    compare_grads(g_gpu, g_ref)

    # direct central differences of the FP64 forward on sampled coordinates
    h = 1e-4
    wts = dimg

    def L(scn, cs):
        out = oracle.render(scn, cs)["image"]
        return sum(float((w * o).sum()) for w, o in zip(wts, out))

    rng = np.random.default_rng(0)
    arrays = {"means": sc.means, "log_scales": sc.log_scales, "quats": sc.quats,
              "opa_logits": sc.opa_logits, "sh": sc.sh}
    for group, arr in arrays.items():
        gmax = np.abs(g_ref[group]).max()
        for fi in rng.choice(arr.size, size=4, replace=False):
            idx = np.unravel_index(fi, arr.shape)
            vals = []
            for s in (1, -1):
                sp = sc.copy()
                a = getattr(sp, group).astype(np.float64)
                a[idx] += s * h
                setattr(sp, group, a)
                vals.append(L(sp, cams))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g_gpu[group][idx] - fd) <= 2e-3 * gmax + 1e-9, (group, idx)
