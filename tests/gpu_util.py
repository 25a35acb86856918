"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and bring results back in the oracle's natural layout."""
import numpy as np
import torch

from paper_2607_14481_b300 import build, raster
from paper_2607_14481_b300.synth import Scene

IMG_TOL = 1e-5     # max-abs per pixel channel, GPU FP32 vs oracle FP64
GRAD_TOL = 1e-3    # per group: ||g_gpu - g_ref||_inf / max(||g_ref||_inf, 1e-8)


def ensure_built():
    build.build()


def gpu_forward(sc: Scene, cams, bg=(0.0, 0.0, 0.0), znear=0.2, clamp_j=True, capacity=None, keep_keys=False,
                tile=(16, 16)):
    ensure_built()
    dev = torch.device("cuda:0")
    arena = raster.Arena.from_scene(sc, dev)
    poses = raster.poses_tensor(cams, dev)
    r = raster.Rasterizer(sc.n, sc.sh_degree, cams, bg=bg, znear=znear, clamp_jacobian=clamp_j,
                          capacity=capacity, device=dev, keep_keys=keep_keys, tile=tile)
    img = r.new_image()
    alpha = r.new_alpha()
    r.forward(arena, poses, img, alpha, check=True)
    torch.cuda.synchronize()
    return r, arena, poses, img, alpha


def gpu_backward(r, arena, poses, dimage_list, dalpha_list=None, image=None):
    """image: the forward's output, selecting the single front-to-back pass
    (when there is no alpha gradient)."""
    dev = arena.buf.device
    dimg = torch.from_numpy(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in dimage_list])).to(dev)
    dal = None
    if dalpha_list is not None:
        dal = torch.from_numpy(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in dalpha_list])).to(dev)
    grads = arena.like()
    grads.buf.fill_(float("nan"))  # every element must be written
    dpose = torch.full((r.views, 6), float("nan"), dtype=torch.float32, device=dev)
    r.backward(arena, poses, dimg, dal, grads, dpose, image)
    torch.cuda.synchronize()
    g = grads.to_natural()
    g["pose"] = dpose.cpu().numpy().astype(np.float64)
    return g


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-8))


def compare_grads(g_gpu, g_ref, tol=GRAD_TOL, groups=("means", "log_scales", "quats", "opa_logits", "sh", "pose")):
    errs = {k: rel_err(g_gpu[k], g_ref[k]) for k in groups}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"gradient parity failed: {errs}"
    assert np.all(g_gpu["means_pad"] == 0.0)
    return errs


def fused_step(r, arena, poses, target, kind, alpha=None):
    """gs_render_fused then gs_render_bwd_gaussians on the rasterizer's current
    tile lists: image, loss, gradients (natural layout, pose included)."""
    dev = arena.buf.device
    img = r.new_image()
    img.fill_(float("nan"))
    loss = torch.full((1,), float("nan"), dtype=torch.float32, device=dev)
    r.fused(target, kind, img, alpha, loss)
    grads = arena.like()
    grads.buf.fill_(float("nan"))
    dpose = torch.full((r.views, 6), float("nan"), dtype=torch.float32, device=dev)
    r.backward_gaussians(arena, poses, grads, dpose)
    torch.cuda.synchronize()
    g = grads.to_natural()
    g["pose"] = dpose.cpu().numpy().astype(np.float64)
    return img, float(loss.item()), g


def target_near(img_views, flags, rng, lo=0.02, hi=0.2):
    """Targets equal to the image plus a random offset of magnitude in
    [lo, hi] and random sign, and equal to the image where the oracle flags a
    pixel (there both losses' gradients are exactly 0).  Returns the per-view
    targets as float32 arrays [3, H, W]."""
    out = []
    for im, f in zip(img_views, flags):
        im = np.asarray(im, np.float32)
        d = rng.uniform(lo, hi, size=im.shape) * rng.choice([-1.0, 1.0], size=im.shape)
        t = (im.astype(np.float64) + d).astype(np.float32)
        out.append(np.where((f != 0)[None], im, t).astype(np.float32))
    return out


def loss_grad(img_views, tgt_views, kind, count):
    """dL/dimage of the L1 (kind 0) or MSE (kind 1) mean loss, in float64 from
    the float32 images and targets (the gradient the fused kernel forms)."""
    out = []
    for im, t in zip(img_views, tgt_views):
        d = np.asarray(im, np.float32).astype(np.float64) - np.asarray(t, np.float32).astype(np.float64)
        out.append(np.sign(d) / count if kind == 0 else 2.0 * d / count)
    return out
