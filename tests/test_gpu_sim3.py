"""The loop-closure update on the GPU (gs_sim3_update) against the FP64
oracle, and the invariance of the GPU's own render when scene and camera
move together."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from paper_2607_14481_b300 import raster, synth
from gpu_util import IMG_TOL, ensure_built, gpu_forward

pytestmark = pytest.mark.gpu


def _sim3(g, s_sigma=0.3):
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([q, g.normal(size=3), [np.exp(g.normal(0, s_sigma))]])


def test_sim3_update_matches_oracle(cuda_device):
    ensure_built()
    g = np.random.default_rng(3)
    sc = synth.random_scene(100_000, 4, 1, (-5, -2, -5), (5, 2, 5), -3.0, 0.5)
    K = 16
    kf = g.integers(-1, K, sc.n).astype(np.int32)
    kf[:10] = K + 3  # ids without a correction: skipped and reported
    S = np.stack([_sim3(g) for _ in range(K)]).astype(np.float32)
    dev = torch.device("cuda:0")
    arena = raster.Arena.from_scene(sc, dev)
    before = arena.to_natural()
    status = raster.sim3_update(arena, torch.from_numpy(kf).to(dev), torch.from_numpy(S).to(dev))
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    after = arena.to_natural()
    kf_o = np.where(kf >= K, -1, kf)
    mu, ls, q = oracle.sim3_update(before["means"], before["log_scales"], before["quats"], kf_o,
                                   S.astype(np.float64))
    scale = np.maximum(1.0, np.abs(mu))
    assert np.all(np.abs(after["means"] - mu) <= 4e-6 * scale)
    assert np.abs(after["log_scales"] - ls).max() <= 2e-6
    assert np.abs(after["quats"] - q).max() <= 2e-6 * max(1.0, np.abs(q).max())
    same = kf_o < 0
    for k in ("means", "log_scales", "quats"):
        assert np.array_equal(after[k][same], before[k][same]), k
    assert np.array_equal(after["opa_logits"], before["opa_logits"])
    assert np.array_equal(after["sh"], before["sh"])


def test_gpu_render_invariant_when_scene_and_camera_move_together(cuda_device):
    sc, cams, _ = synth.plain_small()
    g = np.random.default_rng(5)
    S = _sim3(g)
    S[7] = 1.6
    r, arena, poses, img, alpha = gpu_forward(sc, cams)
    a_img, a_alpha = img.clone(), alpha.clone()
    dev = torch.device("cuda:0")
    raster.sim3_update(arena, torch.zeros(sc.n, dtype=torch.int32, device=dev),
                       torch.from_numpy(S[None].astype(np.float32)).to(dev))
    R = Rotation.from_quat([S[1], S[2], S[3], S[0]]).as_matrix()
    c = cams[0]
    Rc = np.asarray(c.R, np.float64)
    cam2 = synth.Camera((Rc @ R.T).astype(np.float32), (S[7] * np.asarray(c.t, np.float64) - Rc @ R.T @ S[4:7])
                        .astype(np.float32), c.fx, c.fy, c.cx, c.cy, c.width, c.height)
    r.set_cameras([cam2])
    r.forward(arena, raster.poses_tensor([cam2], dev), img, alpha)
    torch.cuda.synchronize()
    # single-precision parameters and pose: the same renders up to FP32 rounding
    ref = oracle.render(sc, cams)
    ok = (ref["flags"][0] & 1) == 0
    d = np.abs(r.split(img.cpu(), 3)[0].numpy() - r.split(a_img.cpu(), 3)[0].numpy())
    assert d[:, ok].max() <= 2 * IMG_TOL
