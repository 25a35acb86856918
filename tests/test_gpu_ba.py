"""GPU local bundle adjustment (gs_ba_solve) against the FP64 oracle on the
same seeded problems: costs, decisions and final states.

Tolerances follow from the arithmetic: residuals and Jacobians are float32
(relative rounding 6e-8 on pixel coordinates of ~1000, i.e. ~1e-4 px), the
reduced system is solved to float64 accuracy, and the step's relative error
is ~1e-5 (float32 Schur terms, cond(S) ~ 1e8 before scaling).  Costs agree to
1e-4 relative; after convergence the states agree to the float32 resolution of
the optimum (rotations 2e-5, translations and landmarks ~1e-4 of the scene
scale, focal 1e-5 relative)."""
import numpy as np
import pytest
import torch

from oracle import ba as oba
from paper_2607_14481_b300 import _lib, synth
from paper_2607_14481_b300.ba import BundleAdjuster, bundle_adjust

pytestmark = pytest.mark.gpu


def _problem(seed, n_cams=8, n_points=300, M=5, n_fixed=3, noise=0.5):
    p = synth.ba_problem(seed, n_cams=n_cams, n_points=n_points, obs_per_point=M, n_fixed=n_fixed, noise_px=noise)
    fixed = np.zeros(n_cams, bool)
    fixed[:n_fixed] = True
    return p, fixed


def _both(p, fixed, iters, obs_cam=None, opt_focal=True, lambda0=1e-3):
    cam = p["obs_cam"] if obs_cam is None else obs_cam
    o = oba.solve(p["poses0"], p["points0"], p["f0"], cam, p["obs_uv"], p["cx"], p["cy"], fixed,
                  opt_focal=opt_focal, iters=iters, lambda0=lambda0)
    g = bundle_adjust(p["poses0"], p["points0"], p["f0"], cam, p["obs_uv"], p["cx"], p["cy"], fixed,
                      opt_focal=opt_focal, iters=iters, lambda0=lambda0)
    return o, g


def _project(P, X, f, p, cam):
    R, t = oba.split_poses(P)
    r, valid = oba.residuals(R, t, np.asarray(X, np.float64), float(f), cam, np.zeros(cam.shape + (2,)),
                             p["cx"], p["cy"])
    return r, valid


def _compare_state(o, g, fixed, p, cam=None, rot=2e-5, trans=2e-4, px=2e-2, cost_rel=2e-6):
    """The GPU's final state against the oracle's: fixed keyframes untouched,
    the oracle's cost of the GPU state within the float32 evaluation noise of
    the oracle's optimum (pixel coordinates ~1000 carry ~1e-4 px of rounding:
    1e-6 px^2 per residual, or 2e-6 of the cost), poses close, reprojections
    within px pixels in RMS (a landmark seen along nearly parallel rays is
    loosely determined in depth: its reprojections may move by a tenth of a
    pixel at no measurable cost)."""
    cam = p["obs_cam"] if cam is None else cam
    P, X, f, tr, status = g
    assert status == 0
    assert np.array_equal(P[fixed], p["poses0"][fixed])  # fixed keyframes are never written
    R, t = oba.split_poses(P)
    m = 2 * int(np.count_nonzero(cam >= 0))
    assert oba.cost(R, t, np.asarray(X, np.float64), float(f), cam, p["obs_uv"], p["cx"], p["cy"]) == \
        pytest.approx(o["cost"], rel=cost_rel, abs=1e-6 * m)
    Po = o["poses"].reshape(-1, 3, 4)
    Pg = P.reshape(-1, 3, 4)
    assert np.abs(Pg[:, :, :3] - Po[:, :, :3]).max() < rot
    assert np.abs(Pg[:, :, 3] - Po[:, :, 3]).max() < trans
    rg, vg = _project(P, X, f, p, cam)
    ro, vo = _project(o["poses"], o["points"], o["f"], p, cam)
    assert np.array_equal(vg, vo)
    assert np.sqrt(np.mean((rg - ro)[vg] ** 2)) < px
    assert np.abs(rg - ro).max() < 10 * px
    assert abs(f - o["f"]) < 1e-5 * o["f"]


def test_one_iteration_matches_oracle(cuda_device):
    p, fixed = _problem(1)
    o, g = _both(p, fixed, 1)
    tr = g[3]
    assert tr[0, 0] == pytest.approx(o["trace"][0, 0], rel=1e-4)
    assert tr[0, 1] == pytest.approx(o["trace"][0, 1], rel=1e-4)
    assert tr[0, 2] == o["trace"][0, 2] and tr[0, 3] == o["trace"][0, 3] == 1.0
    # one step from a perturbed start (far from the optimum the cost is first
    # order in the step's ~1e-5 relative error)
    _compare_state(o, g, fixed, p, cost_rel=2e-5)


@pytest.mark.parametrize("M", [3, 5, 8, 12])
def test_slot_counts_and_group_sizes(cuda_device, M):
    p, fixed = _problem(2 + M, n_cams=max(10, M + 2), n_points=257, M=M, n_fixed=2)
    o, g = _both(p, fixed, 4)
    assert np.allclose(g[3][:, 0], o["trace"][:, 0], rtol=1e-4)
    assert np.array_equal(g[3][:, 3], o["trace"][:, 3])
    _compare_state(o, g, fixed, p)


def test_full_size_ten_iterations(cuda_device):
    """20 keyframes (4 fixed), 10,000 landmarks, 8 slots each: the benchmark's
    problem, 10 iterations."""
    p, fixed = _problem(1, n_cams=20, n_points=10_000, M=8, n_fixed=4)
    o, g = _both(p, fixed, 10)
    tr_o, tr_g = o["trace"], g[3]
    assert np.allclose(tr_g[:, 0], tr_o[:, 0], rtol=1e-4)
    decisive = np.abs(tr_o[:, 1] - tr_o[:, 0]) > 1e-4 * tr_o[:, 0]
    assert np.array_equal(tr_g[decisive, 3], tr_o[decisive, 3])
    assert g[3][-1, 0] == pytest.approx(o["cost"], rel=1e-4)
    _compare_state(o, g, fixed, p)


def test_noise_free_reaches_ground_truth(cuda_device):
    p, fixed = _problem(5, n_cams=8, n_points=400, M=5, n_fixed=3, noise=0.0)
    P, X, f, tr, status = bundle_adjust(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"],
                                        p["cy"], fixed, iters=15)
    assert status == 0
    assert tr[0, 0] > 1e3 and tr[-1, 0] < 1e-3
    assert np.abs(P - p["poses_true"]).max() < 1e-4
    assert abs(f - p["f_true"]) < 1e-5 * p["f_true"]


def test_fixed_focal(cuda_device):
    p, fixed = _problem(6)
    o, g = _both(p, fixed, 5, opt_focal=False)
    assert g[2] == np.float32(p["f0"])
    _compare_state(o, g, fixed, p)


def test_bad_slots_are_ignored_and_flagged(cuda_device):
    p, fixed = _problem(7, n_points=200, M=5)
    bad = p["obs_cam"].copy()
    bad[3, 1] = 99          # out of range
    bad[10, 4] = bad[10, 0]  # repeated keyframe
    clean = bad.copy()
    clean[3, 1] = -1
    clean[10, 4] = -1
    o = oba.solve(p["poses0"], p["points0"], p["f0"], clean, p["obs_uv"], p["cx"], p["cy"], fixed, iters=3)
    P, X, f, tr, status = bundle_adjust(p["poses0"], p["points0"], p["f0"], bad, p["obs_uv"], p["cx"], p["cy"],
                                        fixed, iters=3)
    assert status == _lib.GS_BA_BAD_OBS
    assert np.allclose(tr[:, 0], o["trace"][:, 0], rtol=1e-4)
    assert np.abs(X - o["points"]).max() < 2e-3


def test_unobserved_free_keyframe(cuda_device):
    p, fixed = _problem(13, n_points=120, M=3, n_cams=6, n_fixed=2)
    cam = p["obs_cam"].copy()
    cam[cam == 5] = -1
    o, g = _both(p, fixed, 5, obs_cam=cam)
    assert np.abs(g[0][5] - p["poses0"][5]).max() < 1e-6
    _compare_state(o, g, fixed, p, cam=cam)


def test_deterministic_and_graph_capturable(cuda_device):
    p, fixed = _problem(8, n_cams=12, n_points=3000, M=6, n_fixed=3)
    dev = cuda_device
    cam = torch.as_tensor(p["obs_cam"], device=dev)
    uv = torch.as_tensor(p["obs_uv"], device=dev)
    ba = BundleAdjuster(cam, uv, 12, list(fixed), p["cx"], p["cy"])

    def fresh():
        return (torch.as_tensor(p["poses0"], device=dev).clone(), torch.as_tensor(p["points0"], device=dev).clone(),
                torch.tensor([p["f0"]], dtype=torch.float32, device=dev))

    P1, X1, f1 = fresh()
    ba.solve(P1, X1, f1, iters=6)
    t1 = ba.trace[:6].clone()
    P2, X2, f2 = fresh()
    ba.solve(P2, X2, f2, iters=6)
    assert torch.equal(P1, P2) and torch.equal(X1, X2) and torch.equal(f1, f2)
    assert torch.equal(t1, ba.trace[:6])
    # captured in a CUDA graph: same results on replay
    P3, X3, f3 = fresh()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ba.solve(P3, X3, f3, iters=6)  # warm-up outside capture (kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    P3.copy_(fresh()[0]), X3.copy_(fresh()[1]), f3.copy_(fresh()[2])
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ba.solve(P3, X3, f3, iters=6)
    P3.copy_(fresh()[0]), X3.copy_(fresh()[1]), f3.copy_(fresh()[2])
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(P1, P3) and torch.equal(X1, X3) and torch.equal(f1, f3)


def test_empty_problem(cuda_device):
    dev = cuda_device
    cam = torch.zeros((0, 4), dtype=torch.int32, device=dev)
    uv = torch.zeros((0, 4, 2), dtype=torch.float32, device=dev)
    ba = BundleAdjuster(cam, uv, 3, [True, False, False], 640.0, 360.0)
    poses = torch.eye(3, 4, device=dev).reshape(1, 12).repeat(3, 1).contiguous()
    poses[:, 11] = 1.0
    before = poses.clone()
    X = torch.zeros((0, 3), device=dev)
    f = torch.tensor([1000.0], device=dev)
    ba.solve(poses, X, f, iters=3)
    torch.cuda.synchronize()
    assert torch.equal(poses, before) and f.item() == 1000.0
    assert ba.trace[:3, 3].sum().item() == 0.0 and int(ba.status.item()) == 0
