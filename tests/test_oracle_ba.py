"""Pins of the local bundle adjustment oracle (Sec. 5.1): the Jacobian against
central finite differences through the update, the Schur-complement step
against a direct solve of the full damped normal equations, convergence to
the ground truth on noise-free observations, the chi-square law of the
optimal cost under Gaussian pixel noise, and the gauge/edge cases (fixed
keyframes, empty slots, an unobserved free keyframe)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import ba
from paper_2607_14481_b300 import synth


def _small(seed=3, noise=0.5, n_points=40, n_cams=6, M=4, n_fixed=2):
    p = synth.ba_problem(seed, n_cams=n_cams, n_points=n_points, obs_per_point=M, n_fixed=n_fixed, noise_px=noise)
    fixed = np.zeros(n_cams, bool)
    fixed[:n_fixed] = True
    return p, fixed


def _state(p):
    R, t = ba.split_poses(p["poses0"])
    return R, t, p["points0"].astype(np.float64), float(p["f0"])


def _fd_discrepancy(p, fixed, jac=ba.jacobian, h=1e-6):
    R, t, X, f = _state(p)
    obs_cam, uv = p["obs_cam"], p["obs_uv"]
    J = jac(R, t, X, f, obs_cam, fixed, True).toarray()
    cam_col, f_col, ncc, ncol = ba.layout(R.shape[0], fixed, True, X.shape[0])
    worst = 0.0
    for j in range(ncol):
        d = np.zeros(ncol)
        d[j] = h
        rp, _ = ba.residuals(*ba.retract(R, t, X, f, d, cam_col, f_col, ncc), obs_cam, uv, p["cx"], p["cy"])
        rm, _ = ba.residuals(*ba.retract(R, t, X, f, -d, cam_col, f_col, ncc), obs_cam, uv, p["cx"], p["cy"])
        fd = (rp - rm).reshape(-1) / (2 * h)
        scale = max(1.0, np.abs(J[:, j]).max())
        worst = max(worst, np.abs(fd - J[:, j]).max() / scale)
    return worst


def test_rodrigues_is_the_matrix_exponential():
    g = np.random.default_rng(0)
    for w in [g.normal(size=3), 1e-9 * g.normal(size=3), np.array([np.pi / 2, 0, 0]), np.zeros(3)]:
        K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        assert np.allclose(ba.rodrigues(w), sla.expm(K), atol=1e-14)


def test_jacobian_matches_central_differences():
    p, fixed = _small()
    assert _fd_discrepancy(p, fixed) < 1e-5


def test_planted_rotation_sign_error_is_caught():
    """A plausible mistake (the rotation block with the wrong sign) must fail
    the finite-difference pin."""
    p, fixed = _small()

    def wrong(R, t, X, f, obs_cam, fixed, opt_focal):
        J = ba.jacobian(R, t, X, f, obs_cam, fixed, opt_focal).tolil()
        cam_col, _, _, _ = ba.layout(R.shape[0], fixed, opt_focal, X.shape[0])
        for c in cam_col[cam_col >= 0]:
            J[:, c:c + 3] = -J[:, c:c + 3]
        return J.tocsr()

    assert _fd_discrepancy(p, fixed, jac=wrong) > 1e-2


@pytest.mark.parametrize("lam", [1e-3, 10.0])
def test_schur_step_equals_full_damped_solve(lam):
    p, fixed = _small(n_points=60)
    R, t, X, f = _state(p)
    r, _ = ba.residuals(R, t, X, f, p["obs_cam"], p["obs_uv"], p["cx"], p["cy"])
    J = ba.jacobian(R, t, X, f, p["obs_cam"], fixed, True)
    Hd, g = ba.damped_system(J, r, lam)
    _, _, ncc, _ = ba.layout(R.shape[0], fixed, True, X.shape[0])
    delta, S, b = ba.schur_step(Hd, g, ncc, X.shape[0])
    full = spla.spsolve(Hd.tocsc(), -g)
    assert np.abs(delta - full).max() <= 1e-8 * np.abs(full).max()
    # damping: Marquardt's scaled diagonal
    H = (J.T @ J).tocsr()
    assert np.allclose(Hd.diagonal(), H.diagonal() * (1 + lam), rtol=1e-15)


def test_noise_free_converges_to_ground_truth():
    p, fixed = _small(seed=5, noise=0.0, n_points=200, n_cams=8, M=5, n_fixed=3)
    out = ba.solve(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"], p["cy"], fixed, iters=15)
    assert out["trace"][0, 0] > 1e3
    # the observations are stored in float32: the optimum keeps their rounding
    # error, E ~ sum ulp^2 / 12, and moves the parameters by about that much
    q = np.spacing(np.abs(p["obs_uv"])).astype(np.float64)
    assert out["cost"] < 2.0 * np.sum(q * q / 12.0)
    assert np.abs(out["poses"] - p["poses_true"]).max() < 1e-5
    assert np.abs(out["points"] - p["points_true"]).max() < 1e-4
    assert abs(out["f"] - p["f_true"]) < 1e-6 * p["f_true"]


def test_optimal_cost_follows_chi_square():
    """Under i.i.d. N(0, s^2) pixel noise the least-squares optimum has
    E[cost] = s^2 (m - n) (m residuals, n parameters), std s^2 sqrt(2(m - n))."""
    s = 0.5
    p, fixed = _small(seed=7, noise=s, n_points=1500, n_cams=10, M=6, n_fixed=3)
    out = ba.solve(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"], p["cy"], fixed, iters=10)
    m = 2 * p["obs_cam"].size
    n = 6 * (10 - 3) + 1 + 3 * 1500
    ratio = out["cost"] / (s * s * (m - n))
    assert abs(ratio - 1.0) < 5.0 * np.sqrt(2.0 / (m - n))


def test_fixed_keyframes_and_lm_bookkeeping():
    p, fixed = _small(seed=9, n_points=300, n_cams=8, M=5, n_fixed=3)
    out = ba.solve(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"], p["cy"], fixed,
                   iters=8, lambda0=1e-2)
    assert np.array_equal(out["poses"][fixed], p["poses0"][fixed].astype(np.float64))
    tr = out["trace"]
    lam = 1e-2
    cur = tr[0, 0]
    for E, Ec, l, acc in tr:
        assert l == pytest.approx(lam, rel=1e-12) and E == cur
        assert bool(acc) == (Ec < E)
        if acc:
            cur, lam = Ec, lam * 0.1
        else:
            lam = lam * 10
    assert out["cost"] == pytest.approx(cur, rel=1e-12)


def test_empty_slots_equal_a_narrower_problem():
    p, fixed = _small(seed=11, n_points=80, n_cams=6, M=5)
    cam = p["obs_cam"].copy()
    cam[:, 3:] = -1
    a = ba.solve(p["poses0"], p["points0"], p["f0"], cam, p["obs_uv"], p["cx"], p["cy"], fixed, iters=4)
    b = ba.solve(p["poses0"], p["points0"], p["f0"], p["obs_cam"][:, :3], p["obs_uv"][:, :3], p["cx"], p["cy"],
                 fixed, iters=4)
    assert np.allclose(a["trace"], b["trace"], rtol=1e-10)
    assert np.allclose(a["points"], b["points"], atol=1e-9)


def test_unobserved_free_keyframe_stays():
    p, fixed = _small(seed=13, n_points=80, n_cams=6, M=3)
    cam = p["obs_cam"].copy()
    cam[cam == 5] = -1
    out = ba.solve(p["poses0"], p["points0"], p["f0"], cam, p["obs_uv"], p["cx"], p["cy"], fixed, iters=5)
    assert np.all(np.isfinite(out["poses"]))
    assert np.array_equal(out["poses"][5], p["poses0"][5].astype(np.float64)) or \
        np.abs(out["poses"][5] - p["poses0"][5]).max() < 1e-12
    assert out["cost"] < out["trace"][0, 0]
