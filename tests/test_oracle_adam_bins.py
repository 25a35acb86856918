"""Pins of the oracle's optimiser step and binning.

  * Adam: the special case of a library routine, torch.optim.Adam in float64
    on the CPU, with per-group learning rates, over several steps;
  * pose step: Adam on the twist followed by T <- Exp(xi) T, with Exp checked
    against scipy's matrix exponential of the 4x4 twist;
  * binning: brute force on tiny inputs (every (tile, Gaussian) pair listed
    and ordered by Python's stable sort on (tile, depth bits)), including forced
    depth ties that must stay in Gaussian-id order.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from paper_2607_14481_b300 import synth


def test_adam_matches_torch_float64():
    g = np.random.default_rng(0)
    n1, n2 = 37, 53
    p = g.normal(size=n1 + n2)
    lr = np.concatenate([np.full(n1, 1e-2), np.full(n2, 3e-3)])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    t1 = torch.tensor(p[:n1].copy(), dtype=torch.float64, requires_grad=True)
    t2 = torch.tensor(p[n1:].copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([{"params": [t1], "lr": 1e-2}, {"params": [t2], "lr": 3e-3}],
                           betas=(0.9, 0.999), eps=1e-15, foreach=False)
    for step in range(1, 6):
        grad = g.normal(size=n1 + n2) * (10.0 ** g.uniform(-3, 1))
        oracle.adam(p, grad, m, v, lr, step)
        t1.grad = torch.tensor(grad[:n1])
        t2.grad = torch.tensor(grad[n1:])
        opt.step()
        ref = np.concatenate([t1.detach().numpy(), t2.detach().numpy()])
        assert np.abs(p - ref).max() < 1e-12


def _twist(xi):
    v, w = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


@pytest.mark.parametrize("scale", [1e-7, 1e-3, 0.3, 2.0])
def test_se3_exp_matches_expm(scale):
    g = np.random.default_rng(1)
    for _ in range(5):
        xi = g.normal(size=6) * scale
        R, t = oracle.se3_exp(xi)
        E = scipy.linalg.expm(_twist(xi))
        assert np.abs(R - E[:3, :3]).max() < 1e-13
        assert np.abs(t - E[:3, 3]).max() < 1e-13


def test_pose_adam_is_adam_then_exp():
    g = np.random.default_rng(2)
    V = 3
    poses = np.stack([synth.look_at(g.normal(size=3) * 2, (0, 0, 0), 1, 1, 0, 0, 1, 1).pose12()
                      for _ in range(V)]).astype(np.float64)
    ref = poses.reshape(V, 3, 4).copy()
    m = np.zeros((V, 6))
    v = np.zeros((V, 6))
    x = torch.zeros((V, 6), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([x], lr=1e-3, betas=(0.9, 0.999), eps=1e-15, foreach=False)
    for step in range(1, 4):
        gp = g.normal(size=(V, 6))
        oracle.pose_adam(poses, gp, m, v, 1e-3, step)
        before = x.detach().numpy().copy()
        x.grad = torch.tensor(gp)
        opt.step()
        xi = x.detach().numpy() - before
        for k in range(V):
            T = np.eye(4)
            T[:3] = ref[k]
            T = scipy.linalg.expm(_twist(xi[k])) @ T
            ref[k] = T[:3]
        assert np.abs(poses.reshape(V, 3, 4) - ref).max() < 1e-12


def _brute_bins(depth, rect, tiles):
    entries = []
    base = 0
    bases = []
    for tx, ty in tiles:
        bases.append(base)
        base += tx * ty
    bits = depth.view(np.uint32)
    for v, (tx, ty) in enumerate(tiles):
        for i in range(depth.shape[1]):
            x0, y0, x1, y1 = rect[v, i]
            for yy in range(y0, y1 + 1):
                for xx in range(x0, x1 + 1):
                    gt = bases[v] + yy * tx + xx
                    entries.append(((gt << 32) | int(bits[v, i]), i))
    entries = sorted(entries, key=lambda e: e[0])  # stable: id order kept on ties
    return entries, base


@pytest.mark.parametrize("ties", [0, 3])
def test_bins_brute_force(ties):
    tiles = [(5, 3), (2, 4)]
    depth, rect = synth.random_records(tiles, 40, seed=10 + ties, tie_levels=ties)
    keys, vals, ranges = oracle.bin_records(depth, rect, tiles)
    entries, G = _brute_bins(depth, rect, tiles)
    assert len(entries) == len(keys)
    assert [e[0] for e in entries] == [int(k) for k in keys]
    assert [e[1] for e in entries] == [int(x) for x in vals]
    for g in range(G):
        idx = [k for k, e in enumerate(entries) if (e[0] >> 32) == g]
        if idx:
            assert (ranges[g, 0], ranges[g, 1]) == (idx[0], idx[-1] + 1)
        else:
            assert ranges[g, 0] == ranges[g, 1]
    if ties:
        # equal keys must appear in increasing Gaussian id
        for a, b in zip(entries, entries[1:]):
            if a[0] == b[0]:
                assert a[1] < b[1]
