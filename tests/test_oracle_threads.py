"""The oracle's parallel loops (OpenMP over Gaussians and tiles, gradient
sums per tile then in tile order, pose terms in Gaussian order) give the same
bits at any thread count: the CPU baseline may use every host core without
changing a result."""
import numpy as np
import pytest

import oracle
from paper_2607_14481_b300 import synth


def _run(threads, sc, cams, dimg):
    assert oracle.set_threads(threads) == threads
    out = oracle.render(sc, cams, want_proj=True)
    g = oracle.backward(sc, cams, dimg)
    return out, g


@pytest.mark.parametrize("case", ["plain_small", "diffcheck"])
def test_results_independent_of_thread_count(case):
    if case == "plain_small":
        sc, cams, _ = synth.plain_small()
    else:
        sc, cams, _ = synth.diffcheck()
    g = np.random.default_rng(3)
    dimg = [g.normal(size=(3, c.height, c.width)) for c in cams]
    before = oracle.get_threads()
    try:
        r1, g1 = _run(1, sc, cams, dimg)
        r4, g4 = _run(4, sc, cams, dimg)
    finally:
        oracle.set_threads(before)
    for k in ("image", "alpha", "flags"):
        for a, b in zip(r1[k], r4[k]):
            assert np.array_equal(a, b), k
    assert np.array_equal(r1["proj"], r4["proj"])
    for k in g1:
        assert np.array_equal(g1[k], g4[k]), k
    # the gradients are not trivially zero
    assert np.abs(g1["means"]).max() > 0 and np.abs(g1["pose"]).max() > 0


def test_adam_independent_of_thread_count():
    g = np.random.default_rng(5)
    n = 100_003
    p0, gr = g.normal(size=n), g.normal(size=n)
    lr = np.full(n, 1e-2)
    outs = []
    before = oracle.get_threads()
    try:
        for th in (1, 3):
            oracle.set_threads(th)
            p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
            oracle.adam(p, gr, m, v, lr, 1)
            outs.append((p, m, v))
    finally:
        oracle.set_threads(before)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
