"""Pins of the keyframe-selection oracle (Sec. 6.2): a worked example and the
properties the rule fixes."""
import numpy as np

import oracle


def test_worked_example():
    # counts 100, 4, 6, 0, 50: threshold 5 -> keyframe 1 (4 < 5) and 3 go;
    # with min_keep = 2 only the top two stay (100, 50)
    kf = np.repeat(np.arange(5), [100, 4, 6, 0, 50])
    c, p, kept = oracle.keyframe_weights(kf, 5, min_keep=0)
    assert list(c) == [100, 4, 6, 0, 50]
    assert list(kept) == [True, False, True, False, True]
    assert np.allclose(p, [100 / 156, 0, 6 / 156, 0, 50 / 156])
    _, p2, kept2 = oracle.keyframe_weights(kf, 5, min_keep=4)
    assert list(kept2) == [True, True, True, False, True]  # the four largest stay
    assert np.allclose(p2, np.array([100, 4, 6, 0, 50]) / 160)


def test_properties():
    g = np.random.default_rng(1)
    for _ in range(20):
        K = int(g.integers(1, 300))
        kf = g.integers(-1, K + 3, int(g.integers(0, 20000)))
        c, p, kept = oracle.keyframe_weights(kf, K)
        assert c.sum() == ((kf >= 0) & (kf < K)).sum()
        assert kept.sum() >= min(50, K)
        if c.sum() > 0:
            assert abs(p.sum() - 1) < 1e-12
        assert np.all(p[~kept] == 0)
        assert np.all(p[kept] * c[kept].sum() >= 0)
        big = c >= 0.05 * c.max()
        assert np.all(kept[big])
