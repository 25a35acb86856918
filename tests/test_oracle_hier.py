"""Pins of the progressive-hierarchy oracle (Sec. 6.1 merging and retrieval,
Sec. 6.2 rendering): the screen size in closed form, the 20% trigger on a
worked example, grouping on a worked example and against an independent
brute force (Morton order by a pure-Python bit interleave, float32
distances, greedy dedupe), the parent pull, the merged node's mean in closed
form, the reload, and the cut invariant (every leaf has exactly one active
node on its path to its root) over random sequences of analyses and
reloads."""
import numpy as np
import pytest

import oracle
from paper_2607_14481_b300 import synth

F = 100.0


def _cam(W=200, H=200):
    # at the origin looking down +z (R = I, t = 0)
    return synth.Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), F, F, W / 2, H / 2, W, H)


def _scene(means, log_scale, opa=2.0):
    n = len(means)
    ls = np.full((n, 3), log_scale, np.float64) if np.ndim(log_scale) == 0 else \
        np.repeat(np.asarray(log_scale, np.float64)[:, None], 3, axis=1)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    sh = np.zeros((n, 3, 1))
    return synth.Scene(np.asarray(means, np.float32), ls.astype(np.float32), q.astype(np.float32),
                       np.full(n, opa, np.float32), sh.astype(np.float32))


def _is_cut(st):
    """Every leaf (no children) has exactly one active node on its path to
    its root; no node outside n_nodes is active."""
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
    return not st.active[n:].any()


def test_screen_size_closed_form():
    # S = f * 3 * max scale / z
    sc = _scene([[0.1, -0.2, 5.0]], np.log(0.002))
    st = oracle.HierState(sc, 4)
    out = oracle.hier_analyze(st, _cam())
    s = np.exp(np.float64(sc.log_scales[0, 0]))  # the stored (single-precision) log-scale
    assert abs(out["S"][0] - 3 * F * s / np.float64(sc.means[0, 2])) < 1e-12
    # behind the near plane: infinite, never a candidate
    sc = _scene([[0.0, 0.0, 0.1]], np.log(1e-6))
    out = oracle.hier_analyze(oracle.HierState(sc, 4), _cam())
    assert np.isinf(out["S"][0]) and out["info"]["candidates"] == 0


@pytest.mark.parametrize("k,triggered", [(2, False), (3, True)])
def test_trigger_more_than_20_percent(k, triggered):
    # 10 nodes at depth 5: k of them with S = 3 F 0.001 / 5 = 0.06 px, the
    # rest with S = 3 F 0.05 / 5 = 3 px
    means = [[0.3 * i - 1.5, 0.0, 5.0] for i in range(10)]
    ls = [np.log(0.001) if i < k else np.log(0.05) for i in range(10)]
    st = oracle.HierState(_scene(means, ls), 16)
    out = oracle.hier_analyze(st, _cam())
    assert out["info"]["candidates"] == k and out["info"]["active"] == 10
    assert out["info"]["triggered"] == int(triggered)
    if triggered:
        # the k candidates (no parents) form one group: one new node
        assert out["info"]["groups"] == 1 and st.n_nodes == 11
        assert list(st.parent[:k]) == [10] * k and st.active[10] == 1 and not st.active[:k].any()
        assert sorted(c for c in st.child[10] if c >= 0) == list(range(k))
    else:
        assert st.n_nodes == 10 and st.active[:10].all()
    assert _is_cut(st)


def test_grouping_worked_example_on_a_line():
    # x = 0, 1, 2, 10, 11 (all candidates): the first takes its 3 nearest
    # {1, 2, 10}; the last finds its 3 nearest taken and stays alone
    means = [[x * 0.01, 0.0, 50.0] for x in (0, 1, 2, 10, 11)]
    st = oracle.HierState(_scene(means, np.log(1e-4)), 8)
    out = oracle.hier_analyze(st, _cam())
    assert out["info"]["groups"] == 1 and out["info"]["grouped"] == 4
    assert list(st.parent[:6]) == [5, 5, 5, 5, -1, -1]
    assert list(st.child[5]) == [0, 1, 2, 3]
    assert list(st.active[:6]) == [0, 0, 0, 0, 1, 1]


def _py_morton(m32):
    lo, hi = m32.min(axis=0), m32.max(axis=0)
    out = []
    for p in m32:
        qs = []
        for a in range(3):
            ext = np.float32(hi[a] - lo[a])
            scale = np.float32(1024.0) / ext if ext > 0 else np.float32(0.0)
            t = np.float32(np.float32(p[a] - lo[a]) * scale)
            qs.append(int(min(1023, max(0, np.floor(t)))))
        c = 0
        for bit in range(10):
            for a in range(3):
                c |= ((qs[a] >> bit) & 1) << (3 * bit + a)
        out.append(c)
    return out


def _brute_groups(m32, chunk=64):
    """Independent grouping: Morton order (ties by index), chunks, float32
    squared distances summed x, y, z, 3 nearest (ties by position), greedy."""
    codes = _py_morton(m32)
    order = sorted(range(len(m32)), key=lambda i: (codes[i], i))
    groups = []
    for c0 in range(0, len(order), chunk):
        ids = order[c0:c0 + chunk]
        P = m32[ids]
        knn = []
        for a in range(len(ids)):
            d = []
            for b in range(len(ids)):
                if b == a:
                    continue
                dx, dy, dz = (np.float32(P[b, k] - P[a, k]) for k in range(3))
                s = np.float32(dx * dx)
                s = np.float32(s + np.float32(dy * dy))
                s = np.float32(s + np.float32(dz * dz))
                d.append((float(s), b))
            knn.append([b for _, b in sorted(d)[:3]])
        taken = [False] * len(ids)
        for a in range(len(ids)):
            if taken[a]:
                continue
            g = [a]
            taken[a] = True
            for b in knn[a]:
                if not taken[b]:
                    taken[b] = True
                    g.append(b)
            if len(g) >= 2:
                groups.append([ids[x] for x in g])
            else:
                taken[a] = False
    return groups


@pytest.mark.parametrize("n", [37, 64, 150])
def test_grouping_against_brute_force(n):
    g = np.random.default_rng(n)
    means = np.column_stack([g.uniform(-1, 1, n), g.uniform(-1, 1, n), g.uniform(40, 60, n)]).astype(np.float32)
    st = oracle.HierState(_scene(means, np.log(1e-4)), 2 * n)
    out = oracle.hier_analyze(st, _cam())
    assert out["info"]["triggered"] == 1 and not out["amb"].any()
    want = _brute_groups(means)
    assert out["info"]["groups"] == len(want)
    for gi, grp in enumerate(want):
        node = n + gi
        assert [int(c) for c in st.child[node] if c >= 0] == grp
        assert all(st.parent[c] == node for c in grp)
    # each candidate has at most one parent; groups of 2-4
    assert all(2 <= (st.child[k] >= 0).sum() <= 4 for k in range(n, st.n_nodes))
    assert _is_cut(st)


def test_merged_mean_closed_form():
    # two candidates: the parent's mean is the opacity-weighted mean
    means = [[0.0, 0.0, 50.0], [0.02, 0.0, 50.0]]
    sc = _scene(means, np.log(1e-4))
    sc.opa_logits[:] = [0.5, -1.0]
    st = oracle.HierState(sc, 4)
    oracle.hier_analyze(st, _cam())
    w = 1 / (1 + np.exp(-sc.opa_logits.astype(np.float64)))
    m = sc.means.astype(np.float64)  # the stored (single-precision) means
    want = (w[0] * m[0] + w[1] * m[1]) / w.sum()
    assert np.allclose(st.means[2], want, rtol=1e-12, atol=1e-12)
    assert st.means32[2].dtype == np.float32 and np.allclose(st.means32[2], want, rtol=1e-6)


def _tree(big_parent=True):
    """Leaves 0-3 (children of node 4), node 5 an unrelated active leaf;
    node 4 inactive and its children active."""
    means = [[0.01 * i, 0.0, 50.0] for i in range(4)] + [[0.0, 0.0, 50.0], [0.5, 0.0, 5.0]]
    ls = [np.log(1e-4)] * 4 + [np.log(0.5 if big_parent else 1e-3), np.log(0.05)]
    st = oracle.HierState(_scene(means, ls), 12)
    st.parent[:4] = 4
    st.child[4] = [0, 1, 2, 3]
    st.active[4] = 0
    return st


def test_parent_pull():
    # the four children are candidates (4 of the 5 active nodes): the
    # inactive parent is pulled, no new node
    st = _tree()
    out = oracle.hier_analyze(st, _cam())
    assert out["info"]["triggered"] == 1 and out["info"]["pulled"] == 1 and out["info"]["groups"] == 0
    assert st.n_nodes == 6 and st.active[4] == 1 and not st.active[:4].any() and st.active[5] == 1
    assert _is_cut(st)


def test_no_pull_when_a_child_is_not_a_candidate():
    st = _tree()
    st.log_scales[3] = np.log(0.05)  # child 3 at depth 5: S = 3 F 0.05 / 5 = 3 px, not a candidate
    st.means[3, 2] = 5.0
    st.means32[3, 2] = 5.0
    out = oracle.hier_analyze(st, _cam())
    assert out["info"]["candidates"] == 3 and out["info"]["triggered"] == 1
    # children with a parent are not regrouped: nothing changes
    assert out["info"]["pulled"] == 0 and out["info"]["groups"] == 0
    assert st.n_nodes == 6 and st.active[4] == 0 and st.active[:4].all()


def test_reload_replaces_a_large_node_by_its_children():
    st = _tree()
    st.active[:4] = 0
    st.active[4] = 1
    # node 4 at depth 50 with scale 0.5: S = 3 F 0.5 / 50 = 3 px > 1, in view
    k, amb = oracle.hier_refine(st, _cam())
    assert k == 1 and st.active[:4].all() and st.active[4] == 0 and not amb.any()
    assert oracle.hier_refine(st, _cam())[0] == 0  # a fixpoint
    # behind the camera: not in view, not reloaded
    st2 = _tree()
    st2.active[:4] = 0
    st2.active[4] = 1
    back = synth.Camera(np.diag([-1.0, 1.0, -1.0]).astype(np.float32), np.zeros(3, np.float32), F, F, 100, 100,
                        200, 200)
    assert oracle.hier_refine(st2, back)[0] == 0 and st2.active[4] == 1
    # the view cut refines a copy and leaves the state alone
    cut = oracle.hier_view_cut(st2, _cam())
    assert list(cut[:6]) == [1, 1, 1, 1, 0, 1] and st2.active[4] == 1


def test_active_set_stays_a_cut_over_random_analyses_and_reloads():
    g = np.random.default_rng(7)
    n = 600
    means = np.column_stack([g.uniform(-2, 2, n), g.uniform(-1, 1, n), g.uniform(4, 30, n)])
    sc = _scene(means, g.normal(-5.5, 0.6, n))
    st = oracle.HierState(sc, 4 * n)
    for step in range(12):
        eye = np.array([g.uniform(-1, 1), g.uniform(-0.5, 0.5), g.uniform(-15, 2)])
        cam = synth.look_at(eye, (0, 0, 15), F, F, 100, 100, 200, 200)
        if step % 3 == 2:
            oracle.hier_refine(st, cam, tau_h=1.0)
        else:
            oracle.hier_analyze(st, cam)
        assert _is_cut(st), step
    assert st.n_nodes > n  # merges happened
    depth = np.zeros(st.n_nodes, int)
    for i in range(st.n_nodes):
        c = i
        while st.parent[c] >= 0:
            c = st.parent[c]
            depth[i] += 1
    assert depth.max() >= 1


def test_render_cut_worked_example():
    # node 4 (parent of leaves 0-3) at depth 50 with scale 0.5: S = 3 F 0.5 /
    # 50 = 3 px > 1, so the descent goes on to its children; node 5 is a
    # root leaf.  With scale 1e-3 (S = 0.006 px) the parent itself is drawn.
    sel, amb = oracle.hier_render_cut(_tree(big_parent=True), _cam())
    assert list(sel) == [1, 1, 1, 1, 0, 1] and not amb.any()
    sel, _ = oracle.hier_render_cut(_tree(big_parent=False), _cam())
    assert list(sel) == [0, 0, 0, 0, 1, 1]
    # the active set does not matter
    st = _tree(big_parent=False)
    st.active[:] = 0
    st.active[:4] = 1
    assert list(oracle.hier_render_cut(st, _cam())[0]) == [0, 0, 0, 0, 1, 1]
    # behind the camera S is infinite: the descent reaches every leaf
    back = synth.Camera(np.diag([-1.0, 1.0, -1.0]).astype(np.float32), np.zeros(3, np.float32), F, F, 100, 100,
                        200, 200)
    assert list(oracle.hier_render_cut(_tree(big_parent=False), back)[0]) == [1, 1, 1, 1, 0, 1]


def _brute_render_cut(st, cam, znear=0.2, tau=1.0):
    """Recursive descent from the roots with the screen size written out
    independently: t_z = R[2] . m + t[2], S = f_x 3 max exp(log-scale) / t_z,
    +inf at or behind the near plane."""
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    n = st.n_nodes
    S = np.empty(n)
    for i in range(n):
        tz = float(R[2] @ st.means[i] + t[2])
        S[i] = np.inf if tz <= znear else float(cam.fx) * 3.0 * np.exp(st.log_scales[i].max()) / tz
    sel = np.zeros(n, np.uint8)

    def visit(k):
        kids = [int(c) for c in st.child[k] if c >= 0]
        if kids and S[k] > tau:
            for c in kids:
                visit(c)
        else:
            sel[k] = 1

    for r in range(n):
        if st.parent[r] < 0:
            visit(r)
    return sel


def test_render_cut_against_brute_force_descent():
    g = np.random.default_rng(17)
    n = 500
    means = np.column_stack([g.uniform(-2, 2, n), g.uniform(-1, 1, n), g.uniform(4, 30, n)])
    st = oracle.HierState(_scene(means, g.normal(-5.5, 0.6, n)), 4 * n)
    cams = [synth.look_at((g.uniform(-1, 1), g.uniform(-0.5, 0.5), g.uniform(-15, 2)), (0, 0, 15), F, F, 100, 100,
                          200, 200) for _ in range(8)]
    for c in cams[:6]:
        oracle.hier_analyze(st, c)
    assert st.n_nodes > n
    coarser = 0
    for c in cams:
        for tau in (0.5, 1.0, 4.0):
            sel, amb = oracle.hier_render_cut(st, c, tau=tau)
            want = _brute_render_cut(st, c, tau=tau)
            ok = amb == 0
            assert np.array_equal(sel[ok], want[ok])
            # a cut: every leaf has exactly one selected node on its path
            for i in range(st.n_nodes):
                if st.child[i, 0] >= 0:
                    continue
                k, p = 0, i
                while p >= 0:
                    k += int(sel[p])
                    p = st.parent[p]
                assert k == 1
            coarser += int(sel[n:st.n_nodes].sum())
    assert coarser > 0  # merged nodes are drawn somewhere
