"""gs_bin_sort_noalloc (static-scratch binning) against gs_bin_sort with a
caller workspace: keys, tile ranges, order, counts and pair offsets
bit-identical (integer work), on two calls in a row, and the image composited
from its lists identical; a problem larger than the scratch is rejected."""
import numpy as np
import pytest
import torch

from paper_2607_14481_b300 import _lib, raster, synth
from gpu_util import ensure_built

pytestmark = pytest.mark.gpu

SENTINEL = -7  # written into every output before each call, so unwritten words compare too


def _outputs(r):
    return {"vals": r.vals.clone(), "ranges": r.ranges.clone(), "counts": r.counts.clone(),
            "pair_off": r.pair_off.clone(), "keys": r.keys.clone()}


def _poison(r):
    for t in (r.vals, r.ranges, r.counts, r.pair_off, r.keys):
        t.fill_(SENTINEL)


@pytest.mark.parametrize("case", ["plain_small", "diffcheck_three_views"])
def test_noalloc_sort_equals_workspace_sort_twice(cuda_device, case):
    ensure_built()
    dev = torch.device("cuda:0")
    if case == "plain_small":
        sc, cams, _ = synth.plain_small()
    else:
        sc, cams, _ = synth.diffcheck()
    arena = raster.Arena.from_scene(sc, dev)
    poses = raster.poses_tensor(cams, dev)
    r = raster.Rasterizer(sc.n, sc.sh_degree, cams, capacity=65536, device=dev, keep_keys=True)
    assert r.L.gs_bin_sort_workspace(sc.n, len(cams), 65536) <= _lib.noalloc_scratch_bytes()
    r.project(arena, poses)

    _poison(r)
    r.bin_sort()
    ref = _outputs(r)
    img_ref = r.new_image()
    r.render_fwd(img_ref, None)
    torch.cuda.synchronize()
    assert int(ref["counts"][2]) == 0 and int(ref["counts"][1]) > 0

    for _ in range(2):
        _poison(r)
        r.bin_sort_noalloc()
        got = _outputs(r)
        img = r.new_image()
        r.render_fwd(img, None)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(got[k], ref[k]), k
        assert torch.equal(img, img_ref)


def test_noalloc_sort_rejects_oversize(cuda_device):
    ensure_built()
    dev = torch.device("cuda:0")
    sc = synth.random_scene(70000, 3, 0, (-1, -1, -1), (1, 1, 1), -3.5, 0.4)
    cams = synth.plain_small()[1]
    r = raster.Rasterizer(sc.n, sc.sh_degree, cams, capacity=1_000_000, device=dev)
    need = r.L.gs_bin_sort_workspace(sc.n, 1, 1_000_000)
    assert need > _lib.noalloc_scratch_bytes()
    arena = raster.Arena.from_scene(sc, dev)
    r.project(arena, raster.poses_tensor(cams, dev))
    with pytest.raises(_lib.GsError) as ei:
        r.bin_sort_noalloc()
    assert ei.value.status == _lib.GS_ERR_OOM
    assert "static scratch" in str(ei.value)
    # the rejected call launched nothing; the workspace path still works
    r.bin_sort()
    torch.cuda.synchronize()
    assert int(r.read_counts()[2]) == 0
