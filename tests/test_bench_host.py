"""Host-side accounting of the benchmark (no GPU): the roofline object's
arithmetic, the choice of the dominant stage, the traffic figure's workload
key, and the count of library kernels per training step."""
from types import SimpleNamespace

import pytest

import bench
from paper_2607_14481_b300 import synth


def _workload(n, cams):
    return SimpleNamespace(n=n, cams=list(cams), steps=[SimpleNamespace(cams=list(cams))],
                           arena=SimpleNamespace(padded=(12 + 48) * n),
                           pixels_per_iter=sum(c.width * c.height for c in cams))


STAGES = {"project": 0.08, "bin_sort": 0.22, "render_fwd": 0.23, "loss": 0.017, "render_bwd_pixels": 0.54,
          "render_bwd_gaussians": 0.22, "adam": 0.32}
WORK = {"tested": 119e6, "blended": 62.4e6, "walk": 1.25e6, "listed": 1.81e6}
PEAKS = {"hbm_gbs": 6445.6, "source": "measured", "sm_max_mhz": 2032.0}


def test_roofline_of_the_plain_step():
    cam = synth.forward_trajectory(3, seed=1008)[0]
    assert (cam.width, cam.height) == (1280, 720)
    wl = _workload(1_000_000, [cam])
    r = bench.roofline(wl, STAGES, WORK, PEAKS)
    # the dominant stage is the longest one, bound by FP32 issue
    assert r["kernel"] == "render_bwd_pixels" and r["bound"] == "alu" and r["unit"] == "Gop/s"
    assert r["peak"] == pytest.approx(148 * 128 * 2032e6 / 1e9)
    ops = bench.OPS_TEST * WORK["tested"] + bench.OPS_BWD_BLEND * WORK["blended"]
    assert r["algorithmic"] == pytest.approx(ops)
    assert r["achieved"] == pytest.approx(ops / 0.54e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # its DRAM traffic comes from the capture of this very workload
    assert r["traffic"] == bench.MEASURED_TRAFFIC[("render_bwd_pixels", 1_000_000, (1280, 720), 1)]["bytes"]
    # HBM stages: algorithmic bytes over the stage time against the measured copy bandwidth
    adam = r["per_stage"]["adam"]
    assert adam["bound"] == "hbm" and adam["algorithmic"] == pytest.approx(28.0 * 60 * 1_000_000)
    assert adam["frac"] == pytest.approx(adam["algorithmic"] / 0.32e-3 / 1e9 / 6445.6)
    # the binning stage has no byte bound of its own and is not in the table
    assert "bin_sort" not in r["per_stage"]


def test_traffic_is_null_for_a_workload_that_was_not_captured():
    cams = [synth.with_resolution(c, 1280, 720) for c in synth.loop_views(16, 1009)]
    r = bench.roofline(_workload(1_000_000, cams), STAGES, WORK, PEAKS)
    assert r["kernel"] == "render_bwd_pixels" and r["traffic"] is None and r["traffic_source"] is None


def test_dominant_stage_follows_the_times():
    cam = synth.forward_trajectory(3, seed=1008)[0]
    times = dict(STAGES, adam=0.9)
    r = bench.roofline(_workload(1_000_000, [cam]), times, WORK, PEAKS)
    assert r["kernel"] == "adam" and r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6445.6
    assert r["traffic"] is None


def test_library_kernels_per_training_step():
    # projection 1, binning 11, composite 1, loss 2, per-pixel backward 1,
    # per-Gaussian backward 5, Adam 3; a longest-first schedule adds 2
    assert bench.launches_per_step(1, 3600) == 24
    assert bench.launches_per_step(1, 3600, tile_order=True) == 26
