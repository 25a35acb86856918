"""Host-side accounting of the benchmark (no GPU): the roofline object's
arithmetic with the scope table's per-unit work, the choice of the dominant
stage, the binning's byte model, the traffic figure's source check, the timed
poses, and the count of library kernels per training step."""
import hashlib
import json
import os
from types import SimpleNamespace

import pytest

import bench
from paper_2607_14481_b300 import synth


def _workload(n, cams, tiles=3600):
    return SimpleNamespace(n=n, cams=list(cams), steps=[SimpleNamespace(cams=list(cams))],
                           arena=SimpleNamespace(padded=(12 + 48) * n),
                           rast=SimpleNamespace(num_tiles=tiles),
                           pixels_per_iter=sum(c.width * c.height for c in cams))


STAGES = {"project": 0.08, "bin_sort": 0.22, "render_fwd": 0.23, "loss": 0.017, "render_bwd_pixels": 0.54,
          "render_bwd_gaussians": 0.22, "adam": 0.32}
WORK = {"tested": 119e6, "blended": 62.4e6, "walk": 1.25e6, "listed": 1.81e6, "evaluated": 178e6}
PEAKS = {"hbm_gbs": 6445.6, "source": "measured", "sm_max_mhz": 2032.0}


def test_roofline_of_the_plain_step():
    cam = synth.forward_trajectory(3, seed=1008)[0]
    assert (cam.width, cam.height) == (1280, 720)
    wl = _workload(1_000_000, [cam])
    r = bench.roofline(wl, STAGES, WORK, PEAKS, sms=148)
    # the dominant stage is the longest one, bound by FP32 issue: 45 FP32 + 2 MUFU per evaluated pair
    assert r["kernel"] == "render_bwd_pixels" and r["bound"] == "alu" and r["unit"] == "Gop/s"
    assert r["binding_unit"] == "fp32"
    assert r["peak"] == pytest.approx(148 * 128 * 2032e6 / 1e9)
    assert r["algorithmic"] == pytest.approx(45 * 178e6)
    assert r["achieved"] == pytest.approx(45 * 178e6 / 0.54e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # the forward: 12 FP32 + 1 MUFU per evaluated pair, FP32-bound as well
    f = r["per_stage"]["render_fwd"]
    assert f["algorithmic"] == pytest.approx(12 * 178e6) and f["binding_unit"] == "fp32"
    # the SM count is the device's, not a constant
    r2 = bench.roofline(wl, STAGES, WORK, PEAKS, sms=74)
    assert r2["peak"] == pytest.approx(r["peak"] / 2) and r2["frac"] == pytest.approx(2 * r["frac"])
    # HBM stages: algorithmic bytes over the stage time against the measured copy bandwidth
    adam = r["per_stage"]["adam"]
    assert adam["bound"] == "hbm" and adam["algorithmic"] == pytest.approx(28.0 * 60 * 1_000_000)
    assert adam["frac"] == pytest.approx(adam["algorithmic"] / 0.32e-3 / 1e9 / 6445.6)
    # binning: 12 B emit + 4 passes x 24 B + 8 B ranges per pair, 4 B scan per item (3600 tiles: 44 bits)
    bs = r["per_stage"]["bin_sort"]
    assert bs["radix_passes"] == 4
    assert bs["algorithmic"] == pytest.approx(1.81e6 * (12 + 96 + 8) + 4 * 1_000_000)
    assert bs["frac"] == pytest.approx(bs["algorithmic"] / 0.22e-3 / 1e9 / 6445.6)


def test_mufu_binds_when_fp32_work_is_small():
    r = bench.alu_roofline(1e9, 4, 2, 1e-3, 148, 2032.0)
    assert r["binding_unit"] == "mufu"
    assert r["frac"] == pytest.approx(1e9 / 1e-3 / (148 * 16 * 2032e6 / 2))


def test_binning_passes_grow_with_the_tiles():
    assert bench.bin_sort_bytes(1, 0, 3600)[1] == 4          # 32 + 12 bits
    assert bench.bin_sort_bytes(1, 0, 16 * 8160)[1] == 5     # 32 + 17 bits


def test_traffic_needs_a_capture_of_the_current_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"kernel": "render_bwd_pixels", "workload": "w", "bytes_per_launch": 123.0,
             "source": "k.cu", "source_sha256": hashlib.sha256(b"kernel v1").hexdigest()}
    (prof / "dram_traffic.json").write_text(json.dumps({"entries": [entry]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("render_bwd_pixels", "w")[0] == 123.0
    assert bench.load_traffic("render_bwd_pixels", "other")[0] is None
    src.write_text("kernel v2")
    val, why = bench.load_traffic("render_bwd_pixels", "w")
    assert val is None and "changed" in why


def test_dominant_stage_follows_the_times():
    cam = synth.forward_trajectory(3, seed=1008)[0]
    times = dict(STAGES, adam=0.9)
    r = bench.roofline(_workload(1_000_000, [cam]), times, WORK, PEAKS, sms=148)
    assert r["kernel"] == "adam" and r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6445.6


@pytest.mark.parametrize("K", [1, 7, 20, 100, 150, 300])
def test_timed_poses_cover_the_trajectory(K):
    wl = SimpleNamespace(steps=[None] * 100)
    seq = bench.Workload.sequence(wl, K)
    assert len(seq) == K and seq[0] == 0 and all(0 <= k < 100 for k in seq)
    # spread over the whole trajectory: the gaps are even
    if K >= 2:
        assert max(seq) >= 100 - 100 // K - 1
    if K >= 100:
        assert len(set(seq)) == 100


def test_both_arms_report_the_same_config():
    assert bench.workload_config(1_000_000) == bench.workload_config(1_000_000)
    c = bench.workload_config(1_000_000)
    assert c["gaussians"] == 1_000_000 and c["resolution"] == [1280, 720]


def test_library_kernels_per_training_step():
    # projection 1, binning 5, fused composite + loss + per-pixel backward 1,
    # per-Gaussian backward 5 with the parameters' Adam inside, pose Adam and
    # step counter 2; a longest-first order costs no launch; unfused:
    # composite 1, loss 2, per-pixel backward 1 and a separate parameter Adam;
    # beyond 2^13 tiles the tile scan takes 5 launches instead of 1
    assert bench.launches_per_step(1, 3600) == 14
    assert bench.launches_per_step(1, 3600, tile_order=True) == 14
    assert bench.launches_per_step(1, 3600, fused=False) == 18
    assert bench.launches_per_step(1, 3600, fused_adam=False) == 15
    assert bench.launches_per_step(64, 1 << 19) == 18
    assert bench.launches_per_step(16, 80_000) == 18 and bench.launches_per_step(1, 8192) == 14


def test_roofline_of_the_fused_step():
    cam = synth.forward_trajectory(3, seed=1008)[0]
    st = {"project": 0.08, "bin_sort": 0.21, "render_fused": 0.55, "bwd_gaussians_adam": 0.3, "pose_adam": 0.01}
    r = bench.roofline(_workload(1_000_000, [cam]), st, WORK, PEAKS, sms=148)
    # both traversals per evaluated pair: 12 + 45 FP32, 1 + 2 MUFU
    assert r["kernel"] == "render_fused" and r["binding_unit"] == "fp32"
    assert r["algorithmic"] == pytest.approx(57 * 178e6)
    assert r["frac"] == pytest.approx(57 * 178e6 / 0.55e-3 / (148 * 128 * 2032e6))
    assert "loss" not in r["per_stage"] and "render_fwd" not in r["per_stage"]
    # the per-Gaussian backward with Adam inside: 36 B per pair, 24 B per
    # float + 96 B per Gaussian (60 floats)
    ga = r["per_stage"]["bwd_gaussians_adam"]
    assert ga["bound"] == "hbm" and ga["algorithmic"] == pytest.approx(1.81e6 * 36 + 1_000_000 * (24 * 60 + 96))


def test_fused_schedule_names():
    from paper_2607_14481_b300 import _lib, raster
    tile, bits = raster.parse_fused_schedule("8x32_b64_viewmajor")
    assert tile == (8, 32) and bits == _lib.GS_SCHED_FUSED_BATCH(1)
    tile, bits = raster.parse_fused_schedule("16x16_b32_longest")
    assert tile == (16, 16) and bits == _lib.GS_SCHED_FUSED_BATCH(2) | _lib.GS_SCHED_FUSED_LONGEST_FIRST
    assert raster.parse_fused_schedule("32x8_b128_viewmajor") == ((32, 8), 0)
    for bad in ("8x32_b48_viewmajor", "8x16_b64_viewmajor", "8x32_b64", "8x32_64_longest", "8x32_b64_random"):
        with pytest.raises(ValueError):
            raster.parse_fused_schedule(bad)
