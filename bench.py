#!/usr/bin/env python
"""Benchmark of the rasterizer's training step: forward (projection, tile
binning and sort, blending), loss gradient, backward to all parameters and the
camera pose, and the fused Adam step, at 1M Gaussians.

Workload (synthetic, shaped like the paper's captures): 1,000,000 Gaussians in
a 20 x 5 x 20 m box, SH degree 3, log-scales N(-4, 0.5^2); a 100-pose
forward-moving trajectory at 1280x720, f = 1000; targets are renders of a
seeded perturbed copy of the scene; L1 loss.  One iteration = one view =
one Adam step (plain single-view mode).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+Adam iters/s at 1M Gaussians (plain single-view 1280x720 SH3)"
N_GAUSS = 1_000_000
N_POSES = 100
SEED_SCENE, SEED_TRAJ, SEED_TARGET = 1007, 1008, 1009


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# multi-process (independent replicas; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup(gpus):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Workload:
    def __init__(self, n, device, rank=0):
        import torch
        from paper_2607_14481_b300 import raster, synth
        self.torch = torch
        self.raster = raster
        self.n = n
        self.device = device
        self.scene = synth.box_scene(n, SEED_SCENE + 100 * rank)
        self.cams = synth.forward_trajectory(N_POSES, SEED_TRAJ)
        self.arena = raster.Arena.from_scene(self.scene, device)
        self.grads = self.arena.like()
        self.m = self.arena.like()
        self.v = self.arena.like()
        self.groups = self.arena.adam_groups(lr_means=1.6e-4 * 10.0)
        self.poses = raster.poses_tensor(self.cams, device)
        self.pose_m = torch.zeros((N_POSES, 6), dtype=torch.float32, device=device)
        self.pose_v = torch.zeros((N_POSES, 6), dtype=torch.float32, device=device)
        self.dpose = torch.zeros((N_POSES, 6), dtype=torch.float32, device=device)
        self.pose_uses = [0] * N_POSES
        self.rast = raster.Rasterizer(n, 3, self.cams[:1], device=device)
        self.loss = raster.ImageLoss(device)
        self.img = self.rast.new_image()
        self.dimg = self.rast.new_image()
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.pixels = self.cams[0].width * self.cams[0].height
        self._make_targets(synth)
        self.step_no = 0

    def _make_targets(self, synth):
        torch = self.torch
        pert = self.raster.Arena.from_scene(synth.perturbed(self.scene, SEED_TARGET), self.device)
        self.targets = torch.empty((N_POSES, 3 * self.pixels), dtype=torch.float32, device=self.device)
        kmax = 0
        for k, c in enumerate(self.cams):
            self.rast.set_cameras([c])
            self.rast.forward(pert, self.poses[k:k + 1], self.targets[k], None, check=True)
            kmax = max(kmax, int(self.rast.read_counts()[1]))
        for k, c in enumerate(self.cams):  # the trained scene's own pair counts
            self.rast.set_cameras([c])
            self.rast.forward(self.arena, self.poses[k:k + 1], self.img, None, check=True)
            kmax = max(kmax, int(self.rast.read_counts()[1]))
        # fixed capacity for the timed loop: no host synchronisation inside it
        self.rast.set_capacity(int(kmax * 1.3) + 4096)
        self.kmax = kmax
        self.targets_host = self.targets.cpu().pin_memory()
        self.target_dev = torch.empty_like(self.targets[0])

    def step(self, target, ev=None):
        """One training iteration on the next pose.  ev: optional list of 7
        CUDA events recorded at the stage boundaries."""
        k = self.step_no % N_POSES
        self.step_no += 1
        r = self.rast
        r.set_cameras([self.cams[k]])
        pose = self.poses[k:k + 1]
        rec = (lambda i: ev[i].record()) if ev is not None else (lambda i: None)
        rec(0)
        r.project(self.arena, pose)
        rec(1)
        r.bin_sort()
        rec(2)
        r.render_fwd(self.img, None)
        rec(3)
        self.loss(self.img, target, self.dimg, kind=0)
        rec(4)
        r.backward_pixels(self.dimg, None)
        rec(5)
        r.backward_gaussians(self.arena, pose, self.grads, self.dpose[k:k + 1])
        rec(6)
        self.pose_uses[k] += 1
        self.raster.adam_step(self.arena, self.grads, self.m, self.v, self.step_no, self.groups,
                              status=self.status, pose=pose, dpose=self.dpose[k:k + 1],
                              pose_m=self.pose_m[k:k + 1], pose_v=self.pose_v[k:k + 1], pose_lr=1e-4,
                              pose_step=self.pose_uses[k])
        rec(7)

    def check_device_status(self):
        cnt = self.rast.read_counts()
        assert cnt[2] == 0, f"binning status {cnt[2]} in the timed loop (1 = capacity, 2 = index)"
        return int(self.status.item())


STAGES = ("project", "bin_sort", "render_fwd", "loss", "render_bwd_pixels", "render_bwd_gaussians", "adam")


def run_ours(args, ws, rank, local):
    import torch
    from paper_2607_14481_b300 import build
    if rank == 0:
        build.build()
    barrier(ws)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    wl = Workload(args.n, device, rank)
    torch.cuda.synchronize()
    # warm-up
    for _ in range(max(3, args.warmup)):
        wl.step(wl.targets[wl.step_no % N_POSES])
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs, stage events on the launching stream
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    t0.record()
    for i in range(K):
        wl.step(wl.targets[wl.step_no % N_POSES], evs[i])
    t1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    elapsed_max = allreduce_max(elapsed, ws)
    stage_ms = {s: float(np.mean([evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(K)]))
                for j, s in enumerate(STAGES)}
    bad = wl.check_device_status()
    value = ws * K / elapsed_max

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        loss_host = torch.zeros(K, dtype=torch.float32).pin_memory()
        barrier(ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(K):
            k = wl.step_no % N_POSES
            wl.target_dev.copy_(wl.targets_host[k], non_blocking=True)
            wl.step(wl.target_dev)
            loss_host[i:i + 1].copy_(wl.loss.loss, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        barrier(ws)
        e_el = allreduce_max(e0.elapsed_time(e1) / 1e3, ws)
        e2e = {"value": ws * K / e_el, "unit": "iters/s",
               "h2d_bytes_per_step": int(wl.target_dev.numel() * 4),
               "d2h_bytes_per_step": 4,
               "ms_per_step": 1e3 * e_el / K}
        wl.check_device_status()

    # ---- roofline of the dominant stage
    peaks = load_peaks()
    roof = roofline(wl, stage_ms, peaks)
    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"plain single-view training, {args.n} Gaussians SH3, 1280x720, "
                               f"100-pose forward trajectory, L1 loss",
                   "gaussians": args.n, "views_per_iter": 1, "resolution": [1280, 720],
                   "parallelism": f"replicas{ws}", "l2": "inputs larger than L2 (parameter arena "
                   f"{wl.arena.padded * 4 / 1e6:.0f} MB x4)",
                   "pairs_max": wl.kmax, "capacity": wl.rast.capacity},
        "mpix_per_s": value * wl.pixels / 1e6,
        "stage_ms": stage_ms,
        "e2e": e2e,
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": launches_per_step() * K,
        "nonfinite_flag": bad,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.n, budget_s=20.0)
    return out, rank


def launches_per_step():
    # project 1; bin_sort: init 1 + flags 1 + scan 3 + compact 1 + 4 x (hist 1 + scan 3 + scatter 1) +
    # pair counts 1 + scan 3 + status 1 + emit 1 + 2 x 5 + ranges 1 (+ memset); fwd 1; loss 2;
    # bwd pixels 1; bwd gaussians 2; adam 2
    bin_sort = 1 + 1 + 3 + 1 + 4 * 5 + 1 + 3 + 1 + 1 + 2 * 5 + 1
    return 1 + bin_sort + 1 + 2 + 1 + 2 + 2


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2032))}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6400.0, "source": "fallback", "sm_max_mhz": 2032.0}


def roofline(wl, stage_ms, peaks):
    """Algorithmic bytes of the HBM-bound stages per launch:
    adam 28 B per arena element; project 308 B per (view, Gaussian) at SH3
    (240 B of parameters read, 68 B of splat record written)."""
    n = wl.n
    algo = {"adam": 28.0 * wl.arena.padded,
            "project": (16 * 3 + 3 * 16 * 4 + 68.0) * n,
            "render_bwd_gaussians": None, "render_fwd": None, "render_bwd_pixels": None,
            "bin_sort": None, "loss": 3 * 4 * 3.0 * wl.pixels}
    dom = max(stage_ms, key=stage_ms.get)
    hbm_stages = {k: v for k, v in algo.items() if v is not None}
    pick = dom if dom in hbm_stages else max(hbm_stages, key=lambda k: stage_ms[k])
    t = stage_ms[pick] / 1e3
    ach = hbm_stages[pick] / t / 1e9
    return {"kernel": pick, "dominant_stage": dom, "bound": "hbm", "achieved": ach,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
            "peak_source": peaks["source"] + " (copy, burst)", "traffic": None,
            "algorithmic_bytes": hbm_stages[pick]}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample_step(scene, cams, k, targets=None):
    """One oracle iteration of the sampled workload: forward, L1 loss
    gradient, backward, Adam (FP64) over the sample's parameters."""
    import oracle
    cam = [cams[k % len(cams)]]
    out = oracle.render(scene, cam)
    tgt = targets if targets is not None else [np.zeros_like(out["image"][0])]
    _, dimg = oracle.l1_loss(out["image"], tgt)
    g = oracle.backward(scene, cam, dimg)
    p = np.concatenate([np.asarray(getattr(scene, a), np.float64).ravel()
                        for a in ("means", "log_scales", "quats", "opa_logits", "sh")])
    gg = np.concatenate([g[a].ravel() for a in ("means", "log_scales", "quats", "opa_logits", "sh")])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    oracle.adam(p, gg, m, v, 1e-3, 1)


def cpu_baseline(n, budget_s=20.0, divisor=64, steps=None):
    """The FP64 oracle as it stands, single-threaded, on 1/divisor of the
    Gaussians (the first n/divisor of the same scene) over the full 1280x720
    view; iterations/s scaled by that fraction (the per-iteration work of the
    renderer grows about linearly with the number of Gaussians)."""
    from paper_2607_14481_b300 import synth
    sc = synth.box_scene(n, SEED_SCENE).subset(np.arange(n // divisor))
    cams = synth.forward_trajectory(N_POSES, SEED_TRAJ)
    t0 = time.time()
    done = 0
    while True:
        oracle_sample_step(sc, cams, 10 + done)
        done += 1
        el = time.time() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= budget_s):
            break
    per = el / done
    return {"value": 1.0 / (per * divisor), "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} iteration(s) of fwd+bwd+Adam on {n // divisor} of the {n} Gaussians "
                      f"(1/{divisor}) over full 1280x720 views; value scaled by 1/{divisor}",
            "seconds": el}


def run_reference(args, ws, rank):
    if rank != 0:
        return None, rank
    import oracle  # noqa: F401  (builds the oracle if needed)
    divisor = 64
    from paper_2607_14481_b300 import synth
    sc = synth.box_scene(args.n, SEED_SCENE).subset(np.arange(args.n // divisor))
    cams = synth.forward_trajectory(N_POSES, SEED_TRAJ)
    for i in range(args.warmup):
        oracle_sample_step(sc, cams, i)
    t0 = time.time()
    for i in range(args.steps):
        oracle_sample_step(sc, cams, args.warmup + i)
    el = time.time() - t0
    value = args.steps / (el * divisor)
    sample = (f"per step: fwd+bwd+Adam of the FP64 oracle on {args.n // divisor} of the {args.n} "
              f"Gaussians (1/{divisor}) over one full 1280x720 view; value scaled by 1/{divisor}")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps * divisor,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"plain single-view training, {args.n} Gaussians SH3, 1280x720, "
                               f"100-pose forward trajectory, L1 loss", "gaussians": args.n},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }, rank


def main():
    args = parse_args()
    if args.impl == "reference":
        # the CPU oracle: rank 0 alone works; other ranks exit without work
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        out, rank = run_reference(args, ws, rank)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        return
    ws, rank, local = dist_setup(args.gpus)
    out, rank = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
