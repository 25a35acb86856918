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
import hashlib
import json
import math
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
N_BATCHED = 2_000_000  # Gaussians of the batched 16-view workload
N_POSES = 100
SEED_SCENE, SEED_TRAJ, SEED_TARGET, SEED_STREAM = 1007, 1008, 1009, 4007
SEED_BA = 5001
PAPER_BA_MS = 15.9  # Table "BA runtime": 10 iterations, 20 poses x 10,000 landmarks, on an RTX 4090


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--gaussians", "--n", dest="n", type=int, default=N_GAUSS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--stream-max", type=int, default=5_000_000)
    ap.add_argument("--no-ba", action="store_true")
    ap.add_argument("--no-lod", action="store_true")
    ap.add_argument("--lod-only", action="store_true",
                    help="run only the level-of-detail measurement (one JSON line)")
    ap.add_argument("--ba-only", action="store_true",
                    help="run only the local bundle adjustment measurement (one JSON line)")
    ap.add_argument("--fused-schedule", default=None,
                    help="pin the fused pass's schedule (an autotune candidate name, e.g. 8x32_b64_viewmajor) "
                         "instead of autotuning it; for profiling runs")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched measurement at --gaussians (one JSON line)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# multi-process (independent replicas; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup(gpus, backend=None):
    """One process per GPU (torchrun environment); NCCL on GPUs, gloo for the
    host-only checks of this logic."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class _NvmlLib:
    """The few read-only NVML queries the clock sampler makes, through the
    driver's libnvidia-ml with ctypes, for hosts without the Python binding.
    Reason bits are the NVML API's clocks-event-reason values."""
    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc):
        if rc != 0:
            raise RuntimeError(f"NVML error {rc}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2())

    def nvmlShutdown(self):
        self.lib.nvmlShutdown()

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.C.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.C.c_uint(i), self.C.byref(h)))
        return h

    def nvmlDeviceGetClockInfo(self, h, kind):
        v = self.C.c_uint()
        self._ok(self.lib.nvmlDeviceGetClockInfo(h, self.C.c_int(kind), self.C.byref(v)))
        return v.value

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        v = self.C.c_uint()
        self._ok(self.lib.nvmlDeviceGetMaxClockInfo(h, self.C.c_int(kind), self.C.byref(v)))
        return v.value

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.C.c_ulonglong()
        self._ok(self.lib.nvmlDeviceGetCurrentClocksThrottleReasons(h, self.C.byref(v)))
        return v.value


class ClockSampler:
    """SM clock and clock-event reasons while the timed loops run: read-only
    NVML queries every 5 ms from a thread (the timed region is a fraction of
    a second), else nvidia-smi at its 200 ms period."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.nv = None
        self.lines = []
        self.samples = []

    def start(self):
        try:
            try:
                import pynvml
            except ImportError:
                pynvml = _NvmlLib()
            pynvml.nvmlInit()
            self.h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            self.smax = float(pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM))
            self.bits = dict(zip(self.REASONS, (pynvml.nvmlClocksEventReasonHwSlowdown,
                                                pynvml.nvmlClocksEventReasonHwThermalSlowdown,
                                                pynvml.nvmlClocksEventReasonSwThermalSlowdown,
                                                pynvml.nvmlClocksEventReasonSwPowerCap)))
            self.nv = pynvml
            self.done = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        except Exception:
            self.nv = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _poll(self):
        nv = self.nv
        while not self.done.is_set():
            try:
                sm = float(nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM))
                r = int(nv.nvmlDeviceGetCurrentClocksEventReasons(self.h))
            except Exception:
                return
            self.samples.append((sm, r))
            self.done.wait(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nv is not None:
            self.done.set()
            self.thread.join(timeout=2)
            try:
                self.nv.nvmlShutdown()
            except Exception:
                pass
            sm = [x for x, _ in self.samples]
            reasons = sorted({nm for _, r in self.samples for nm, b in self.bits.items() if r & b})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.smax,
                    "reasons": reasons, "samples": len(sm), "source": "NVML every 5 ms"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(self.REASONS, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi every 200 ms"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
STAGES = ("project", "bin_sort", "render_fused", "bwd_gaussians_adam", "pose_adam")
STAGES_UNFUSED = ("project", "bin_sort", "render_fwd", "loss", "render_bwd_pixels", "render_bwd_gaussians", "adam")


class Workload:
    """Scene, optimiser state and per-view training steps for one set of views.

    plain: one view per iteration, cycling through the 100-pose trajectory,
    one captured CUDA graph per pose.  batched: all views of `cams` in every
    iteration (one Adam step), one captured graph."""

    def __init__(self, n, device, cams, batched, rank=0, use_graphs=True, fused=True, fused_schedule=None):
        import torch
        from paper_2607_14481_b300 import raster, synth, train
        self.torch, self.raster = torch, raster
        self.n, self.device, self.batched = n, device, batched
        self.cams = list(cams)
        self.scene = synth.box_scene(n, SEED_SCENE + 100 * rank)
        self.arena = raster.Arena.from_scene(self.scene, device)
        self.grads, self.m, self.v = self.arena.like(), self.arena.like(), self.arena.like()
        self.groups = self.arena.adam_groups(lr_means=1.6e-4 * 10.0)
        # the fused path also takes the parameters' Adam step inside the
        # per-Gaussian backward (same rates as the groups)
        P = len(self.cams)
        self.poses = raster.poses_tensor(self.cams, device)
        self.pose_m = torch.zeros((P, 6), dtype=torch.float32, device=device)
        self.pose_v = torch.zeros((P, 6), dtype=torch.float32, device=device)
        self.pose_steps = torch.zeros(P, dtype=torch.int32, device=device)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.adam = raster.adam_params(3, lr_means=1.6e-4 * 10.0, step_dev=self.step_dev, status=self.status)
        # plain: one view per step, buffers sized for the largest view
        views = self.cams if batched else [max(self.cams, key=lambda c: c.width * c.height)]
        self.rast = raster.Rasterizer(n, 3, views, device=device)
        self.loss = raster.ImageLoss(device)
        # targets: renders of a perturbed copy of the scene
        pert = raster.Arena.from_scene(synth.perturbed(self.scene, SEED_TARGET), device)
        groups = [self.cams] if batched else [[c] for c in self.cams]
        self.view_pixels = [sum(c.width * c.height for c in g) for g in groups]
        self.targets = [torch.empty(3 * px, dtype=torch.float32, device=device) for px in self.view_pixels]
        kmax = 0
        for k, g in enumerate(groups):
            self.rast.set_cameras(g)
            sl = slice(0, P) if batched else slice(k, k + 1)
            self.rast.forward(pert, self.poses[sl], self.targets[k], None, check=True)
            kmax = max(kmax, int(self.rast.read_counts()[1]))
            self.rast.forward(self.arena, self.poses[sl], self.rast.new_image(), None, check=True)
            kmax = max(kmax, int(self.rast.read_counts()[1]))
        del pert
        self.fused = fused
        k = len(groups) // 2
        sl = slice(0, P) if batched else slice(k, k + 1)
        timg = self.rast.new_image() if batched else torch.empty(3 * max(self.view_pixels), device=device)
        if fused:
            # tile shape, splats per batch and work order of the fused pass, on
            # the middle view group; then the pair capacity for that tile shape
            self.rast.set_capacity(int(kmax * 1.5) + 4096)
            self.rast.set_cameras(groups[k])
            if fused_schedule:
                # pinned (profiling runs: the autotuner's timings are not
                # comparable under a profiler)
                self.rast.set_fused_schedule(fused_schedule)
                self.tuning = {"tile": list(self.rast.tile), "schedule": int(self.rast.cfg.schedule),
                               "pinned": fused_schedule}
            else:
                self.tuning = self.rast.autotune_fused(self.arena, self.poses[sl], self.targets[k], 0,
                                                       timg[:3 * self.view_pixels[k]], self.loss.loss, reps=3)
            kmax = 0
            for j, g in enumerate(groups):
                self.rast.set_cameras(g)
                slj = slice(0, P) if batched else slice(j, j + 1)
                self.rast.forward(self.arena, self.poses[slj], timg[:3 * self.view_pixels[j]], None, check=True)
                kmax = max(kmax, int(self.rast.read_counts()[1]))
            self.rast.set_capacity(int(kmax * 1.3) + 4096)  # fixed: no host synchronisation per step
        else:
            self.rast.set_capacity(int(kmax * 1.3) + 4096)
            # blend schedule of the separate kernels, on the middle view group
            self.rast.set_cameras(groups[k])
            ti = self.rast.new_image()
            tdimg = self.rast.new_image()
            self.rast.forward(self.arena, self.poses[sl], ti, None, check=True)
            self.loss(ti, self.targets[k], tdimg, 0)
            self.tuning = self.rast.autotune(ti, tdimg, reps=3)
            del ti, tdimg
        self.kmax = kmax
        del timg
        img = self.rast.new_image() if batched else torch.empty(3 * max(self.view_pixels), device=device)
        dimg = torch.empty_like(img)
        self.steps = []
        for k, g in enumerate(groups):
            sl = slice(0, P) if batched else slice(k, k + 1)
            px = self.view_pixels[k]
            self.steps.append(train.TrainStep(
                self.arena, self.grads, self.m, self.v, self.groups, self.rast, self.poses[sl], self.targets[k],
                self.step_dev, pose_m=self.pose_m[sl], pose_v=self.pose_v[sl], pose_steps=self.pose_steps[sl],
                pose_lr=1e-4, loss_kind=0, status=self.status, image=img[:3 * px], dimage=dimg[:3 * px],
                loss=raster.ImageLoss(device), cams=g, fused=fused, adam=self.adam if fused else None))
        if use_graphs:
            self.pool = torch.cuda.graph_pool_handle()
            for st in self.steps:
                st.capture(pool=self.pool)
            # every graph replayed once, so no timed step is a graph's first replay
            for st in self.steps:
                st.run()
            torch.cuda.synchronize()
        self.targets_host = [t.cpu().pin_memory() for t in self.targets]
        self.i = 0
        self.pixels_per_iter = self.view_pixels[0] if batched else self.cams[0].width * self.cams[0].height

    def step(self):
        st = self.steps[self.i % len(self.steps)]
        self.i += 1
        st.run()
        return st

    def sequence(self, K):
        """Trajectory positions of K timed steps spread evenly over the whole
        trajectory (step i takes pose floor(i P / K) of the P poses), so the
        timed window covers every part of it whatever K is."""
        P = len(self.steps)
        return [(i * P) // K % P for i in range(K)]

    def instrumented_step(self, ev, k=None):
        """The same iteration (trajectory position k, default the next one)
        run eagerly with CUDA events at the stage boundaries (on the launching
        stream)."""
        if k is None:
            k = self.i % len(self.steps)
        st = self.steps[k]
        self.i += 1
        r = st.rast
        r.set_cameras(st.cams)
        e = iter(ev)
        next(e).record()
        r.project(st.arena, st.poses)
        next(e).record()
        r.bin_sort()
        next(e).record()
        if self.fused:
            r.fused(st.targets, st.kind, st.img, None, st.loss.loss)
            next(e).record()
        else:
            r.render_fwd(st.img, None)
            next(e).record()
            st.loss(st.img, st.targets, st.dimg, st.kind)
            next(e).record()
            r.backward_pixels(st.dimg, None, st.img)
            next(e).record()
        if st.adam is not None:
            r.backward_gaussians_adam(st.arena, st.poses, st.grads, st.m, st.v, st.adam, st.dpose)
            groups = []
        else:
            r.backward_gaussians(st.arena, st.poses, st.grads, st.dpose)
            groups = st.groups
        next(e).record()
        self.raster.adam_step(st.arena, st.grads, st.m, st.v, 0, groups, status=st.status, pose=st.poses,
                              dpose=st.dpose, pose_m=st.pose_m, pose_v=st.pose_v, pose_lr=st.pose_lr,
                              step_dev=st.step_dev, pose_steps_dev=st.pose_steps)
        next(e).record()

    def stages(self):
        return STAGES if self.fused else STAGES_UNFUSED

    def check_device_status(self):
        cnt = self.rast.read_counts()
        assert cnt[2] == 0, f"binning status {cnt[2]} (1 = capacity, 2 = index)"
        return int(self.status.item())


def timed_loop(wl, K, ws, e2e=False):
    """K iterations between a barrier + synchronize on both sides; device time
    from CUDA events on the launching stream, max over ranks.  The K steps
    take the poses of wl.sequence(K) (spread over the whole trajectory).

    e2e: every iteration also copies its target image from pinned host memory
    (on a copy stream, one iteration ahead, so the copy of iteration i + 1
    overlaps the compute of iteration i; iteration i waits for its own copy,
    and a copy into a target buffer waits for the last iteration that read
    it) and reads its loss back to pinned host memory: on a third stream
    once the iteration's kernels are done, so the next iteration does not
    wait behind the copy (each trajectory position has its own loss word, and
    an iteration waits for the read of its word's previous value; the end
    event waits for the last read)."""
    import torch
    seq = wl.sequence(K)
    loss_host = torch.zeros(max(K, 1), dtype=torch.float32).pin_memory() if e2e else None
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream() if e2e else None
    readback = torch.cuda.Stream() if e2e else None
    done_ev = [None] * len(wl.steps)  # last iteration that read each target buffer
    read_ev = [None] * len(wl.steps)  # last read of each position's loss word

    def issue_copy(k):
        ev = torch.cuda.Event()
        with torch.cuda.stream(copy):
            if done_ev[k] is not None:
                copy.wait_event(done_ev[k])
            wl.steps[k].targets.copy_(wl.targets_host[k], non_blocking=True)
            ev.record(copy)
        return ev

    barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    t0.record()
    ready = issue_copy(seq[0]) if e2e else None
    for i in range(K):
        k = seq[i]
        st = wl.steps[k]
        if e2e:
            comp.wait_event(ready)
            if read_ev[k] is not None:
                comp.wait_event(read_ev[k])
        st.run()
        if e2e:
            done_ev[k] = torch.cuda.Event()
            done_ev[k].record(comp)
            with torch.cuda.stream(readback):
                readback.wait_event(done_ev[k])
                loss_host[i:i + 1].copy_(st.loss.loss, non_blocking=True)
                read_ev[k] = torch.cuda.Event()
                read_ev[k].record(readback)
            if i + 1 < K:
                ready = issue_copy(seq[i + 1])
    if e2e:
        comp.wait_stream(readback)
    t1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if e2e and not bool(torch.isfinite(loss_host[:K]).all()):
        raise RuntimeError("a loss read back in the end-to-end loop is not finite")
    barrier(ws)
    wl.i += K
    return allreduce_max(t0.elapsed_time(t1) / 1e3, ws)


def stage_times(wl, K):
    """Per-stage device times (CUDA events on the launching stream) of K eager
    iterations over poses spread along the trajectory, and the blend work
    counts of each iteration's tile lists (their means).  Each iteration is
    queued behind a 2 ms spin of the device, so that the host has issued its
    launches before the device reaches them and no stage time includes the
    host's launch latency (the work counts synchronise every iteration)."""
    import torch
    names = wl.stages()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(K)]
    counts = []
    seq = wl.sequence(K)
    for i in range(K):
        torch.cuda._sleep(4_000_000)  # outside the range that profiles select
        torch.cuda.nvtx.range_push("eager")
        wl.instrumented_step(evs[i], seq[i])
        counts.append(wl.rast.render_stats())
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = {s: float(np.mean([evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(K)]))
          for j, s in enumerate(names)}
    work = {k: float(np.mean([c[k] for c in counts])) for k in counts[0]}
    return ms, work


def run_batched(n, device, cams16, K, warmup, ws, rank, fused_schedule=None):
    """16 views of uneven size per iteration (one Adam step), one CUDA graph."""
    import torch
    wb = Workload(n, device, cams16, batched=True, rank=rank, fused_schedule=fused_schedule)
    for _ in range(max(3, warmup)):
        wb.step()
    torch.cuda.synchronize()
    Kb = max(5, K // 8)
    eb = timed_loop(wb, Kb, ws)
    wb.check_device_status()
    sb, wkb = stage_times(wb, min(Kb, 10))
    out = {"gaussians": n, "views_per_iter": 16, "iters_per_s": ws * Kb / eb,
           "view_iters_per_s": ws * 16 * Kb / eb,
           "mpix_per_s": ws * Kb * wb.pixels_per_iter / eb / 1e6,
           "ms_per_iter": 1e3 * eb / Kb, "steps": Kb,
           "pixels_per_iter": wb.pixels_per_iter, "pairs_max": wb.kmax,
           "resolutions": [[c.width, c.height] for c in cams16], "stage_ms": sb,
           "blend_schedule": wb.tuning,
           "roofline": roofline(wb, sb, wkb, load_peaks(), sm_count(device))}
    del wb
    torch.cuda.empty_cache()
    # the same 16 views trained one per Adam step (the plain mode on this view
    # mix): what batching them into one step buys
    wp = Workload(n, device, cams16, batched=False, rank=rank)
    for _ in range(max(3, warmup)):
        wp.step()
    torch.cuda.synchronize()
    Kp = 16 * max(2, Kb // 2)
    ep = timed_loop(wp, Kp, ws)
    wp.check_device_status()
    out["plain_same_views"] = {"view_iters_per_s": ws * Kp / ep, "ms_per_view_iter": 1e3 * ep / Kp, "steps": Kp,
                               "blend_schedule": wp.tuning}
    out["vs_plain_same_views"] = out["view_iters_per_s"] / out["plain_same_views"]["view_iters_per_s"]
    del wp
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local):
    import torch
    from paper_2607_14481_b300 import build, synth
    if rank == 0:
        build.build()
    barrier(ws)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    K = args.steps
    # ---- plain single-view training (the headline)
    wl = Workload(args.n, device, synth.forward_trajectory(N_POSES, SEED_TRAJ), batched=False, rank=rank,
                  fused_schedule=args.fused_schedule)
    for _ in range(max(3, args.warmup)):
        wl.step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)  # over both timed loops (device-timed and end-to-end)
    clocks.start()
    elapsed = timed_loop(wl, K, ws)
    bad = wl.check_device_status()
    value = ws * K / elapsed
    e2e = None
    if not args.no_e2e:
        e_el = timed_loop(wl, K, ws, e2e=True)
        e2e = {"value": ws * K / e_el, "unit": "iters/s",
               "h2d_bytes_per_step": int(wl.targets[0].numel() * 4), "d2h_bytes_per_step": 4,
               "ms_per_step": 1e3 * e_el / K}
    clk = clocks.stop()
    if not args.no_e2e:
        wl.check_device_status()
    stage_ms, work = stage_times(wl, min(K, 30))
    wl.check_device_status()
    peaks = load_peaks()
    roof = roofline(wl, stage_ms, work, peaks, sm_count(device), workload_key=traffic_key(args.n))
    poses_timed = wl.sequence(K)
    plain_pixels = wl.pixels_per_iter
    n_launch = launches_per_step(1, wl.rast.num_tiles, bool(wl.tuning["schedule"] & 7))
    plain_tuning = wl.tuning
    del wl
    torch.cuda.empty_cache()

    # ---- the same plain step with the three separate blend launches
    # (composite, loss, per-pixel backward) instead of the fused pass
    unfused = None
    if not args.no_unfused:
        wu = Workload(args.n, device, synth.forward_trajectory(N_POSES, SEED_TRAJ), batched=False, rank=rank,
                      fused=False)
        for _ in range(max(3, args.warmup)):
            wu.step()
        torch.cuda.synchronize()
        eu = timed_loop(wu, K, ws)
        wu.check_device_status()
        su, _ = stage_times(wu, min(K, 10))
        unfused = {"value": ws * K / eu, "unit": "iters/s", "ms_per_step": 1e3 * eu / K, "stage_ms": su,
                   "fused_speedup": value / (ws * K / eu), "blend_schedule": wu.tuning}
        del wu
        torch.cuda.empty_cache()

    # ---- batched: 16 views of uneven size per iteration (one Adam step), at
    # the headline's Gaussian count and at the batched workload's 2M
    batched = None
    if not args.no_batched:
        cams16 = synth.loop_views(16, SEED_TRAJ + 1)
        batched = run_batched(args.n, device, cams16, K, args.warmup, ws, rank)
        batched["vs_plain_view_iters"] = batched["view_iters_per_s"] / (ws * K / elapsed)
        # equal work per view: the same 16 loop views, all at the plain mode's 1280x720
        eq = run_batched(args.n, device, [synth.with_resolution(c, 1280, 720) for c in cams16], K,
                         args.warmup, ws, rank)
        batched["equal_work_720p"] = {k: eq[k] for k in ("view_iters_per_s", "mpix_per_s", "ms_per_iter",
                                                         "pixels_per_iter", "pairs_max", "stage_ms")}
        batched["equal_work_720p"]["vs_plain_view_iters"] = eq["view_iters_per_s"] / (ws * K / elapsed)
        if args.n != N_BATCHED:
            batched["at_2m"] = run_batched(N_BATCHED, device, cams16, K, args.warmup, ws, rank)

    stream = None
    if not args.no_stream and rank == 0:
        stream = run_streaming(args.stream_max)
    loop = run_loop_closure(5_000_000, device) if rank == 0 else None
    local_ba = run_local_ba(device, cpu=(ws == 1 and not args.no_cpu_baseline)) \
        if rank == 0 and not args.no_ba else None
    lod = run_lod(device) if rank == 0 and not args.no_lod else None

    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.n, ws),
        "poses_timed": {"trajectory_poses": N_POSES, "timed_steps": K, "first": poses_timed[0],
                        "last": poses_timed[-1], "distinct": len(set(poses_timed)),
                        "rule": "step i takes pose floor(i * 100 / K) mod 100; every pose's graph replayed "
                                "once before timing"},
        "blend_schedule": plain_tuning,
        "mpix_per_s": value * plain_pixels / 1e6,
        "stage_ms": stage_ms,
        "unfused": unfused,
        "e2e": e2e,
        "roofline": roof,
        "batched": batched,
        "streaming": stream,
        "loop_closure": loop,
        "local_ba": local_ba,
        "lod": lod,
        "clocks": clk,
        "gpu_launches": n_launch * K,
        "nonfinite_flag": bad,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.n)
    return out, rank


def workload_config(n, ws=1):
    """The workload both arms measure (identical dict in both JSON lines)."""
    return {"workload": f"plain single-view training, {n} Gaussians SH3, 1280x720, 100-pose forward "
                        f"trajectory, L1 loss (fwd + bwd incl. pose + Adam per iteration)",
            "gaussians": n, "views_per_iter": 1, "resolution": [1280, 720], "sh_degree": 3,
            "parallelism": f"replicas{ws}",
            "l2": "inputs larger than L2 (parameter arena 240 MB, x4 with gradients and moments)"}


def traffic_key(n):
    return f"plain 1280x720 SH3 n={n}"


def run_loop_closure(n, device, reps=20, n_kf=160, seed=SEED_STREAM):
    """The loop-closure update (gs_sim3_update) of n SH3 Gaussians tagged
    with n_kf keyframes: device time per update (CUDA events, inputs larger
    than L2) against the measured HBM copy bandwidth; 100 B per Gaussian
    (keyframe id 4 B, means / scales / rotation 48 B read and 48 B written)."""
    import torch
    from paper_2607_14481_b300 import raster
    g = np.random.default_rng(seed)
    arena = raster.Arena(n, 3, device)
    arena.quat[:, 0] = 1.0
    kf = torch.from_numpy(g.integers(0, n_kf, n).astype(np.int32)).to(device)
    q = g.normal(size=(n_kf, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    S = np.concatenate([q, 0.01 * g.normal(size=(n_kf, 3)), np.ones((n_kf, 1))], axis=1).astype(np.float32)
    S = torch.from_numpy(S).to(device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    for _ in range(3):
        raster.sim3_update(arena, kf, S, status)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        raster.sim3_update(arena, kf, S, status)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peaks = load_peaks()
    gbs = 100.0 * n / (ms / 1e3) / 1e9
    return {"gaussians": n, "keyframes": n_kf, "ms": ms, "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
            "frac": gbs / peaks["hbm_gbs"], "bytes_per_gaussian": 100,
            "l2": "inputs larger than L2 (5M x 52 B read)"}


def run_local_ba(device, iters=10, reps=30, cpu=True, seed=SEED_BA):
    """Local bundle adjustment (gs_ba_solve) on the problem of the paper's BA
    timing table: 20 keyframes (4 fixed), 10,000 landmarks, 8 observing
    keyframes each, shared focal optimised, 0.5 px observation noise; `iters`
    Levenberg-Marquardt iterations captured in one CUDA graph, timed with CUDA
    events (device-resident inputs; the 28 MB workspace stays in L2, as it
    does in the pipeline).  e2e: the one-shot host API (observations, poses
    and landmarks copied in, results copied out) per solve.  cpu_baseline:
    the FP64 oracle's `iters` iterations on the same problem, on this host."""
    import torch
    from paper_2607_14481_b300 import synth
    from paper_2607_14481_b300.ba import BundleAdjuster, bundle_adjust
    p = synth.ba_problem(seed, n_cams=20, n_points=10_000, obs_per_point=8, n_fixed=4)
    fixed = [True] * 4 + [False] * 16
    cam = torch.as_tensor(p["obs_cam"], device=device)
    uv = torch.as_tensor(p["obs_uv"], device=device)
    ba = BundleAdjuster(cam, uv, 20, fixed, p["cx"], p["cy"], max_iters=iters)
    P0 = torch.as_tensor(p["poses0"], device=device)
    X0 = torch.as_tensor(p["points0"], device=device)
    f0 = torch.tensor([p["f0"]], dtype=torch.float32, device=device)
    P, X, f = P0.clone(), X0.clone(), f0.clone()

    def reset():
        P.copy_(P0)
        X.copy_(X0)
        f.copy_(f0)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            reset()
            ba.solve(P, X, f, iters=iters)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ba.solve(P, X, f, iters=iters)
    times = []
    for _ in range(reps):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    trace = ba.trace[:iters].cpu().numpy()
    status = int(ba.status.item())
    # end to end through the host API (fresh workspace each call, as a user would)
    bundle_adjust(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"], p["cy"], fixed,
                  iters=iters)
    t0 = time.perf_counter()
    n_e2e = 5
    for _ in range(n_e2e):
        bundle_adjust(p["poses0"], p["points0"], p["f0"], p["obs_cam"], p["obs_uv"], p["cx"], p["cy"], fixed,
                      iters=iters)
    e2e_ms = 1e3 * (time.perf_counter() - t0) / n_e2e
    ms = statistics.median(times)
    out = {"workload": "20 keyframes (4 fixed) x 10,000 landmarks x 8 observations, shared focal, "
                       f"{iters} LM iterations", "iterations": iters, "ms": ms, "ms_min": min(times),
           "ms_per_iteration": ms / iters, "launches": 2 + 4 * iters + 1,
           "initial_cost": float(trace[0, 0]), "final_cost": float(trace[-1, 0] if not trace[-1, 3] else trace[-1, 1]),
           "accepted": int(trace[:, 3].sum()), "status": status,
           "e2e_ms": e2e_ms, "paper_ms_rtx4090": PAPER_BA_MS,
           "note": "the paper's figure is another GPU's (context, not a target)"}
    if cpu:
        # the oracle in a fresh single-threaded interpreter (BLAS/OpenMP pools of 1)
        code = ("import json, sys, time; sys.path.insert(0, %r); import numpy as np; "
                "from paper_2607_14481_b300 import synth; from oracle import ba as oba; "
                "p = synth.ba_problem(%d, n_cams=20, n_points=10000, obs_per_point=8, n_fixed=4); "
                "fx = np.array([True] * 4 + [False] * 16); t0 = time.perf_counter(); "
                "o = oba.solve(p['poses0'], p['points0'], p['f0'], p['obs_cam'], p['obs_uv'], p['cx'], p['cy'], "
                "fx, iters=%d); print(json.dumps({'ms': 1e3 * (time.perf_counter() - t0), 'cost': o['cost']}))"
                % (os.path.dirname(os.path.abspath(__file__)), seed, iters))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
        o = json.loads(res.stdout.strip().splitlines()[-1])
        cpu_ms = o["ms"]
        out["cpu_baseline"] = {"value": cpu_ms, "unit": "ms per solve", "cores": 1, "kind": "oracle",
                               "sample": f"the full problem, {iters} iterations (numpy/scipy FP64)",
                               "final_cost": o["cost"]}
    return out


def run_lod(device, n_frames=100, per_frame=50_000, reps=5, keyframe_every=10, loop_m=1000.0, seed=SEED_STREAM):
    """The progressive hierarchy (Sec. 6.1 merging and retrieval, Sec. 6.2
    rendering) on a large streamed scene: n_frames x per_frame Gaussians
    spawned in the frustums of a camera walking a loop_m loop (10 m between
    frames; about 1.5 px on screen when spawned, so most of the scene is
    sub-pixel from any one camera), in overlapping groups of four as on a
    reconstructed surface (synth.frustum_clusters), SH3, node rows for twice
    the leaves.  An analysis
    (merge below tau_l = 0.5 px when more than 20% qualify, then reload above
    tau_h = 1 px) runs from every keyframe_every-th camera, in loop order,
    each timed with CUDA events.  Then, for the 1080p views of frames 0, 25,
    50 and 75: the splats the projection keeps and the tile pairs with all
    leaves, with the final active set refined for the view (what a training
    view optimises) and with the render cut from the roots at tau = 1 px
    (what a render draws, Sec. 6.2), and the time of projection + binning +
    composite of each (mean of `reps`)."""
    import torch
    from paper_2607_14481_b300 import raster, synth
    cams = [synth.stream_camera(k, n_frames, loop_m=loop_m) for k in range(n_frames)]
    parts = [synth.frustum_clusters(cams[k], per_frame, seed * 7919 + k) for k in range(n_frames)]
    sc = synth.Scene(*(np.concatenate([getattr(p, f) for p in parts]) for f in
                       ("means", "log_scales", "quats", "opa_logits", "sh")))
    del parts
    n = sc.n
    arena = raster.Arena.from_scene(sc, device, capacity=2 * n)
    del sc
    hier = raster.Hierarchy(arena, n)

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    analyses = []
    for k in range(0, n_frames, keyframe_every):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        hier.analyze(cams[k])
        e1.record()
        hier.refine(cams[k])
        e2.record()
        torch.cuda.synchronize()
        st = hier.state()
        info = st["info"]
        analyses.append({"frame": k, "analyze_ms": e0.elapsed_time(e1), "reload_ms": e1.elapsed_time(e2),
                         "nodes": st["n_nodes"], "active": int(st["active"][:st["n_nodes"]].sum()),
                         "candidates": int(info[2]), "triggered": int(info[1]), "groups": int(info[5]),
                         "pulled": int(info[4])})
    st = hier.state()
    rows = st["n_nodes"]
    out = {"leaves": n, "loop_m": loop_m, "node_rows": rows, "active": int(st["active"][:rows].sum()),
           "merged_nodes": rows - n, "analyses": analyses,
           "analysis_ms_mean": float(np.mean([a["analyze_ms"] + a["reload_ms"] for a in analyses])),
           "tau_l": 0.5, "tau_h": 1.0, "views": {}}

    class _Leaves:  # the first n rows of the node arena (its SH stride), as projection parameters
        def struct(self):
            return arena.struct(n)

    leaves = _Leaves()
    for k in (0, n_frames // 4, n_frames // 2, 3 * n_frames // 4):
        poses = raster.poses_tensor([cams[k]], device)
        res = {}
        for name in ("leaves", "active_cut", "render_cut"):
            r = raster.Rasterizer(n if name == "leaves" else rows, 3, [cams[k]], device=device)
            img = r.new_image()
            if name == "leaves":
                pj = lambda: r.project(leaves, poses)
            else:
                pj = lambda: r.project_hier(hier, poses, tau_h=1.0, from_roots=name == "render_cut")
            pj()
            r.set_capacity(max(4096, r.capacity))
            r.bin_sort()
            torch.cuda.synchronize()
            c = r.read_counts()
            if c[2] & 1:
                r.set_capacity(int(c[1] * 1.25) + 4096)
            pj()
            r.bin_sort()
            torch.cuda.synchronize()
            c = r.read_counts()

            def fwd():
                pj()
                r.bin_sort()
                r.render_fwd(img, None)
            res[name] = {"rendered_splats": int(c[0]), "pairs": int(c[1]), "project_bin_render_ms": timed(fwd, reps)}
            del r, img
            torch.cuda.empty_cache()
        res["splat_ratio"] = res["render_cut"]["rendered_splats"] / max(1, res["leaves"]["rendered_splats"])
        res["speedup"] = res["leaves"]["project_bin_render_ms"] / res["render_cut"]["project_bin_render_ms"]
        out["views"][f"frame{k}"] = res
    out["paper_traversal_ms"] = "5-30 (the paper's hierarchy traversal per frame; another GPU; context)"
    del hier, arena, leaves
    torch.cuda.empty_cache()
    return out


def run_streaming(n_max, seed=SEED_STREAM, rate_hz=30.0, n0=100_000):
    """The streaming session loop: the scene grows from n0 to n_max Gaussians
    while frames arrive in real time at rate_hz; every frame adds its new
    Gaussians (U{10k..50k}, in the frame camera's frustum) and submits
    U{1..8} render / train requests at 540p-1080p as one group; every 10th
    frame is a keyframe whose camera analyses the progressive hierarchy
    (renders draw its render cut, trains the active set's cut; tau = 1 px);
    admission by an 80 GB HBM budget.  Frame-update latency = a train request's
    arrival (its frame's arrival) to the completion of the Adam step that
    used it."""
    import time
    from paper_2607_14481_b300 import session, synth
    avg_new = 30_000
    n_frames = max(1, (n_max - n0) // avg_new)
    cfg = session.default_config(n_max + 60_000, sh_degree=3, max_batch_views=8, max_width=1920, max_height=1080,
                                 max_inflight=2, hbm_budget_gb=80.0, pair_factor=8.0, lod=True, lod_tau=1.0)
    g = np.random.default_rng(seed)
    # train targets in pinned host memory, as frames a capture pipeline has
    # written there: the session reads them in place (borrowed), no copy at submit
    import torch
    targets = {wh: [torch.from_numpy(g.random((3, wh[1], wh[0]), dtype=np.float32)).pin_memory() for _ in range(2)]
               for wh in synth.STREAM_RESOLUTIONS}
    frames = [synth.stream_frame(k, n_frames, seed) for k in range(n_frames)]
    ids = []
    analyses = 0
    with session.Session(cfg) as s:
        s.add(synth.frustum_gaussians(synth.stream_camera(0, n_frames), n0, seed + 1))
        n = n0
        t0 = session.now() + 0.5
        for k, (cam, new, reqs) in enumerate(frames):
            t_arr = t0 + k / rate_hz
            while session.now() < t_arr:
                time.sleep(min(0.002, max(0.0, t_arr - session.now())))
            if n + new.n <= n_max + 60_000:
                s.add(new)
                n += new.n
            if k % 10 == 9:  # a keyframe: analyse the hierarchy (skipped while the last one runs)
                analyses += int(s.analyze(cam))
            s.hold(True)
            for i, (kind, w, h) in enumerate(reqs):
                c = synth.with_resolution(cam, w, h)
                tgt = targets[(w, h)][(k + i) % 2] if kind == 1 else None
                ids.append((kind, s.submit(kind, c, target=tgt, arrival=t_arr, borrow_target=tgt is not None)))
            s.hold(False)
        s.drain(timeout_ms=600_000)
        st = s.stats()
        times = [(kind, s.times(i)) for kind, i in ids]
    lat = {0: [], 1: []}
    last = t0
    for kind, (a, d) in times:
        lat[kind].append(1e3 * (d - a))
        last = max(last, d)
    wall = last - t0

    def pct(x, q):
        return float(np.percentile(x, q)) if x else None

    return {"frames": n_frames, "rate_hz": rate_hz, "requests": len(ids), "train_requests": len(lat[1]),
            "gaussians_start": n0, "gaussians_final": int(st["gaussians"]),
            "frame_update_p50_ms": pct(lat[1], 50), "frame_update_p99_ms": pct(lat[1], 99),
            "render_p50_ms": pct(lat[0], 50), "render_p99_ms": pct(lat[0], 99),
            "iterations": int(st["iterations"]), "iters_per_s": st["iterations"] / wall, "wall_s": wall,
            "batches": int(st["batches"]), "retries": int(st["retries"]), "analyses_issued": analyses,
            "analyses_swapped_in": int(st["lod_builds"]),
            "hbm_in_use_gb": st["hbm_in_use"] / 2 ** 30, "hbm_budget_gb": st["hbm_budget"] / 2 ** 30,
            "contexts": int(st["contexts"]),
            "workload": "camera on a 200 m loop, frames at 30 Hz, U{10k..50k} new Gaussians per frame in the "
                        "frame camera's frustum, U{1..8} requests per frame (render/train p = 0.5, 540p-1080p; train "
                        "targets in pinned host memory, borrowed by the session), "
                        "progressive hierarchy analysed every 10th frame (renders: render cut, trains: the active "
                        "set's cut, tau = 1 px), 80 GB HBM budget"}


def launches_per_step(views, num_tiles, tile_order=False, fused=True, fused_adam=None):
    """Kernels one training step launches: projection 1; binning 5 (zeroing
    of counters and ranges, pair-offset scan with the count pass, tile scan
    with the length grouping and any longest-first order, keys (the wide
    splats' chunks in the same launch), tile sort; more than 2^13 tiles take
    a three-kernel device scan and two ordering kernels instead of the
    one-CTA tile scan); the fused
    composite + loss + per-pixel backward 1 (or, unfused, composite 1, loss
    2, per-pixel backward 1); per-Gaussian backward 5 (pair sums,
    projection, SH, pose chunks and total); Adam 3 (parameters, poses, step
    counter), 2 when the parameters' step runs inside the SH kernel
    (fused_adam, by default with the fused pass)."""
    if fused_adam is None:
        fused_adam = fused
    tile_scan = 1 if num_tiles <= (1 << 13) else 3 + 2
    bin_sort = 1 + 1 + tile_scan + 1 + 1
    blend = 1 if fused else 1 + 2 + 1
    return 1 + bin_sort + blend + 5 + (2 if fused_adam else 3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2032))}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6400.0, "source": "fallback", "sm_max_mhz": 2032.0}


# Per evaluated (pixel, splat) pair of the plain per-pixel loop (a pair is
# evaluated when the pixel reaches the splat in its tile's list: up to and
# including the splat that stops it):
#   forward composite  ~12 FP32 operations + 1 MUFU (the exponential);
#   backward           ~45 FP32 operations + 2 MUFU / divides (two traversals:
#                      the forward's decisions and the gradient walk).
# Algorithmic operation counts, not the kernels' own (their per-warp culling
# skips pairs no pixel of a warp can reach, which still count here).
OPS_FWD_FP32, OPS_FWD_MUFU = 12, 1
OPS_BWD_FP32, OPS_BWD_MUFU = 45, 2
FP32_PER_SM_CLK, MUFU_PER_SM_CLK = 128, 16
RADIX_DIGIT_BITS = 11  # the LSD radix sort the binning's algorithmic bytes are counted for


def bin_sort_bytes(pairs, items, tiles):
    """Algorithmic bytes of binning: per pair 12 B emitted (key + value), a
    stable LSD radix sort of the significant key bits (32 depth bits + the
    tile bits) at 24 B per pass over 11-bit digits, 8 B of range reads; 4 B of
    scan per (view, Gaussian)."""
    bits = 32 + max(1, math.ceil(math.log2(max(2, tiles))))
    passes = math.ceil(bits / RADIX_DIGIT_BITS)
    return pairs * (12 + 24 * passes + 8) + 4 * items, passes


def sm_count(device=None):
    import torch
    return int(torch.cuda.get_device_properties(device if device is not None else 0).multi_processor_count)


def alu_roofline(pairs, fp32_per, mufu_per, t_s, sms, clk_mhz):
    """Algorithmic FP32 operations per second against the bound of the pair
    rate: min(SMs x 128 FP32 / clk / fp32_per, SMs x 16 MUFU / clk / mufu_per)."""
    clk = clk_mhz * 1e6
    fp32_pairs = sms * FP32_PER_SM_CLK * clk / fp32_per
    mufu_pairs = sms * MUFU_PER_SM_CLK * clk / mufu_per
    binding = "fp32" if fp32_pairs <= mufu_pairs else "mufu"
    peak_pairs = min(fp32_pairs, mufu_pairs)
    rate = pairs / t_s
    return {"bound": "alu", "achieved": rate * fp32_per / 1e9, "peak": peak_pairs * fp32_per / 1e9,
            "unit": "Gop/s", "frac": rate / peak_pairs, "binding_unit": binding,
            "pairs_per_s": rate, "algorithmic": pairs * fp32_per,
            "per_pair": {"fp32": fp32_per, "mufu": mufu_per}}


def load_traffic(kernel, workload_key):
    """DRAM bytes per launch of `kernel` from the machine-readable capture
    summary, if one was taken on this workload with the current source of the
    kernel (sha256 of its .cu file); else None and the reason."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as fh:
            entries = json.load(fh)["entries"]
    except (OSError, KeyError, ValueError):
        return None, "no capture summary"
    for e in entries:
        if e.get("kernel") != kernel or e.get("workload") != workload_key:
            continue
        src = os.path.join(ROOT, e["source"])
        try:
            with open(src, "rb") as fh:
                sha = hashlib.sha256(fh.read()).hexdigest()
        except OSError:
            return None, "kernel source missing"
        if sha != e.get("source_sha256"):
            return None, "kernel source changed since the capture"
        return float(e["bytes_per_launch"]), f"ncu capture ({e.get('kernel_name', kernel)})"
    return None, "no capture of this kernel on this workload"


def roofline(wl, stage_ms, work, peaks, sms, workload_key=None):
    """Achieved fraction of each stage's bound, with the algorithmic work per
    unit of the hot path's scope table: HBM bytes for projection, binning,
    the per-Gaussian backward, Adam and the loss; FP32 / MUFU operations per
    evaluated pair for the blend stages.  The dominant stage's object is the
    JSON line's roofline."""
    n = wl.n
    V = len(wl.steps[0].cams)
    K = work["listed"]
    E = work["evaluated"]
    clk = peaks["sm_max_mhz"]
    bs_bytes, passes = bin_sort_bytes(K, n * V, wl.rast.num_tiles)
    F = wl.arena.padded / n  # floats per Gaussian (60 at SH degree 3)
    hbm = {
        "project": (240.0 + 48.0) * n * V,
        "bin_sort": bs_bytes,
        "render_bwd_gaussians": 36.0 * K + 480.0 * n,
        "adam": 28.0 * wl.arena.padded,
        # fused: 36 B per pair summed; per Gaussian its parameters read once
        # (4 B per float), the means / scale / rotation gradients written and
        # read back (12 floats), and the moments read and parameters and
        # moments written (20 B per float): the gradient round trip of the
        # separate Adam is gone
        "bwd_gaussians_adam": 36.0 * K + (24.0 * F + 96.0) * n,
        "loss": 36.0 * wl.pixels_per_iter,
    }
    table = {}
    for k, amount in hbm.items():
        if k not in stage_ms:
            continue
        t = stage_ms[k] / 1e3
        ach = amount / t / 1e9
        table[k] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "algorithmic": amount}
    table["bin_sort"]["radix_passes"] = passes
    if "render_fused" in stage_ms:
        # composite + loss + backward: both traversals' work per evaluated pair
        table["render_fused"] = alu_roofline(E, OPS_FWD_FP32 + OPS_BWD_FP32, OPS_FWD_MUFU + OPS_BWD_MUFU,
                                             stage_ms["render_fused"] / 1e3, sms, clk)
    else:
        table["render_fwd"] = alu_roofline(E, OPS_FWD_FP32, OPS_FWD_MUFU, stage_ms["render_fwd"] / 1e3, sms, clk)
        table["render_bwd_pixels"] = alu_roofline(E, OPS_BWD_FP32, OPS_BWD_MUFU,
                                                  stage_ms["render_bwd_pixels"] / 1e3, sms, clk)
    dom = max(table, key=lambda k: stage_ms[k])
    out = dict(table[dom])
    tr, tr_note = load_traffic(dom, workload_key) if workload_key else (None, "no workload key")
    out.update({"kernel": dom, "traffic": tr, "traffic_note": tr_note,
                "peak_source": (f"{peaks['source']} HBM copy (burst)" if out["bound"] == "hbm" else
                                f"{sms} SMs x (128 FP32 | 16 MUFU) per clock x {clk:g} MHz"),
                "sms": sms, "work_counts": work, "per_stage": table})
    return out


# ---------------------------------------------------------------------------
# CPU oracle baseline: full iterations of the same workload
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OracleStep:
    """One oracle iteration of the workload: FP64 forward render of one
    1280x720 view of the whole scene, L1 loss gradient, analytic backward,
    Adam over every parameter.  The target is a seeded uniform image (the
    work does not depend on its values)."""

    def __init__(self, n, seed=SEED_SCENE):
        import oracle  # noqa: F401  (builds the oracle if needed)
        from paper_2607_14481_b300 import synth
        self.sc = synth.box_scene(n, seed)
        self.cams = synth.forward_trajectory(N_POSES, SEED_TRAJ)
        g = np.random.default_rng(SEED_TARGET)
        self.target = g.random((3, 720, 1280))
        self.p = np.concatenate([np.asarray(getattr(self.sc, a), np.float64).ravel()
                                 for a in ("means", "log_scales", "quats", "opa_logits", "sh")])
        self.m = np.zeros_like(self.p)
        self.v = np.zeros_like(self.p)
        self.t = 0

    def __call__(self, k):
        import oracle
        cam = [self.cams[k % len(self.cams)]]
        out = oracle.render(self.sc, cam)
        _, dimg = oracle.l1_loss(out["image"], [self.target])
        g = oracle.backward(self.sc, cam, dimg)
        gg = np.concatenate([g[a].ravel() for a in ("means", "log_scales", "quats", "opa_logits", "sh")])
        self.t += 1
        oracle.adam(self.p, gg, self.m, self.v, 1e-3, self.t)


def cpu_baseline(n):
    """The FP64 oracle as it stands timed on full iterations of the workload
    (1M Gaussians, one 1280x720 view, fwd + bwd + Adam) on this host: one
    iteration with every core (OpenMP over Gaussians and tiles; the result
    does not depend on the thread count) and one single-threaded."""
    import oracle
    step = OracleStep(n)
    cores = host_cores()
    before = oracle.get_threads()
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    step(50)
    t_all = time.perf_counter() - t0
    oracle.set_threads(1)
    t0 = time.perf_counter()
    step(51)
    t_one = time.perf_counter() - t0
    oracle.set_threads(before)
    return {"value": 1.0 / t_all, "unit": "iters/s", "cores": cores, "threads": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "seconds": t_all,
            "sample": f"one full iteration (fwd + bwd + Adam) of {n} Gaussians SH3 on one 1280x720 view "
                      f"(pose 50), FP64, {cores} threads; no scaling",
            "single_thread": {"value": 1.0 / t_one, "unit": "iters/s", "seconds": t_one, "threads": 1,
                              "sample": "one full iteration (pose 51), 1 thread"}}


def run_reference(args, ws, rank):
    """The oracle as the reference arm: each step one full iteration of the
    workload on every host core (rank 0 only)."""
    if rank != 0:
        return None, rank
    import oracle
    step = OracleStep(args.n)
    cores = host_cores()
    oracle.set_threads(cores)
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    el = time.perf_counter() - t0
    value = args.steps / el
    sample = (f"per step: one full fwd+bwd+Adam iteration of the FP64 oracle on all {args.n} Gaussians over "
              f"one 1280x720 view, {cores} threads; no scaling")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.n, ws),
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "threads": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
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
    if args.lod_only:
        import torch
        print(json.dumps({"lod": run_lod(torch.device("cuda", 0))}), flush=True)
        return
    if args.ba_only:
        import torch
        out = run_local_ba(torch.device("cuda", 0), cpu=not args.no_cpu_baseline)
        print(json.dumps({"local_ba": out}), flush=True)
        return
    if args.batched_only:
        import torch
        from paper_2607_14481_b300 import build, synth
        build.build()
        torch.cuda.set_device(0)
        out = run_batched(args.n, torch.device("cuda", 0), synth.loop_views(16, SEED_TRAJ + 1), args.steps,
                          args.warmup, 1, 0, fused_schedule=args.fused_schedule)
        print(json.dumps({"batched": out}), flush=True)
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
