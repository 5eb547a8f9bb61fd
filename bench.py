#!/usr/bin/env python
"""Benchmark of the fused image-graph path on GB300.

Default workload (one JSON line on rank 0): the edge graph
Gaussian3x3 -> Sobel3x3 -> Magnitude -> Threshold(100) + Phase on 1920x1080
U8 frames (seeded rectangles + sigma-10 noise, BORDER_REPLICATE).  One step
processes a batch of --frames frames resident in HBM with one persistent fused
launch (hvxProcessGraphBatch, replayed from a captured CUDA graph).  The batch
(--frames x 6.2 MB of external bytes) is larger than L2, so no flush is needed.

Reported: fused Mpix/s (value), the unfused one-launch-per-node form on the
same frames, the HBM roofline of the fused kernel on external bytes, an
end-to-end number with host<->device copies in the timed region, the CPU
oracle timed on the host (cpu_baseline), and SM clocks sampled during the
timed region.

--impl reference times the CPU oracle on the same metric (the reference arm).
--workload gauss | harris | serve measure the other workloads of the project
(Gaussian3x3 640x480, Harris 4096x2160, Poisson serving mix).

Multi-GPU (torchrun, one rank per GPU): replicas only -- every rank runs the
same per-GPU batch on its own frames; value = all frames / max rank time.
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

W, H_ = 1920, 1080


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--workload", default="edge", choices=["edge", "gauss", "harris", "serve"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []  # (arrival time, line)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)  # the sampler is running before the timed region opens
        except OSError:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()
        time.sleep(2.5 * self.interval_ms / 1000)  # the sample that covers the end

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = self.t0 or 0.0
        t1 = (self.t1 or 1e30) + 2.5 * self.interval_ms / 1000
        sel = [ln for (t, ln) in self.lines if t0 <= t <= t1]
        for ln in sel:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, torch):
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, torch):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
def cpu_oracle_edge(n_frames: int):
    """The CPU oracle (single-threaded C) over n_frames 1080p edge-graph frames."""
    import oracle as O
    from paper_2008_11476_gb300 import synth
    frames = [synth.rects_noise(W, H_, seed=2 + i) for i in range(min(n_frames, 4))]
    t0 = time.perf_counter()
    for i in range(n_frames):
        O.edge_graph(frames[i % len(frames)])
    dt = time.perf_counter() - t0
    return n_frames * W * H_ / 1e6 / dt, dt


def reference_arm(args, world, rank):
    if rank != 0:
        return
    # each step: a bounded sample of the workload (4 frames of the batch)
    per_step = 4
    for _ in range(args.warmup):
        cpu_oracle_edge(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_edge(per_step)
    dt = time.perf_counter() - t0
    mpix = args.steps * per_step * W * H_ / 1e6
    v = mpix / dt
    line = {
        "impl": "reference", "metric": "fused-graph Mpix/s (edge graph 1920x1080)",
        "value": round(v, 3), "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": edge_config(args),
        "cpu_baseline": {"value": round(v, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} frames of 1920x1080 per step"},
        "e2e": {"value": round(v, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def edge_config(args):
    return {"workload": f"edge graph Gaussian3x3->Sobel3x3->Magnitude->Threshold(100)+Phase, "
                        f"1920x1080 U8, {args.frames} frames per step, BORDER_REPLICATE",
            "global_batch": args.frames * max(1, args.gpus), "frames_per_gpu": args.frames,
            "width": W, "height": H_, "parallelism": f"replicas x{args.gpus}",
            "l2": "inputs+outputs per step larger than L2 (no flush)"}


# ---------------------------------------------------------------------------
def time_steps(torch, fn, steps, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def run_edge(args, world, rank, local, torch):
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    F = args.frames
    distinct = [synth.rects_noise(W, H_, seed=2 + 1000 * rank + i) for i in range(min(F, 8))]
    pitch = W  # 1920: a multiple of 16
    t_in = torch.empty((F, H_, pitch), dtype=torch.uint8, device="cuda")
    t_ph = torch.empty_like(t_in)
    t_mk = torch.empty_like(t_in)
    for i in range(F):
        t_in[i].copy_(torch.from_numpy(distinct[i % len(distinct)]))
    torch.cuda.synchronize()
    fused, plain = [], []
    for i in range(F):
        a = H.hvxCreateImageFromHandle(ctx, W, H_, H.HVX_DF_U8, t_in[i].data_ptr(), pitch)
        p = H.hvxCreateImageFromHandle(ctx, W, H_, H.HVX_DF_U8, t_ph[i].data_ptr(), pitch)
        m = H.hvxCreateImageFromHandle(ctx, W, H_, H.HVX_DF_U8, t_mk[i].data_ptr(), pitch)
        fused.append(PG.edge_graph(ctx, a, p, m))
        plain.append(PG.edge_graph(ctx, a, p, m, fusion=False))
    assert PG.kernel_kinds(fused[0]) == ["fused_edge_tma"]
    n_plain_launch = H.hvxQueryGraph(plain[0], H.HVX_GRAPH_NUM_LAUNCHES)

    def step_fused():
        H.hvxProcessGraphBatch(fused, sh)

    def step_plain():
        for g in plain:
            H.hvxScheduleGraph(g, sh)

    # correctness spot check of the timed configuration (sampled frame)
    step_fused()
    torch.cuda.synchronize()
    if rank == 0:
        import_ok = True
        try:
            import oracle as O
            rp, rm = O.edge_graph(distinct[0])
            assert (t_ph[0].cpu().numpy() == rp).all() and (t_mk[0].cpu().numpy() == rm).all()
        except ImportError:
            import_ok = False
        del import_ok

    for _ in range(args.warmup):
        step_fused()
    barrier(world, torch)
    clk = ClockSampler(local).start()
    clk.mark_start()
    t_fused = time_steps(torch, step_fused, args.steps, stream)
    clk.mark_end()
    clk.stop()
    barrier(world, torch)
    t_fused = reduce_max(t_fused, world, torch)

    # unfused one-launch-per-node form on the same frames (fewer steps)
    plain_steps = max(2, args.steps // 4)
    for _ in range(2):
        step_plain()
    barrier(world, torch)
    t_plain = time_steps(torch, step_plain, plain_steps, stream)
    t_plain = reduce_max(t_plain, world, torch)

    # end to end: pinned host frames in, outputs back, through the same C ABI call
    h_in = torch.empty((F, H_, pitch), dtype=torch.uint8).pin_memory()
    h_in.copy_(t_in.cpu())
    h_ph = torch.empty_like(h_in).pin_memory()
    h_mk = torch.empty_like(h_in).pin_memory()

    def step_e2e():
        t_in.copy_(h_in, non_blocking=True)
        H.hvxProcessGraphBatch(fused, sh)
        h_ph.copy_(t_ph, non_blocking=True)
        h_mk.copy_(t_mk, non_blocking=True)

    e2e_steps = max(2, args.steps // 4)
    step_e2e()
    barrier(world, torch)
    t_e2e = time_steps(torch, step_e2e, e2e_steps, stream)
    t_e2e = reduce_max(t_e2e, world, torch)

    H.hvxWaitBatch(ctx, sh)  # surfaces any device-side error

    if rank != 0:
        H.hvxReleaseContext(ctx)
        return
    mpix_step = F * W * H_ / 1e6 * world
    value = mpix_step * args.steps / t_fused
    plain_v = mpix_step * plain_steps / t_plain
    e2e_v = mpix_step * e2e_steps / t_e2e
    peaks, src = measured_peaks()
    ext_bytes = 3 * W * H_ * F  # input + phase + mask, per launch (per GPU)
    kernel_s = t_fused / args.steps
    achieved = ext_bytes / kernel_s / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        n = 48
        v_cpu, dt = cpu_oracle_edge(n)
        cpu = {"value": round(v_cpu, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} frames of 1920x1080 through the C oracle, single thread "
                         f"({dt:.1f} s)"}
    line = {
        "metric": "fused-graph Mpix/s (edge graph 1920x1080)",
        "value": round(value, 1), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_fused / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded rectangles + sigma 10 noise)", "config": edge_config(args),
        "unfused": {"value": round(plain_v, 1), "unit": "Mpix/s",
                    "launches_per_frame": n_plain_launch,
                    "ms_per_step": round(t_plain / plain_steps * 1e3, 4)},
        "fused_over_unfused": round(value / plain_v, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                     "frac": round(achieved / peaks.get("hbm_gbs", 6800.0), 4),
                     "traffic": None, "peak_source": src,
                     "kernel": "edge_batch_kernel",
                     "algorithmic_bytes_per_launch": ext_bytes},
        "e2e": {"value": round(e2e_v, 1), "unit": "Mpix/s",
                "h2d_bytes_per_step": int(F * H_ * pitch),
                "d2h_bytes_per_step": int(2 * F * H_ * pitch)},
        "gpu_launches": args.steps,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    H.hvxReleaseContext(ctx)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.workload == "edge":
        run_edge(args, world, rank, local, torch)
    else:
        raise SystemExit(f"workload {args.workload} is not available")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
