#!/usr/bin/env python
"""Benchmark of the fused image-graph path on GB300.

Default workload (one JSON line on rank 0): the edge graph
Gaussian3x3 -> Sobel3x3 -> Magnitude -> Threshold(100) + Phase on 1920x1080
U8 frames (seeded rectangles + sigma-10 noise, BORDER_REPLICATE).  One step
processes a batch of --frames frames resident in HBM with one persistent fused
launch (hvxProcessGraphBatch, replayed from a captured CUDA graph).  The batch
(--frames x 6.2 MB of external bytes) is larger than L2, so no flush is needed.

The line reports: fused Mpix/s (value); the unfused one-launch-per-node form
on the same frames; the HBM roofline of the fused kernel on external bytes; an
end-to-end number with host<->device copies in the timed region; the other
workloads under "configs" (Gaussian3x3 on one 640x480 image per launch, the
Harris graph on 4096x2160, 256 images of uneven sizes in one launch, batched
Gaussian3x3 on 1080p frames), each with its own timing, roofline and clocks;
serving (Poisson arrivals of a Gaussian / edge / Harris mix) with p50 / p99
latency against one-request-at-a-time unfused serving, at 2000 req/s and at
saturation; the CPU oracle timed on the host (cpu_baseline), whose outputs on
the sampled frames are also compared with the GPU's (parity); SM clocks
sampled during each timed region.

--impl reference times the CPU oracle on the same metric (the reference arm).
--workload gauss | harris | batch | serve measure the other workloads:
  gauss   Gaussian3x3 on one 640x480 U8 image per step (launch latency bound)
  gauss-batch  Gaussian3x3 on --frames 1920x1080 frames per step, one launch
  harris  Harris graph on 4096x2160 U8, BORDER_UNDEFINED, 16 frames per step
  batch   256 images of uneven sizes (w 320..3840, h 240..2160) through the
          edge graph in one autotuned persistent launch, vs 256 unfused runs
  serve   Poisson 2000 req/s, 50/30/20 Gaussian/edge/Harris, sizes
          640x480 .. 7680x4320, 40 GB budget, fused vs one-at-a-time unfused
  morph   Dilate3x3 / Erode3x3 / Median3x3 / AbsDiff / Threshold / And graph
          on 1920x1080 frames (staged-tile executor), fused vs unfused
  apps    the nine applications of the paper's evaluation (Gauss .. Tomasi)
          on 1920x1080 frames, fused vs unfused

Multi-GPU (one rank per GPU, launched by torch.distributed.run; a bare
`--gpus N` with N > 1 re-launches itself that way): replicas only -- every
rank runs the same per-GPU batch on its own frames; value = all frames / max
rank time.
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
METRIC = "fused-graph Mpix/s (edge graph 1920x1080)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--workload", default="edge",
                    choices=["edge", "gauss", "gauss-batch", "harris", "batch", "serve",
                             "morph", "apps"])
    ap.add_argument("--serve-seconds", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="edge workload: skip the other workloads' sub-results")
    ap.add_argument("--e2e-streams", type=int, default=2,
                    help="edge workload: streams the end-to-end calls rotate over")
    ap.add_argument("--e2e-chunks", type=int, default=2,
                    help="edge workload: hvxScheduleGraphBatchHost calls per step (each "
                         "call pipelines its frames' copies and kernels internally)")
    ap.add_argument("--apps", default=None,
                    help="apps workload: comma-separated subset (e.g. Gauss,Tomasi)")
    ap.add_argument("--codegen", default="auto", choices=["auto", "only"],
                    help="apps workload: 'only' runs generated kernels in place of the "
                         "hand-written corner kernel (HVX_CODEGEN_ONLY), to compare them")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons in the timed region."""

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
        for t, ln in self.lines:
            if not t0 <= t <= t1:
                continue
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


EDGE_SOURCES = ["kernels_edge.cu", "device_common.cuh", "kernel_params.h", "phase_table.h",
                "launchers.h", "point_math.cuh", "reduce_math.cuh"]


def kernel_source_hash(files=EDGE_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2008_11476_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


EDGE_KERNEL = "edge_batch_kernel<MASK_PHASE>"
HARRIS_SOURCES = ["kernels_harris.cu", "device_common.cuh", "kernel_params.h", "launchers.h",
                  "point_math.cuh"]
HARRIS_KERNEL = "harris_fast_batch_kernel<HARRIS>"
KERNEL_SOURCES = {EDGE_KERNEL: EDGE_SOURCES, HARRIS_KERNEL: HARRIS_SOURCES}


def recorded_counters(kernel: str, frames: int):
    """The committed ncu record of `kernel` (profiles/dram_traffic.json):
    DRAM bytes and thread-instructions per pixel of one launch of `frames`
    frames, or None when the kernel's sources changed since the counters were
    taken or the launch size differs."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("frames") != frames or \
            rec.get("source_sha256") != kernel_source_hash(KERNEL_SOURCES[kernel]):
        return None
    return rec


def recorded_traffic(kernel: str, frames: int):
    rec = recorded_counters(kernel, frames)
    return None if rec is None else int(rec["dram_read_bytes"] + rec["dram_write_bytes"])


def recorded_instr_per_px(kernel: str, frames: int):
    """Thread-instructions per output pixel (ncu smsp__inst_executed.sum x 32
    / pixels of the launch), from the same hash-checked record."""
    rec = recorded_counters(kernel, frames)
    if rec is None or not rec.get("warp_instructions") or not rec.get("pixels"):
        return None
    return round(32.0 * rec["warp_instructions"] / rec["pixels"], 1)


def issue_roofline(mpix_s, instr_per_px, clocks):
    """Instruction-issue roofline of a kernel bound by issue: achieved
    thread-instructions/s against 152 SMs x 4 schedulers x 32 lanes x clock."""
    if instr_per_px is None:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = 152 * 4 * 32 * mhz * 1e6 / 1e12
    ach = mpix_s * 1e6 * instr_per_px / 1e12
    return {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2),
            "unit": "T thread-instr/s", "frac": round(ach / peak, 4),
            "instr_per_px": instr_per_px, "sm_mhz": mhz}


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
    """Largest value over the ranks (the slowest replica sets the time)."""
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, torch):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def time_steps(torch, fn, steps, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def timed_with_clocks(torch, fn, steps, stream, local):
    clk = ClockSampler(local).start()
    clk.mark_start()
    t = time_steps(torch, fn, steps, stream)
    clk.mark_end()
    clk.stop()
    return t, clk.summary()


def replica_time(world, torch, step, steps, timer):
    """Time `steps` calls of `step` with `timer` (returns (seconds, clocks)),
    bracketed by barriers; the replicas' time is the slowest rank's.
    Returns (max seconds over ranks, this rank's seconds, clocks)."""
    barrier(world, torch)
    t, clocks = timer(step, steps)
    barrier(world, torch)
    return reduce_max(t, world, torch), t, clocks


def replica_mpix_s(px_per_rank_step: float, world: int, steps: int, t_max: float) -> float:
    """Whole-job rate: the pixels every rank processed over the slowest time."""
    return px_per_rank_step * world * steps / t_max / 1e6


def rank_seeds(rank: int, n: int, base: int) -> list[int]:
    """Seeds of a rank's own frames (replicas process different frames)."""
    return [base + 1000 * rank + i for i in range(n)]


def hbm_roofline(ext_bytes: float, seconds_per_launch: float, kernel: str, traffic=None):
    peaks, src = measured_peaks()
    ach = ext_bytes / seconds_per_launch / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "traffic": traffic, "peak_source": src,
            "kernel": kernel, "algorithmic_bytes_per_launch": int(ext_bytes)}


def parity_of(pairs, rule="bit-exact"):
    """pairs: (gpu array, oracle array) of the sampled frames' outputs."""
    bad = int(sum(int(np.count_nonzero(a != b)) for a, b in pairs))
    n = int(sum(a.size for a, _ in pairs))
    return {"rule": rule, "outputs_compared": n, "mismatches": bad, "ok": bad == 0}


def library_env():
    """HVX_* tuning variables set for this run (they change kernel choices, so
    a line measured with any of them says so)."""
    return {k: v for k, v in sorted(os.environ.items()) if k.startswith("HVX_")}


def edge_config(args, world):
    cfg = {"workload": f"edge graph Gaussian3x3->Sobel3x3->Magnitude->Threshold(100)+Phase, "
                       f"1920x1080 U8, {args.frames} frames per step, BORDER_REPLICATE",
           "global_batch": args.frames * max(1, world), "frames_per_gpu": args.frames,
           "width": W, "height": H_, "parallelism": f"replicas x{world}",
           "l2": "inputs+outputs per step larger than L2 (no flush)"}
    if library_env():
        cfg["env"] = library_env()
    return cfg


# ---------------------------------------------------------------------------
# CPU oracle legs (the only places bench.py runs oracle/)

def cpu_oracle_edge(n_frames: int, threads: int = 1):
    """The CPU oracle (C, one frame per call) over n_frames 1080p edge-graph
    frames, on `threads` host threads (the C calls run without the GIL)."""
    import oracle as O
    from paper_2008_11476_gb300 import synth
    frames = [synth.rects_noise(W, H_, seed=2 + i) for i in range(min(n_frames, 4))]
    O.edge_graph(frames[0][:64, :64].copy())  # load the library outside the timing
    t0 = time.perf_counter()
    if threads <= 1:
        for i in range(n_frames):
            O.edge_graph(frames[i % len(frames)])
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda i: O.edge_graph(frames[i % len(frames)]), range(n_frames)))
    dt = time.perf_counter() - t0
    return n_frames * W * H_ / 1e6 / dt, dt


def reference_arm(args, world, rank):
    if rank != 0:
        return
    per_step = 4  # a bounded sample of the workload per step: 4 frames of the batch
    for _ in range(args.warmup):
        cpu_oracle_edge(1)
    steps = min(args.steps, 20)
    t0 = time.perf_counter()
    for _ in range(steps):
        cpu_oracle_edge(per_step)
    dt = time.perf_counter() - t0
    v = steps * per_step * W * H_ / 1e6 / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "Mpix/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(dt / steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": edge_config(args, world),
        "cpu_baseline": {"value": round(v, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} frames of 1920x1080 per step, {steps} steps"},
        "e2e": {"value": round(v, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def wrap_frames(ctx, torch, H, arrays, w, h, pitch):
    """Device tensors (n, h, pitch) holding `arrays` (cycled), wrapped as images."""
    n = len(arrays)
    t = torch.empty((n, h, pitch), dtype=torch.uint8, device="cuda")
    for i, a in enumerate(arrays):
        t[i, :, :w].copy_(torch.from_numpy(a))
    imgs = [H.hvxCreateImageFromHandle(ctx, w, h, H.HVX_DF_U8, t[i].data_ptr(), pitch)
            for i in range(n)]
    return t, imgs


def empty_frames(ctx, torch, H, n, w, h, pitch):
    t = torch.empty((n, h, pitch), dtype=torch.uint8, device="cuda")
    imgs = [H.hvxCreateImageFromHandle(ctx, w, h, H.HVX_DF_U8, t[i].data_ptr(), pitch)
            for i in range(n)]
    return t, imgs


def run_edge(args, world, rank, local, torch):
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth

    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    F = args.frames
    distinct = [synth.rects_noise(W, H_, seed=s) for s in rank_seeds(rank, min(F, 8), 2)]
    pitch = W  # 1920: a multiple of 16
    t_in, ins = wrap_frames(ctx, torch, H, [distinct[i % len(distinct)] for i in range(F)], W,
                            H_, pitch)
    t_ph, phs = empty_frames(ctx, torch, H, F, W, H_, pitch)
    t_mk, mks = empty_frames(ctx, torch, H, F, W, H_, pitch)
    torch.cuda.synchronize()
    fused = [PG.edge_graph(ctx, a, p, m) for a, p, m in zip(ins, phs, mks)]
    plain = [PG.edge_graph(ctx, a, p, m, fusion=False) for a, p, m in zip(ins, phs, mks)]
    assert PG.kernel_kinds(fused[0]) == ["fused_edge_tma"]
    n_plain_launch = H.hvxQueryGraph(plain[0], H.HVX_GRAPH_NUM_LAUNCHES)

    def step_fused():
        H.hvxProcessGraphBatch(fused, sh)

    def step_plain():
        for g in plain:
            H.hvxScheduleGraph(g, sh)

    step_fused()  # builds, autotunes and captures the batch launch
    for _ in range(args.warmup):
        step_fused()
    t_fused, _, clocks = replica_time(world, torch, step_fused, args.steps,
                                      _timer(torch, stream, local))
    gpu0 = (t_ph[0].cpu().numpy(), t_mk[0].cpu().numpy())

    plain_steps = max(2, min(args.steps, 40) // 4)
    for _ in range(2):
        step_plain()
    t_plain, _, _ = replica_time(world, torch, step_plain, plain_steps, _plain_timer(torch, stream))

    # end to end through the C ABI on host data: every step is two
    # hvxScheduleGraphBatchHost calls of 32 frames on two streams (copies in
    # from pinned host memory, the fused batch, both outputs back); each call
    # pipelines parts of its batch over two copy streams and the launch
    # stream so that copies in both directions overlap the kernels.  The host link (about 210 GB/s
    # in, 193 GB/s out, 341 GB/s both ways) bounds this number, not the kernel.
    h_in = torch.empty((F, H_, pitch), dtype=torch.uint8).pin_memory()
    h_in.copy_(t_in.cpu())
    h_ph = torch.empty_like(h_in).pin_memory()
    h_mk = torch.empty_like(h_in).pin_memory()
    chunk = max(1, F // args.e2e_chunks)
    chunks = [(i, min(F, i + chunk)) for i in range(0, F, chunk)]
    streams = [torch.cuda.Stream() for _ in range(max(1, args.e2e_streams))]
    sub = [fused[a:b] for a, b in chunks]
    copies = []
    for a, b in chunks:
        items = []
        for f in range(a, b):
            items += [(ins[f], h_in[f].data_ptr(), pitch, True),
                      (phs[f], h_ph[f].data_ptr(), pitch, False),
                      (mks[f], h_mk[f].data_ptr(), pitch, False)]
        copies.append(H.host_copies(items))

    def step_e2e():
        for i, gs in enumerate(sub):
            H.hvxScheduleGraphBatchHost(gs, copies[i], streams[i % len(streams)].cuda_stream)

    def time_e2e(steps):
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for st in streams:
            st.wait_event(start)
        for _ in range(steps):
            step_e2e()
        for st in streams:  # the timed region ends when the last result is on the host
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        end.record(stream)
        end.synchronize()
        return start.elapsed_time(end) / 1e3

    e2e_steps = max(4, min(args.steps, 40) // 2)
    time_e2e(2)
    barrier(world, torch)
    t_e2e = reduce_max(time_e2e(e2e_steps), world, torch)
    assert (h_mk[F - 1].numpy() == t_mk[F - 1].cpu().numpy()).all()
    H.hvxWaitBatch(ctx, sh)  # surfaces any device-side error

    serving = None
    if not args.no_serve and rank == 0:
        secs = args.serve_seconds if args.serve_seconds is not None else 1.5
        serving = serve_compare(ctx, H, PG, synth, secs, instances=3, sat_rate=200000.0,
                                sat_seconds=0.05)
    H.hvxReleaseContext(ctx)
    del t_in, t_ph, t_mk, h_in, h_ph, h_mk
    torch.cuda.empty_cache()
    configs = None
    if not args.no_configs:
        cpu = not args.no_cpu_baseline
        configs = {}
        for name, fn in (("config1_gauss_640x480", measure_gauss640),
                         ("config3_harris_4096x2160", measure_harris),
                         ("config4_batch256_uneven", measure_batch256),
                         ("gauss_batch_1080p", measure_gauss_batch)):
            configs[name] = fn(world, rank, local, torch, cpu)
            torch.cuda.empty_cache()
    if rank != 0:
        return
    mpix_step = F * W * H_ / 1e6 * world
    value = mpix_step * args.steps / t_fused
    plain_v = mpix_step * plain_steps / t_plain
    e2e_v = mpix_step * e2e_steps / t_e2e
    peaks, src = measured_peaks()
    ext_bytes = 3 * W * H_ * F  # input + phase + mask, per launch (per GPU)
    kernel_s = t_fused / args.steps
    achieved = ext_bytes / kernel_s / 1e9
    cpu = cpu_all = parity = None
    if not args.no_cpu_baseline:
        import oracle as O
        parity = parity_of(list(zip(gpu0, O.edge_graph(distinct[0]))))
        n = 48
        v_cpu, dt = cpu_oracle_edge(n)
        cpu = {"value": round(v_cpu, 3), "unit": "Mpix/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} frames of 1920x1080 through the C oracle, single thread "
                         f"({dt:.1f} s)"}
        nt = max(1, os.cpu_count() or 1)
        n_all = 6 * nt
        v_all, dt_all = cpu_oracle_edge(n_all, nt)
        cpu_all = {"value": round(v_all, 3), "unit": "Mpix/s", "cores": nt, "kind": "oracle",
                   "sample": f"{n_all} frames of 1920x1080 through the C oracle, one frame per "
                             f"call on {nt} threads ({dt_all:.1f} s)"}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_fused / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded rectangles + sigma 10 noise)",
        "config": edge_config(args, world),
        "unfused": {"value": round(plain_v, 1), "unit": "Mpix/s",
                    "launches_per_frame": n_plain_launch,
                    "ms_per_step": round(t_plain / plain_steps * 1e3, 4)},
        "fused_over_unfused": round(value / plain_v, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                     "frac": round(achieved / peaks.get("hbm_gbs", 6800.0), 4),
                     "traffic": recorded_traffic(EDGE_KERNEL, F),
                     "peak_source": src, "kernel": "edge_batch_kernel",
                     "algorithmic_bytes_per_launch": ext_bytes,
                     # the bound that holds: instruction issue (the kernel's
                     # instructions per pixel from its hash-checked ncu
                     # record, times the live pixel rate, against 152 SMs x 4
                     # schedulers x 32 lanes x the sampled SM clock)
                     "issue": issue_roofline(value / world,
                                             recorded_instr_per_px(EDGE_KERNEL, F), clocks)},
        "e2e": {"value": round(e2e_v, 1), "unit": "Mpix/s",
                "h2d_bytes_per_step": int(F * H_ * pitch),
                "d2h_bytes_per_step": int(2 * F * H_ * pitch)},
        "configs": configs,
        "serving": serving,
        "gpu_launches": args.steps,
        "parity": parity,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
SERVE_SIZES = [(640, 480), (1920, 1080), (3840, 2160), (7680, 4320)]
SERVE_KINDS = ["gaussian", "edge", "harris"]


def build_serve_pool(ctx, H, PG, synth, fused: bool, instances: int):
    """`instances` resident graphs per (kind, size), each with its own images."""
    pool = {}
    base = {s: synth.uniform_u8(s[0], s[1], seed=5 + i) for i, s in enumerate(SERVE_SIZES)}
    for k, kind in enumerate(SERVE_KINDS):
        for si, (w, h) in enumerate(SERVE_SIZES):
            lst = []
            for _ in range(instances):
                inp = PG.upload(ctx, base[(w, h)], H.HVX_DF_U8)
                if kind == "gaussian":
                    g = PG.gaussian_graph(ctx, inp, PG.empty(ctx, w, h, H.HVX_DF_U8), fusion=fused)
                elif kind == "edge":
                    g = PG.edge_graph(ctx, inp, PG.empty(ctx, w, h, H.HVX_DF_U8),
                                      PG.empty(ctx, w, h, H.HVX_DF_U8), fusion=fused)
                else:
                    g = PG.harris_graph(ctx, inp, PG.empty(ctx, w, h, H.HVX_DF_U8), fusion=fused)
                lst.append(g)
            pool[(k, si)] = lst
    return pool


def serve_run(H, synth, pool, srv, seconds: float, rate: float, seed: int):
    """Poisson arrivals at `rate` for `seconds`: at each wake-up of the
    submitting loop, every request whose arrival time has passed is submitted
    in one hvxServerSubmitMany call (so offered rates above what one call per
    request allows are still offered on time).  Latency runs from submission
    to completion; Mpix/s is the completed work over the time from the first
    submission to the last completion."""
    n = max(1, int(rate * seconds))
    arrivals = synth.poisson_arrivals(rate, n, seed)
    kinds = synth.choice(seed, 13, n, [0.5, 0.3, 0.2])
    sizes = synth.choice(seed, 14, n, [0.25] * 4)
    rr = {}
    # warm-up: every graph once
    for lst in pool.values():
        for g in lst:
            H.hvxServerWait(srv, H.hvxServerSubmit(srv, g))
    H.hvxServerResetStats(srv)
    order = []
    for i in range(n):
        key = (int(kinds[i]), int(sizes[i]))
        j = rr.get(key, 0)
        rr[key] = j + 1
        lst = pool[key]
        order.append(lst[j % len(lst)])
    tickets = []
    i = 0
    t0 = time.perf_counter()
    while i < n:
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            if arrivals[i] - now > 0.002:
                time.sleep(arrivals[i] - now - 0.001)
            continue
        k = i
        while k < n and arrivals[k] <= now:
            k += 1
        tickets += H.hvxServerSubmitMany(srv, order[i:k])
        i = k
    fails = 0
    for t in tickets:
        st, _ = H.hvxServerWait(srv, t)
        fails += st != H.HVX_SUCCESS
    elapsed = time.perf_counter() - t0
    st = H.hvxServerStats(srv)
    return {"requests": n, "failed": fails, "p50_ms": round(st["p50_ms"], 4),
            "p99_ms": round(st["p99_ms"], 4), "mean_ms": round(st["mean_ms"], 4),
            "max_ms": round(st["max_ms"], 3),
            "queue_wait_p99_ms": round(st["wait_p99_ms"], 4),
            "queue_wait_max_ms": round(st["wait_max_ms"], 3),
            "mpix_per_s": round(st["mpix_completed"] / elapsed, 1),
            "max_in_flight": int(st["max_in_flight"]),
            "offered_req_per_s": rate, "achieved_req_per_s": round(n / elapsed, 1),
            "seconds": round(elapsed, 3)}


SERVE_WORKLOAD = ("Poisson arrivals, 50/30/20 Gaussian3x3/edge/Harris graphs, sizes "
                  "640x480/1920x1080/3840x2160/7680x4320 uniform, 40 GB budget, uniform-byte "
                  "inputs")


def serve_compare(ctx, H, PG, synth, seconds, instances=4, rate=2000.0, sat_rate=None,
                  sat_seconds=0.05):
    """Fused continuous serving (16 slots, 8 streams) against one request at a
    time on unfused graphs, at `rate`, and when sat_rate is given, both at
    an offered rate above either's capacity (saturation)."""
    budget = 40 << 30
    fused_pool = build_serve_pool(ctx, H, PG, synth, True, instances)
    plain_pool = build_serve_pool(ctx, H, PG, synth, False, instances)
    out = {"workload": SERVE_WORKLOAD, "budget_bytes": budget, "slots": 16, "streams": 8}
    runs = [("fused_continuous", fused_pool, 16, 8), ("unfused_one_at_a_time", plain_pool, 1, 1)]
    for name, pool, slots, nst in runs:
        srv = H.hvxCreateServer(ctx, budget, slots, nst)
        out[name] = serve_run(H, synth, pool, srv, seconds, rate, seed=5)
        H.hvxReleaseServer(srv)
    if sat_rate:
        sat = {"offered_req_per_s": sat_rate,
               "note": "offered load above both forms' capacity: Mpix/s is what each "
                       "form sustains; latency includes the queueing"}
        for name, pool, slots, nst in runs:
            srv = H.hvxCreateServer(ctx, budget, slots, nst)
            sat[name] = serve_run(H, synth, pool, srv, sat_seconds, sat_rate, seed=8)
            H.hvxReleaseServer(srv)
        sat["fused_over_unfused_mpix"] = round(sat["fused_continuous"]["mpix_per_s"] /
                                               sat["unfused_one_at_a_time"]["mpix_per_s"], 2)
        out["saturation"] = sat
    out["p99_unfused_over_fused"] = round(out["unfused_one_at_a_time"]["p99_ms"] /
                                          max(out["fused_continuous"]["p99_ms"], 1e-9), 2)
    for pool in (fused_pool, plain_pool):
        for lst in pool.values():
            for g in lst:
                H.hvxReleaseGraph(g)
    return out


def _timer(torch, stream, local):
    return lambda f, n: timed_with_clocks(torch, f, n, stream, local)


def _plain_timer(torch, stream):
    return lambda f, n: (time_steps(torch, f, n, stream), None)


def _oracle_timed(fn, min_s=0.0):
    """Run the oracle call fn() once (or until min_s seconds passed); returns
    (last result, runs, seconds)."""
    t0 = time.perf_counter()
    runs = 0
    while True:
        out = fn()
        runs += 1
        if time.perf_counter() - t0 >= min_s:
            break
    return out, runs, time.perf_counter() - t0


def measure_gauss640(world, rank, local, torch, cpu, steps=2000, warmup=50):
    """Config 1: Gaussian3x3 on one 640x480 U8 image per launch.  400 images
    (246 MB of inputs and outputs, larger than L2) are cycled, so every launch
    reads an image that left L2 since its previous use."""
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    w, h, n_img = 640, 480, 400
    seed = rank_seeds(rank, 1, 1)[0]
    img = synth.uniform_u8(w, h, seed=seed)
    t_in, ins = wrap_frames(ctx, torch, H, [img] * n_img, w, h, w)
    t_out, outs = empty_frames(ctx, torch, H, n_img, w, h, w)
    graphs = [PG.gaussian_graph(ctx, a, o) for a, o in zip(ins, outs)]
    assert PG.kernel_kinds(graphs[0]) == ["gaussian3x3_tma"]
    it = [0]

    def step():
        H.hvxScheduleGraph(graphs[it[0] % n_img], sh)
        it[0] += 1

    for _ in range(warmup):
        step()
    t, _, clocks = replica_time(world, torch, step, steps, _timer(torch, stream, local))
    H.hvxWaitBatch(ctx, sh)
    gpu = t_out[0].cpu().numpy()
    H.hvxReleaseContext(ctx)
    per = t / steps
    r = {"workload": "Gaussian3x3 on one 640x480 U8 image per launch (uniform bytes 0-255, "
                     "seed 1), BORDER_REPLICATE, OpenVX truncating /16; launches back to back "
                     "on one stream over 400 image buffers",
         "value": round(replica_mpix_s(w * h, world, steps, t), 1), "unit": "Mpix/s",
         "us_per_launch": round(per * 1e6, 3), "steps": steps,
         "roofline": hbm_roofline(2 * w * h, per, "gauss_kernel"),
         "bound_note": "launch latency: 0.6 MB per launch would take 0.1 us at the HBM peak",
         "l2": "400 distinct image buffers cycled (246 MB, larger than L2)",
         "gpu_launches": steps, "clocks": clocks}
    if cpu and rank == 0:
        import oracle as O
        ref, runs, dt = _oracle_timed(lambda: O.gaussian3x3(img).data, 0.3)
        r["cpu_baseline"] = {"value": round(runs * w * h / 1e6 / dt, 3), "unit": "Mpix/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"{runs} runs of the 640x480 image, single thread"}
        r["parity"] = parity_of([(gpu, ref)])
    return r


def measure_gauss_batch(world, rank, local, torch, cpu, F=64, steps=40, warmup=5):
    """Gaussian3x3 alone on F 1920x1080 frames per step, one batched launch:
    the HBM roofline of the Gaussian kernel (2 B/px)."""
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    distinct = [synth.uniform_u8(W, H_, seed=s) for s in rank_seeds(rank, min(F, 8), 1)]
    t_in, ins = wrap_frames(ctx, torch, H, [distinct[i % len(distinct)] for i in range(F)], W, H_, W)
    t_o, outs = empty_frames(ctx, torch, H, F, W, H_, W)
    graphs = [PG.gaussian_graph(ctx, a, o) for a, o in zip(ins, outs)]
    assert PG.kernel_kinds(graphs[0]) == ["gaussian3x3_tma"]

    def step():
        H.hvxProcessGraphBatch(graphs, sh)

    step()
    for _ in range(warmup):
        step()
    t, _, clocks = replica_time(world, torch, step, steps, _timer(torch, stream, local))
    H.hvxWaitBatch(ctx, sh)
    gpu = t_o[0].cpu().numpy()
    H.hvxReleaseContext(ctx)
    per = t / steps
    r = {"workload": f"Gaussian3x3 on {F} 1920x1080 U8 frames per step (uniform bytes) in one "
                     "persistent launch, BORDER_REPLICATE",
         "value": round(replica_mpix_s(W * H_ * F, world, steps, t), 1), "unit": "Mpix/s",
         "ms_per_step": round(per * 1e3, 4), "steps": steps,
         "roofline": hbm_roofline(2 * W * H_ * F, per, "gauss_batch_kernel"),
         "l2": "inputs + outputs per step (265 MB) larger than L2",
         "gpu_launches": steps, "clocks": clocks}
    if cpu and rank == 0:
        import oracle as O
        ref, runs, dt = _oracle_timed(lambda: O.gaussian3x3(distinct[0]).data)
        r["cpu_baseline"] = {"value": round(runs * W * H_ / 1e6 / dt, 3), "unit": "Mpix/s",
                             "cores": 1, "kind": "oracle", "sample": "1 frame, single thread"}
        r["parity"] = parity_of([(gpu, ref)])
    return r


def measure_harris(world, rank, local, torch, cpu, steps=5, warmup=3, codegen="auto"):
    """Config 3: the Harris graph on 16 4096x2160 frames per step, fused: one
    batched launch for all 16 (the value) and one launch per frame; the
    unfused one-launch-per-node form (9 launches per frame) on the same
    frames."""
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    w, h, F = 4096, 2160, 16
    distinct = [synth.rects_noise(w, h, seed=s) for s in rank_seeds(rank, 4, 3)]
    t_in, ins = wrap_frames(ctx, torch, H, [distinct[i % 4] for i in range(F)], w, h, w)
    t_mk, mks = empty_frames(ctx, torch, H, F, w, h, w)
    fused = [PG.harris_graph(ctx, a, m) for a, m in zip(ins, mks)]
    if codegen == "only":
        for g in fused:
            H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
            H.hvxVerifyGraph(g)
    plain = [PG.harris_graph(ctx, a, m, fusion=False) for a, m in zip(ins, mks)]
    if codegen != "only":
        assert PG.kernel_kinds(fused[0]) == ["fused_harris_tma"]

    def step_fused():
        for gr in fused:
            H.hvxScheduleGraph(gr, sh)

    def step_batch():
        H.hvxProcessGraphBatch(fused, sh)

    def step_plain():
        for gr in plain:
            H.hvxScheduleGraph(gr, sh)

    for _ in range(warmup):
        step_fused()
        step_batch()
    t, _, clocks = replica_time(world, torch, step_fused, steps, _timer(torch, stream, local))
    tb, _, clocks_b = replica_time(world, torch, step_batch, steps, _timer(torch, stream, local))
    step_fused()  # frame outputs from the per-frame kernel for the parity check
    H.hvxWaitGraph(fused[-1])
    gpu = t_mk[0].cpu().numpy()
    step_plain()
    tp, _, _ = replica_time(world, torch, step_plain, 2, _plain_timer(torch, stream))
    H.hvxWaitGraph(plain[-1])
    n_plain = H.hvxQueryGraph(plain[0], H.HVX_GRAPH_NUM_LAUNCHES)
    H.hvxReleaseContext(ctx)
    px = w * h * F
    r = {"workload": "Harris graph Sobel3x3 -> gx^2, gy^2, gx*gy -> 5x5 window sums -> "
                     "response det - (1/25) trace^2 -> Threshold(1e6) -> U8 mask; 4096x2160 U8 "
                     "(seeded rectangles + sigma 10 noise), BORDER_UNDEFINED, 16 frames per "
                     "step in one fused launch (hvxProcessGraphBatch)",
         "value": round(replica_mpix_s(px, world, steps, tb), 1), "unit": "Mpix/s",
         "ms_per_step": round(tb / steps * 1e3, 4), "steps": steps,
         "roofline": dict(hbm_roofline(2 * px, tb / steps, "harris_fast_batch_kernel",
                                       traffic=recorded_traffic(HARRIS_KERNEL, F)),
                          issue=issue_roofline(px * steps / tb / 1e6,
                                               recorded_instr_per_px(HARRIS_KERNEL, F),
                                               clocks_b)),
         "one_launch_per_frame": {"value": round(replica_mpix_s(px, world, steps, t), 1),
                                  "unit": "Mpix/s", "ms_per_step": round(t / steps * 1e3, 4),
                                  "roofline": hbm_roofline(2 * w * h, t / steps / F,
                                                           "harris_fast_kernel"),
                                  "gpu_launches": steps * F, "clocks": clocks},
         "unfused": {"value": round(replica_mpix_s(px, world, 2, tp), 1), "unit": "Mpix/s",
                     "launches_per_frame": n_plain},
         "l2": "16 frame buffers per step (283 MB), larger than L2",
         "codegen": codegen, "gpu_launches": steps, "clocks": clocks_b}
    r["fused_over_unfused"] = round(r["value"] / r["unfused"]["value"], 2)
    if cpu and rank == 0:
        import oracle as O
        (ref, _), runs, dt = _oracle_timed(lambda: O.harris_graph(distinct[0]))
        r["cpu_baseline"] = {"value": round(runs * w * h / 1e6 / dt, 3), "unit": "Mpix/s",
                             "cores": 1, "kind": "oracle",
                             "sample": "1 frame of 4096x2160, single thread"}
        r["parity"] = parity_of([(gpu, ref)])
    return r


def measure_batch256(world, rank, local, torch, cpu, steps=10, warmup=3):
    """Config 4: 256 U8 images of seeded uneven sizes through the edge graph in
    one persistent fused launch (replayed from a captured CUDA graph, grid
    chosen by the autotuner); against one fused launch per image and 256
    unfused runs of 5 launches each."""
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    sizes = synth.batch_sizes(256, seed=4)
    bases = [synth.rects_noise(3840, 2160, seed=s) for s in rank_seeds(rank, 4, 40)]
    offs = synth.randint(4, 20, 512, 0, 1 << 20)
    graphs, plain, keep, crops, outs = [], [], [], [], []
    for i, (w, h) in enumerate(sizes):
        b = bases[i % 4]
        ox = int(offs[2 * i]) % (3840 - w + 1)
        oy = int(offs[2 * i + 1]) % (2160 - h + 1)
        crop = np.ascontiguousarray(b[oy:oy + h, ox:ox + w])
        pitch = (w + 15) // 16 * 16
        t_in, (a,) = wrap_frames(ctx, torch, H, [crop], w, h, pitch)
        t_o, (p, m) = empty_frames(ctx, torch, H, 2, w, h, pitch)
        keep += [t_in, t_o]
        crops.append(crop)
        outs.append(t_o)
        graphs.append(PG.edge_graph(ctx, a, p, m))
        plain.append(PG.edge_graph(ctx, a, p, m, fusion=False))
    mpix = sum(w * h for w, h in sizes) / 1e6

    def step_fused():
        H.hvxProcessGraphBatch(graphs, sh)

    def step_per_image():
        for g in graphs:
            H.hvxScheduleGraph(g, sh)

    def step_plain():
        for g in plain:
            H.hvxScheduleGraph(g, sh)

    # first with every tile 128 x 120 (only the grid tuned), then re-verified
    # (a new plan, so a new batch entry) with the tile shape tuned per size class
    prev = os.environ.get("HVX_AUTOTUNE")
    os.environ["HVX_AUTOTUNE"] = "grid"
    try:
        step_fused()
        for _ in range(warmup):
            step_fused()
        t_fixed, _, clocks_fixed = replica_time(world, torch, step_fused, steps,
                                                _timer(torch, stream, local))
    finally:
        if prev is None:
            del os.environ["HVX_AUTOTUNE"]
        else:
            os.environ["HVX_AUTOTUNE"] = prev
    H.hvxWaitBatch(ctx, sh)
    for g in graphs:
        H.hvxVerifyGraph(g)
    t_build = time.perf_counter()
    step_fused()  # build + shape and grid autotune + capture
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    for _ in range(warmup):
        step_fused()
    t, _, clocks = replica_time(world, torch, step_fused, steps, _timer(torch, stream, local))
    H.hvxWaitBatch(ctx, sh)
    tuned_rows, tuned_grid = H.hvxQueryBatch(graphs)
    by_class = {}
    for (w, h), r in zip(sizes, tuned_rows):
        k = "h<480" if h < 480 else "480<=h<1080" if h < 1080 else "h>=1080"
        by_class.setdefault(k, {"tile": f"128x{8 * r}", "images": 0})
        by_class[k]["images"] += 1
    # sampled images for the parity check: the first and the smallest
    pick = sorted({0, int(np.argmin([w * h for w, h in sizes]))})
    gpu = {i: (outs[i][0][:, :sizes[i][0]].cpu().numpy(), outs[i][1][:, :sizes[i][0]].cpu().numpy())
           for i in pick}
    step_per_image()
    ti, _, _ = replica_time(world, torch, step_per_image, 3, _plain_timer(torch, stream))
    step_plain()
    tp, _, _ = replica_time(world, torch, step_plain, 3, _plain_timer(torch, stream))
    H.hvxWaitBatch(ctx, sh)
    H.hvxReleaseContext(ctx)
    value = replica_mpix_s(mpix * 1e6, world, steps, t)
    unf = replica_mpix_s(mpix * 1e6, world, 3, tp)
    r = {"workload": "256 U8 images, w~U{320..3840}, h~U{240..2160} (seed 4; crops of seeded "
                     f"rectangles + noise frames), {mpix:.1f} Mpix per step, edge graph "
                     "BORDER_REPLICATE, one persistent fused launch replayed from a CUDA graph",
         "value": round(value, 1), "unit": "Mpix/s", "ms_per_step": round(t / steps * 1e3, 4),
         "steps": steps,
         "roofline": hbm_roofline(3 * mpix * 1e6, t / steps, "edge_batch_kernel"),
         "per_image_fused_launches": {"value": round(replica_mpix_s(mpix * 1e6, world, 3, ti), 1),
                                      "unit": "Mpix/s", "launches_per_step": 256},
         "unfused_256_runs": {"value": round(unf, 1), "unit": "Mpix/s",
                              "launches_per_step": 256 * 5},
         "batched_over_unfused": round(value / unf, 2),
         "first_call_s": round(t_build, 3),
         "autotuned": {"tile_by_size_class": by_class, "grid": tuned_grid,
                       "note": "first call times each image-height class in its own launch "
                               "with 128x120 / 128x80 / 128x40 tiles, then the per-class "
                               "launches against one launch of every image at 128x120 (split "
                               "kept only if 2% faster), then 1..4 CTAs per SM"},
         "fixed_shape_128x120": {"value": round(replica_mpix_s(mpix * 1e6, world, steps,
                                                               t_fixed), 1),
                                 "unit": "Mpix/s", "ms_per_step": round(t_fixed / steps * 1e3, 4),
                                 "clocks": clocks_fixed},
         "l2": "larger than L2 (1.9 GB of external bytes per step)",
         "gpu_launches": steps, "clocks": clocks}
    if cpu and rank == 0:
        import oracle as O
        pairs, t_cpu, px_cpu = [], 0.0, 0
        for i in pick:
            (rp, rm), _, dt = _oracle_timed(lambda i=i: O.edge_graph(crops[i]))
            t_cpu += dt
            px_cpu += sizes[i][0] * sizes[i][1]
            pairs += [(gpu[i][0], rp), (gpu[i][1], rm)]
        r["cpu_baseline"] = {"value": round(px_cpu / 1e6 / t_cpu, 3), "unit": "Mpix/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"images {pick} of the batch, single thread"}
        r["parity"] = parity_of(pairs)
    return r


def _print_sub(rank, world, metric, r, **extra):
    if rank == 0:
        line = {"metric": metric, "n_gpus": world, "higher_is_better": True,
                "data": "synthetic", **extra, **r}
        print(json.dumps(line), flush=True)


def run_gauss(args, world, rank, local, torch):
    r = measure_gauss640(world, rank, local, torch, not args.no_cpu_baseline,
                         steps=max(args.steps, 400), warmup=max(args.warmup, 3))
    _print_sub(rank, world, "Gaussian3x3 640x480 Mpix/s (one image per launch)", r, dtype="u8")


def run_gauss_batch(args, world, rank, local, torch):
    r = measure_gauss_batch(world, rank, local, torch, not args.no_cpu_baseline, F=args.frames,
                            steps=args.steps, warmup=args.warmup)
    _print_sub(rank, world, "Gaussian3x3 Mpix/s (batched 1920x1080 frames)", r, dtype="u8")


def run_harris(args, world, rank, local, torch):
    r = measure_harris(world, rank, local, torch, not args.no_cpu_baseline,
                       steps=max(3, args.steps // 10), warmup=args.warmup, codegen=args.codegen)
    _print_sub(rank, world, "Harris graph 4096x2160 Mpix/s (fused)", r, dtype="u8/s32")


def run_batch(args, world, rank, local, torch):
    r = measure_batch256(world, rank, local, torch, not args.no_cpu_baseline,
                         steps=max(5, args.steps // 10), warmup=args.warmup)
    _print_sub(rank, world, "batched edge graph Mpix/s (256 uneven images, one launch)", r,
               dtype="u8")


def morph_graph(ctx, H, src, out, fusion=True):
    """Closing (Dilate3x3 -> Erode3x3), |closing - input| > 20, AND the input's
    Median3x3: six Table 2 nodes, BORDER_REPLICATE."""
    g = H.hvxCreateGraph(ctx)
    d, c, diff, mask, med = (H.hvxCreateVirtualImage(g) for _ in range(5))
    for n in (H.hvxDilate3x3Node(g, src, d), H.hvxErode3x3Node(g, d, c),
              H.hvxMedian3x3Node(g, src, med)):
        H.hvxSetNodeBorder(n, H.HVX_BORDER_REPLICATE, 0)
    H.hvxAbsDiffNode(g, c, src, diff)
    H.hvxThresholdNode(g, diff, H.HVX_THRESHOLD_BINARY, 20, 0, 255, 0, mask)
    H.hvxAndNode(g, med, mask, out)
    H.hvxSetGraphFusion(g, fusion)
    H.hvxVerifyGraph(g)
    return g


def run_morph(args, world, rank, local, torch):
    """Morphology graph (Dilate3x3, Erode3x3, Median3x3, AbsDiff, Threshold,
    And) on 1920x1080 frames, one launch per frame: the staged-tile executor."""
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    F = 16
    distinct = [synth.rects_noise(W, H_, seed=40 + i) for i in range(4)]
    t_in, ins = wrap_frames(ctx, torch, H, [distinct[i % 4] for i in range(F)], W, H_, W)
    t_o, outs = empty_frames(ctx, torch, H, F, W, H_, W)
    fused = [morph_graph(ctx, H, a, o) for a, o in zip(ins, outs)]
    plain = [morph_graph(ctx, H, a, o, fusion=False) for a, o in zip(ins, outs)]
    assert PG.kernel_kinds(fused[0]) == ["staged_tile"]

    def step_fused():
        for gr in fused:
            H.hvxScheduleGraph(gr, sh)

    def step_plain():
        for gr in plain:
            H.hvxScheduleGraph(gr, sh)

    for _ in range(args.warmup):
        step_fused()
    barrier(world, torch)
    steps = max(3, args.steps // 10)
    t, clocks = timed_with_clocks(torch, step_fused, steps, stream, local)
    t = reduce_max(t, world, torch)
    step_plain()
    tp = reduce_max(time_steps(torch, step_plain, 3, stream), world, torch)
    H.hvxWaitGraph(fused[-1])
    H.hvxReleaseContext(ctx)
    if rank == 0:
        peaks, src = measured_peaks()
        mp = W * H_ * F / 1e6
        ext = 2 * W * H_
        per_launch_s = t / steps / F
        print(json.dumps({
            "metric": "morphology graph 1920x1080 Mpix/s (fused)",
            "value": round(mp * steps / t * world, 1), "unit": "Mpix/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(t / steps * 1e3, 4),
            "higher_is_better": True, "dtype": "u8", "data": "synthetic (seeded rectangles + "
                                                                 "sigma 10 noise)",
            "config": {"workload": "Dilate3x3 -> Erode3x3 -> AbsDiff(input) -> Threshold(20), "
                                   "AND Median3x3(input); 1920x1080 U8, BORDER_REPLICATE, 16 "
                                   "frames per step (one launch each)",
                       "l2": "16 distinct frames per step, larger than L2",
                       "codegen": args.codegen},
            "unfused": {"value": round(mp * 3 / tp, 1), "unit": "Mpix/s", "launches_per_frame": 6},
            "roofline": {"bound": "hbm", "achieved": round(ext / per_launch_s / 1e9, 1),
                         "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": round(ext / per_launch_s / 1e9 / peaks.get("hbm_gbs", 6800), 4),
                         "peak_source": src, "kernel": "generic_kernel",
                         "algorithmic_bytes_per_launch": ext},
            "gpu_launches": steps * F, "clocks": clocks}), flush=True)


def run_apps(args, world, rank, local, torch):
    """The applications of the paper's evaluation (Section 6) on 1920x1080
    frames, one launch (or one launch per node, unfused) per frame: Mpix/s
    fused and unfused, the fused kernel, and the HBM fraction on external
    bytes."""
    from paper_2008_11476_gb300 import apps as A
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx = H.hvxCreateContext()
    F = 16
    distinct = [synth.rects_noise(W, H_, seed=50 + i) for i in range(4)]
    t_in, ins = wrap_frames(ctx, torch, H, [distinct[i % 4] for i in range(F)], W, H_, W)
    peaks, src = measured_peaks()
    bpp = {H.HVX_DF_U8: 1, H.HVX_DF_S16: 2}
    res = {}
    steps = max(3, args.steps // 20)
    wanted = set(args.apps.split(",")) if args.apps else None
    for name, build in A.APPS:
        if wanted and name not in wanted:
            continue
        fused, plain = [], []
        for a in ins:
            g, outs = build(ctx, a, W, H_, True)
            if args.codegen == "only":
                H.hvxSetGraphCodegen(g, H.HVX_CODEGEN_ONLY)
                H.hvxVerifyGraph(g)
            fused.append(g)
            g2, _ = build(ctx, a, W, H_, False)
            plain.append(g2)
        ext = W * H_ * (1 + sum(bpp[f] for _, _, f in outs))

        def run(gs):
            for gr in gs:
                H.hvxScheduleGraph(gr, sh)

        def batch():
            H.hvxProcessGraphBatch(fused, sh)

        for _ in range(args.warmup):
            run(fused)
            batch()
        run(plain)
        barrier(world, torch)
        tf = reduce_max(time_steps(torch, lambda: run(fused), steps, stream), world, torch)
        tb = reduce_max(time_steps(torch, batch, steps, stream), world, torch)
        tp = reduce_max(time_steps(torch, lambda: run(plain), steps, stream), world, torch)
        px = W * H_ * F * steps * world
        fv, bv, pv = px / tf / 1e6, px / tb / 1e6, px / tp / 1e6
        gen = H.hvxQueryGraph(fused[0], H.HVX_GRAPH_GENERATED_KERNELS)
        kind = "generated" if gen else PG.kernel_kinds(fused[0])[0]
        res[name] = {"batched_mpix_s": round(bv, 1), "fused_mpix_s": round(fv, 1),
                     "unfused_mpix_s": round(pv, 1), "speedup_batched_vs_unfused": round(bv / pv, 2),
                     "speedup_fused_vs_unfused": round(fv / pv, 2),
                     "kernel": kind,
                     # generated and corner kernels cover all frames in one launch
                     "batch_launches": 1 if kind in ("generated", "fused_harris_tma") else F,
                     "unfused_launches_per_frame": H.hvxQueryGraph(plain[0],
                                                                   H.HVX_GRAPH_NUM_LAUNCHES),
                     "external_bytes_per_px": ext // (W * H_),
                     "hbm_frac_batched": round(ext * F * steps / tb / 1e9 /
                                               peaks.get("hbm_gbs", 6800), 4)}
        H.hvxWaitGraph(fused[-1])
        for gr in fused + plain:
            H.hvxReleaseGraph(gr)
    H.hvxReleaseContext(ctx)
    if rank == 0:
        gm = float(np.exp(np.mean([np.log(v["batched_mpix_s"]) for v in res.values()])))
        gf = float(np.exp(np.mean([np.log(v["fused_mpix_s"]) for v in res.values()])))
        gu = float(np.exp(np.mean([np.log(v["unfused_mpix_s"]) for v in res.values()])))
        print(json.dumps({
            "metric": "paper application suite Mpix/s (1920x1080, geometric mean, fused, "
                      "16 frames per batch call)",
            "geomean_fused_one_call_per_frame": round(gf, 1),
            "geomean_unfused_one_call_per_frame": round(gu, 1),
            "value": round(gm, 1), "unit": "Mpix/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "u8/s16",
            "data": "synthetic (seeded rectangles + sigma 10 noise)",
            "config": {"workload": "Gauss, Laplacian, FChain, SobelX, EdgFig2, Sobel, Unsharp, "
                                   "Harris, Tomasi (Section 6) on 16 1920x1080 U8 frames per "
                                   "step: one hvxProcessGraphBatch call (one launch where the "
                                   "frames share a generated kernel), or one call per frame",
                       "l2": "16 distinct frames per step, larger than L2",
                       "codegen": args.codegen},
            "apps": res, "peak_source": src,
            "gpu_launches": steps * sum(v["batch_launches"] for v in res.values())}), flush=True)


def run_serve(args, world, rank, local, torch):
    from paper_2008_11476_gb300 import graphs as PG
    from paper_2008_11476_gb300 import hvx as H
    from paper_2008_11476_gb300 import synth
    ctx = H.hvxCreateContext()
    secs = args.serve_seconds if args.serve_seconds is not None else 5.0
    res = serve_compare(ctx, H, PG, synth, secs, instances=4, sat_rate=200000.0,
                        sat_seconds=0.05)
    # offered-rate sweep of the fused server up to saturation, and a 256 MB
    # budget run where admission waits for memory
    pool = build_serve_pool(ctx, H, PG, synth, True, 4)
    sweep = []
    for rate in (2000.0, 5000.0, 10000.0, 20000.0, 40000.0, 80000.0):
        srv = H.hvxCreateServer(ctx, 40 << 30, 16, 8)
        sweep.append(serve_run(H, synth, pool, srv, 0.5, rate, seed=6))
        H.hvxReleaseServer(srv)
    srv = H.hvxCreateServer(ctx, 256 << 20, 16, 8)
    small = serve_run(H, synth, pool, srv, 1.0, 2000.0, seed=7)
    H.hvxReleaseServer(srv)
    for lst in pool.values():
        for g in lst:
            H.hvxReleaseGraph(g)
    H.hvxReleaseContext(ctx)
    if rank == 0:
        f = res["fused_continuous"]
        print(json.dumps({"metric": "serving p50/p99 ms and Mpix/s", "value": f["p99_ms"],
                          "unit": "ms (p99)", "higher_is_better": False, "n_gpus": world,
                          "dtype": "u8", "data": "synthetic", "serving": res,
                          "rate_sweep_fused": sweep, "budget_256MB_fused": small}),
              flush=True)


def relaunch_replicas(n: int) -> int:
    """`--gpus N` (N > 1) run without a launcher: start N ranks of this same
    command with torch.distributed.run (one process per GPU, loopback
    rendezvous) and return their exit status."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={n}", "--master-addr=127.0.0.1", f"--master-port={port}",
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_replicas(args.gpus))
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    import torch
    if world > torch.cuda.device_count():
        sys.exit(f"bench.py: {world} ranks but {torch.cuda.device_count()} visible GPUs")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fn = {"edge": run_edge, "gauss": run_gauss, "gauss-batch": run_gauss_batch,
          "harris": run_harris, "batch": run_batch, "serve": run_serve,
          "morph": run_morph, "apps": run_apps}[args.workload]
    fn(args, world, rank, local, torch)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
