"""The multi-GPU form is replicas only (independent frames per rank, no data
path collective).  These CPU tests run bench.py's rank logic as two gloo
processes: timing is the max over ranks, and the reference arm prints from
rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    got = bench.reduce_max(1.5 + rank, w, torch)
    bench.barrier(w, torch)
    q.put((rank, got))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29731
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 2.5), (1, 2.5)]


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank0_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--gpus", "2"],
                         capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if rank == 0:
        assert len(lines) == 1
        d = json.loads(lines[0])
        assert d["impl"] == "reference" and d["unit"] == "Mpix/s" and d["value"] > 0
        assert d["cpu_baseline"]["kind"] == "oracle"
    else:
        assert lines == []


def _rank_path_worker(rank, world, port, q):
    """bench.py's replica timing with the GPU step replaced by a sleep: rank r
    takes (r + 1) x 10 ms per step."""
    import time

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def step():
        time.sleep(0.01 * (rank + 1))

    def timer(f, n):
        t0 = time.perf_counter()
        for _ in range(n):
            f()
        return time.perf_counter() - t0, {"sm_mhz": None}

    t_max, t_local, clocks = bench.replica_time(world, torch, step, 3, timer)
    v = bench.replica_mpix_s(1920 * 1080 * 64, world, 3, t_max)
    q.put((rank, bench.rank_seeds(rank, 8, 2), t_max, t_local, v))
    dist.destroy_process_group()


def test_edge_rank_path_over_two_gloo_ranks():
    """Each rank has its own frames (disjoint seeds); the time is the slowest
    rank's on every rank; the whole-job rate counts every rank's frames."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_path_worker, args=(r, 2, 29733, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, m0, l0, v0), (r1, s1, m1, l1, v1) = res
    assert not set(s0) & set(s1)
    assert m0 == m1 == max(l0, l1) and l1 > l0 >= 0.03
    assert v0 == v1 == pytest.approx(1920 * 1080 * 64 * 2 * 3 / m0 / 1e6)


def test_bare_multi_gpu_run_relaunches_itself():
    """`bench.py --gpus 2` without a launcher starts two ranks itself (here the
    reference arm, which needs no GPU): one JSON line, from rank 0."""
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--gpus", "2"],
                         capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
