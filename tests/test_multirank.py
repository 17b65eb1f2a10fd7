"""Host logic of the multi-rank benchmark on CPU: two ranks over gloo.

The render path does not shard (every rank renders its own cameras), so N GPUs run N replicas: each
rank takes its own camera order with a fixed number of frames, the job's time is the slowest
rank's (a MAX collective), and the reported throughput is every rank's pixels over that time.  The
reference arm runs on rank 0 only; the other ranks exit at once.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if ROOT not in sys.path:
            sys.path.insert(0, ROOT)
        import bench
        cpu = torch.device("cpu")
        slowest = bench.max_over_ranks(1.5 + rank, world, cpu)  # rank 1 is the slow one
        order = bench.replica_order(rank, 100, 8)
        torch.distributed.barrier()
        q.put((rank, slowest, order))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_own_cameras():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        rank, slowest, order = q.get(timeout=120)
        got[rank] = (slowest, order)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == got[1][0] == 2.5
    # each rank renders the same number of frames from its own offset of the orbit
    assert len(got[0][1]) == len(got[1][1]) == 8
    assert got[0][1] != got[1][1]
    assert got[1][1][0] == 37


def test_job_throughput_is_all_ranks_pixels_over_the_slowest_time():
    sys.path.insert(0, ROOT)
    import bench
    assert abs(bench.job_mpix_s(1, 640_000, 0.5) - 1280.0) < 1e-9
    assert abs(bench.job_mpix_s(4, 640_000, 0.5) - 5120.0) < 1e-9  # weak scaling: 4 replicas
    assert bench.max_over_ranks(3.25, 1, torch.device("cpu")) == 3.25  # no collective at N = 1


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
