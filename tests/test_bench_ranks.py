"""The multi-rank logic of bench.py on the CPU: gloo ranks, world size 2.

bench.py --gpus N runs N independent replicas (the path does not shard), times the job by
its slowest rank and reports the whole-job throughput.  The reference arm runs on rank 0
only; other ranks leave without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"))  # rank times 1.5 s and 2.5 s
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_gloo_world_2():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == 2.5 and out[1] == 2.5


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.25, 1, None) == 3.25


def test_job_throughput_is_weak_scaling():
    # 5.37 GB per replica per step, 10 steps in 1.25 s on each of 4 ranks
    y = 40.0 * 512**3
    one = bench.job_throughput(y, 10, 1.25, 1)
    assert bench.job_throughput(y, 10, 1.25, 4) == pytest.approx(4 * one)
    assert one == pytest.approx(y * 10 / 1.25 / 1e9)


def test_reference_arm_other_ranks_leave_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
