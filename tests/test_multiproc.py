"""Multi-process host logic of the benchmark on CPU ranks (gloo, world size 2).

The step is not sharded: N GPUs run N independent replicas.  What needs checking without a GPU is the timing
aggregation (max over ranks, whole-job throughput) and that the reference arm
prints from rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    sys.path.insert(0, ROOT)
    import bench

    tot, value = bench.reduce_timing(100.0 * (rank + 1), 10, 2)
    out[rank] = (tot, value)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_timing_takes_max_over_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        tot, value = out[r]
        assert tot == 200.0                      # slowest rank
        assert abs(value - 2 * 10 / 0.2) < 1e-9  # 20 steps in 0.2 s


def test_single_rank_timing_is_local():
    sys.path.insert(0, ROOT)
    import bench

    tot, value = bench.reduce_timing(50.0, 5, 1)
    assert tot == 50.0 and abs(value - 100.0) < 1e-9


@pytest.mark.slow
def test_reference_arm_prints_on_rank0_only():
    """Rank 1 of the reference arm exits 0 without output or work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
