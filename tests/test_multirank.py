"""Host-side multi-rank logic of the benchmark on CPU (gloo, world size 2):
max-over-ranks timing, whole-job aggregation, and the reference arm's
rank-0-only rule.  No GPU is used."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    mx = bench.max_over_ranks(local_ms, world)
    val = bench.whole_job_gflops(6.0e9, 4, world, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, val))


def test_two_rank_max_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in res:
        assert mx == 15.0                                  # the slowest rank's time
        assert abs(val - 2 * 6.0e9 * 4 / 15e-3 / 1e9) < 1e-9   # whole-job GFLOP/s


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=3, warmup=3, impl="reference", no_oracle=False)
    assert bench.run_reference(args) == 0      # returns at once, prints nothing


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert abs(bench.whole_job_gflops(1e9, 10, 1, 1000.0) - 10.0) < 1e-12
    assert bench.flops((1 << 10,)) == 5 * 1024 * 10
