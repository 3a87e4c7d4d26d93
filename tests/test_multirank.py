"""Multi-process host logic of bench.py on CPU: two gloo ranks.

The GPU path runs replicas (one tracker per rank, no data-path collective);
what crosses ranks is the timing: the slowest rank's time and the whole-job
throughput over all ranks' particles.  The reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
        value = bench.job_value(1000, ws, ms)
        env = bench.dist_env()
        # the reference arm does no work on ranks other than 0 (returns before building the oracle)
        ran = None
        if rank != 0:
            class A:
                steps, warmup, inner, gpus = 1, 0, 1, ws
            ran = bench.run_reference(A())
        q.put((rank, ms, value, env, ran))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_value():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env, ran in out:
        assert ms == 15.0                                  # the slowest rank
        assert value == pytest.approx(1000 * 2 / 15e-3)    # both ranks' units over that time
        assert env == (2, rank, rank)
        assert ran is None


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import torch

    import bench

    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.job_value(10, 1, 2.0) == pytest.approx(5000.0)
