"""The bench's multi-rank host logic on CPU ranks (gloo, world size 2).

The workload shards across ranks as independent replicas (each rank runs
its own batch of right-hand sides; no data-path collective): the only
collectives are the barriers around the timed region and the maximum of
the ranks' times. These run here on two CPU processes.
"""

import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench
    w_, r_, l_ = bench.dist_setup(None)
    bench.dist_init(w_, l_, "gloo")
    bench.barrier(w_)
    ms = 100.0 + 50.0 * r_  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, w_, "cpu")
    value = bench.job_value(16, 3, w_, ms_max)
    ref = None
    if r_ == 1:  # the reference arm does its work on rank 0 only
        args = argparse.Namespace(warmup=1, steps=1)
        ref = bench.run_reference(args, bench.workload(argparse.Namespace(dims=None, m=None, k=None, nrhs=None)),
                                  w_, r_)
    bench.barrier(w_)
    dist.destroy_process_group()
    q.put((r_, w_, ms_max, value, ref))


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, ms_max, value, ref in out:
        assert w == 2
        assert ms_max == 150.0  # the slowest rank's time, on every rank
        assert value == pytest.approx(16 * 3 * 2 / 0.150)  # all ranks' right-hand sides
        assert ref is None
