"""The multi-GPU path is replicas only (one independent system per rank, no
collective on the data path); what crosses ranks is the timing: the job's
time is the slowest rank's, and its throughput counts every rank's work.
These run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(values[rank], dist, "cpu")
        out[rank] = m
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    values = [3.5, 7.25]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == max(values)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(4.0, None, "cpu") == 4.0


def test_whole_job_rate_counts_every_rank():
    # 2 ranks, 1e12 flops each, slowest rank 100 ms -> 2e13 flop/s = 20000 GFLOP/s
    assert bench.whole_job_rate(1e12, 2, 100.0) == pytest.approx(20000.0)
    assert bench.whole_job_rate(1e12, 1, 100.0) == pytest.approx(10000.0)
