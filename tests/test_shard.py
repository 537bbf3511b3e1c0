"""Config 4's batch spread over ranks by cost: a greedy longest-first
partition by n^3, each rank solving its share, and one all-gather of the
per-system iteration counts and flags (no exchange on the data path).  The
partition is checked directly; the gather runs as two gloo ranks on the CPU
with a stand-in solve that records which systems it was given."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0808_2794_gb300 import inputs, solver


def _ns():
    rng = np.random.default_rng(0)
    return np.rint(np.exp(rng.uniform(np.log(16), np.log(512), size=4096))).astype(int)


def test_partition_covers_every_system_once_and_balances():
    ns = _ns()
    for world in (1, 2, 3, 8):
        parts = solver.shard_by_cost(ns, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ns)))
        load = [sum(int(ns[i]) ** 3 for i in p) for p in parts]
        # greedy longest-first: no rank exceeds the mean by more than the largest system
        assert max(load) - sum(load) / world <= max(int(n) ** 3 for n in ns)
        if world > 1:
            assert max(load) / min(load) < 1.01


def test_partition_is_deterministic_and_longest_first():
    ns = [5, 100, 7, 100, 3]
    # 100 -> rank 0, 100 -> rank 1, 7 -> rank 0 (tie), 5 -> rank 1, 3 -> rank 1 (lighter)
    assert solver.shard_by_cost(ns, 2) == [[1, 2], [3, 0, 4]]
    assert solver.shard_by_cost([], 3) == [[], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = _ns()[:300]
        seen = []

        def get_system(i):
            seen.append(i)
            return (i, int(ns[i])), None

        def fake_solve(As, Bs):
            # a deterministic stand-in for the GPU solve: iter = n mod 7, flags = 32 for odd n
            it = np.array([n % 7 for _, n in As], dtype=np.int32)
            fl = np.array([32 if n % 2 else 0 for _, n in As], dtype=np.uint32)
            return [None] * len(As), it, fl

        mine, Xs, iters, flags = solver.gesv_batched_sharded(ns, get_system, solve=fake_solve)
        out[rank] = (list(mine), seen, iters.tolist(), flags.tolist())
    finally:
        dist.destroy_process_group()


def test_sharded_batch_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ns = _ns()[:300]
    mine0, seen0, it0, fl0 = out[0]
    mine1, seen1, it1, fl1 = out[1]
    assert sorted(seen0) == sorted(mine0) and sorted(seen1) == sorted(mine1)  # only its own systems
    assert sorted(mine0 + mine1) == list(range(len(ns)))  # every system exactly once
    assert it0 == it1 and fl0 == fl1  # every rank ends with the whole batch's results
    assert it0 == [int(n) % 7 for n in ns] and fl0 == [32 if n % 2 else 0 for n in ns]
