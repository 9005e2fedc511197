"""Multi-rank host logic on the CPU: two gloo ranks (127.0.0.1).

Every domain of an uneven sweep goes to exactly one rank, the split is
balanced, and the reductions the bench uses (slowest rank's time, all
ranks' units) give the whole-job throughput.
"""
import os
import socket

import pytest

from paper_0708_4182_gb300 import replicas
from paper_0708_4182_gb300 import workloads as wl


def sweep_costs(count=256):
    return [c["nx"] * c["ny"] for c in wl.batched_channels(count, seed=0)]


def test_partition_covers_every_unit_once_and_balances():
    costs = sweep_costs()
    for world in (1, 2, 3, 4, 8):
        parts = [replicas.partition(costs, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        ld = replicas.loads(costs, world)
        # LPT: the largest load exceeds the mean by at most the largest unit
        assert max(ld) - sum(costs) / world <= max(costs)
    with pytest.raises(ValueError):
        replicas.partition(costs, 2, 2)


def test_partition_edge_cases():
    assert replicas.partition([], 0, 2) == []
    assert replicas.partition([5], 0, 3) == [0] and replicas.partition([5], 1, 3) == []
    # equal costs: round robin in index order
    assert replicas.partition([1] * 6, 0, 2) == [0, 2, 4]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = sweep_costs()
        mine = replicas.partition(costs, rank, world)
        units = float(sum(costs[i] for i in mine))
        elapsed = 1.0 + rank          # rank 1 is the slow one
        total = replicas.sum_over_ranks(units)
        slowest = replicas.max_over_ranks(elapsed)
        thr = replicas.job_throughput(units, elapsed)
        n_domains = replicas.sum_over_ranks(len(mine))
        dist.barrier()
        out.put((rank, total, slowest, thr, n_domains))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
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
    costs = sweep_costs()
    for rank, total, slowest, thr, n in res:
        assert total == sum(costs)
        assert slowest == 2.0
        assert thr == pytest.approx(sum(costs) / 2.0)
        assert n == len(costs)


def test_single_process_reductions_are_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10.0, 2.0) == 5.0
