"""The N > 1 host path on CPU: two gloo ranks (no GPU).

Covers the max-over-ranks step time used by bench.py under torchrun and the deterministic
assignment of ensemble instances to ranks (every rank must compute the same disjoint cover).
"""
import os
import socket

import pytest

from paper_2401_06132_gb300 import replicas, workloads as W

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        slowest = replicas.max_over_ranks(ms)
        draws = W.ensemble_draws(64)
        costs = [d["edge"] ** 3 * (d["p"] + 1) ** 3 for d in draws]
        mine = replicas.assign_instances(costs, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_partition():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, gathered in res:
        assert slowest == 15.0
        allidx = sorted(i for part in gathered for i in part)
        assert allidx == list(range(64))               # disjoint cover of every instance
    assert res[0][2] == res[1][2]                      # same assignment on both ranks


def test_assignment_is_balanced_and_deterministic():
    draws = W.ensemble_draws(64)
    costs = [d["edge"] ** 3 * (d["p"] + 1) ** 3 for d in draws]
    for world in (1, 2, 4, 8):
        parts = replicas.assign_instances(costs, world)
        assert parts == replicas.assign_instances(costs, world)
        loads = [sum(costs[i] for i in part) for part in parts]
        assert sorted(i for part in parts for i in part) == list(range(64))
        assert max(loads) <= sum(costs) / world + max(costs)   # greedy LPT bound


def test_replica_throughput_counts_all_ranks():
    assert replicas.replica_throughput(1_000_000, 4, 2.0, 8) == pytest.approx(16.0)
