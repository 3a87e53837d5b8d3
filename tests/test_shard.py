"""Partition of ensemble members over ranks (the multi-GPU path of the
batched ensemble: members are independent, so ranks share no data).

CPU only: the partition itself, and a world-size-2 gloo run of the same
rank logic bench.py uses (every rank derives the same partition from the
seeded recipes, the ranks' parts cover every member once, and the step time
is the maximum over ranks)."""
import os
import socket

import pytest

from paper_2106_07154_gb300 import shard
from paper_2106_07154_gb300 import workloads as W


def test_greedy_partition_covers_and_balances():
    recipes = W.ensemble_recipes()
    weights = [r["n"] * r["M"] for r in recipes]
    for parts in (1, 2, 3, 8):
        p = shard.greedy_partition(weights, parts)
        flat = sorted(i for part in p for i in part)
        assert flat == list(range(len(weights)))
        loads = [sum(weights[i] for i in part) for part in p]
        # LPT bound: no part exceeds the mean by more than the largest item
        assert max(loads) <= sum(weights) / parts + max(weights)
    assert shard.greedy_partition(weights, 4) == shard.greedy_partition(list(weights), 4)


def test_greedy_partition_small_cases():
    assert shard.greedy_partition([5, 3, 3], 2) == [[0], [1, 2]]
    assert shard.greedy_partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert shard.greedy_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard.greedy_partition([1], 0)


def test_member_weight():
    assert shard.member_weight(100, 0, 8) == 300
    assert shard.member_weight(100, 10, 4) == 300 + 120


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    recipes = W.ensemble_recipes()
    weights = [r["n"] * r["M"] for r in recipes]
    parts = shard.greedy_partition(weights, world)
    mine = parts[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    cells = torch.tensor([sum(recipes[i]["n"] for i in mine)], dtype=torch.int64)
    dist.all_reduce(cells)
    t = torch.tensor([10.0 + rank], dtype=torch.float64)      # this rank's step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, gathered, int(cells.item()), float(t.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_partition():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (_, g0, c0, t0), (_, g1, c1, t1) = res
    assert g0 == g1                                   # every rank agrees on the partition
    assert sorted(g0[0] + g0[1]) == list(range(64))   # disjoint cover of all members
    recipes = W.ensemble_recipes()
    assert c0 == c1 == sum(r["n"] for r in recipes)
    assert t0 == t1 == 11.0                           # max over ranks
