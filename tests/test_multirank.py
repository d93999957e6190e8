"""Multi-rank host logic on CPU (gloo, world size 2): the max-over-ranks
timing reduction and the sharding of independent dose pairs across ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.reduce_max(1.5 + rank, world)
        costs = [5, 3, 9, 1, 4, 4, 7]
        mine = bench.shard_pairs(costs, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_max_reduction_and_pair_sharding_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, gathered in results:
        assert slowest == 2.5
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(7))                       # every pair exactly once
        loads = [sum([5, 3, 9, 1, 4, 4, 7][i] for i in part) for part in gathered]
        assert max(loads) - min(loads) <= 9                 # greedy balance


def test_single_rank_is_identity():
    assert bench.reduce_max(3.25, 1) == 3.25
    assert bench.shard_pairs([1, 2, 3], 1, 0) == [0, 1, 2]
