"""The N > 1 host path on CPU ranks (gloo, world size 2): LPT sharding of the ragged
batch covers every image exactly once with balanced loads on every rank, and the timing
reduction returns the maximum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1605_06399_gb300 import shard, synth


def test_lpt_properties():
    g = synth.rng(5)
    costs = [float(c) for c in g.integers(1, 1000, size=97)]
    for world in (1, 2, 3, 8):
        sh = shard.lpt_shards(costs, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in sh]
        assert max(loads) - min(loads) <= max(costs)
        assert sh == shard.lpt_shards(costs, world)       # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = synth.workload_batch(n=64)
        costs = [shard.image_cost(it.width, it.height, it.op, it.k) for it in items]
        mine = shard.lpt_shards(costs, world)[rank]
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        t = shard.max_over_ranks(10.0 + rank, dist)
        q.put((rank, sorted(mine), everyone, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
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
    shards = res[0][2]
    assert res[1][2] == shards                        # every rank sees the same plan
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(64))
    assert [r[1] for r in res] == [sorted(s) for s in shards]
    assert all(r[3] == 11.0 for r in res)             # max over ranks
