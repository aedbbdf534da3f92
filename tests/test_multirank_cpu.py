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


# ------------------------------------------------------------------ row bands
def test_row_band_plan():
    for height, world, halo in [(10, 3, 2), (2, 4, 1), (7, 8, 3), (1000, 4, 5), (1, 1, 2)]:
        bands = shard.row_bands(height, world, halo)
        assert sorted(r for (y0, y1, _, _) in bands for r in range(y0, y1)) == list(range(height))
        sizes = [y1 - y0 for (y0, y1, _, _) in bands]
        assert max(sizes) - min(sizes) <= 1
        for (y0, y1, e0, e1) in bands:
            if y1 > y0:
                assert (e0, e1) == (max(0, y0 - halo), min(height, y1 + halo))


def _band_main(rank, world, port, q, height, width, halo):
    import numpy as np
    import torch
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = np.random.default_rng(77)
        img = g.random((height, width))                       # every rank draws the same image
        bands = shard.row_bands(height, world, halo)
        y0, y1, e0, e1 = bands[rank]
        ext = torch.full((e1 - e0, width), float("nan"), dtype=torch.float64)
        ext[y0 - e0:y1 - e0] = torch.from_numpy(img[y0:y1])   # own rows only
        shard.exchange_halos(ext, bands, rank, dist)
        ok_ext = bool(torch.equal(ext, torch.from_numpy(img[e0:e1])))
        errs = {}
        if y1 > y0:
            e = ext.numpy()
            w5, w11 = g.standard_normal((5, 5)), g.standard_normal((11, 11))
            for name, f in (("conv5 clamp", lambda a: oracle.conv2d(a, w5)),
                            ("conv11 constant", lambda a: oracle.conv2d(a, w11, "constant", 0.5)),
                            ("sep r4", lambda a: oracle.sepconv(a, synth.gaussian_taps(4), synth.gaussian_taps(4))),
                            ("harris 5", lambda a: oracle.harris(a, synth.sobel_x(), synth.sobel_y(),
                                                                 synth.gaussian_window(5, 1.0)))):
                band = f(e)[y0 - e0:y1 - e0]
                whole = f(img)[y0:y1]
                errs[name] = float(np.max(np.abs(band - whole)))
        q.put((rank, ok_ext, errs))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,height", [(2, 37), (3, 40), (4, 9)])
def test_gloo_row_bands_match_the_whole_image(world, height):
    """Bands with a halo of 5 rows (the 11x11 radius, and Sobel 1 + window 2 for Harris):
    after the exchange every extended band equals the image's rows, and the oracle run
    on it gives the whole image's values on the band's own rows, exactly."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_main, args=(r, world, port, q, height, 23, 5)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_ext, errs in res:
        assert ok_ext, f"rank {rank}: halo rows differ from the image"
        for name, e in errs.items():
            assert e == 0.0, f"rank {rank} {name}: band differs from the whole image by {e}"
