"""Host-side work partitioning across ranks (one process per GPU).

Independent images shard across ranks with no collective on the data path (weak
scaling): ``lpt_shards`` assigns images to ranks longest-processing-time first, so the
busiest rank carries at most the lightest rank's load plus one image.

One large image splits into row bands (strong scaling), with one exchange step:
``row_bands`` gives each rank its rows and the halo of r rows on each side that a
radius-r stencil reads, and ``exchange_halos`` fills a rank's extended band from its
neighbours (point-to-point sends of r rows each way; NCCL between GPUs, gloo on CPU).
A stencil run on the extended band is exact on the band's own rows: each of them reads
rows at most r away, all present, and the boundary rule applies only at the image's
true first and last rows, which are the extended band's edges there.

``max_over_ranks`` is the timing reduction the benchmark uses.
"""
from __future__ import annotations


def image_cost(width: int, height: int, op: str, k: int) -> float:
    """Relative cost of one image: pixels x (flops per pixel + a memory term)."""
    flops = 2 * k * k if op == "conv" else 4 * k
    return float(width) * float(height) * (flops + 16)


def lpt_shards(costs, world: int):
    """Split item indices into `world` lists: items in decreasing cost (ties by index),
    each to the currently lightest rank (ties by rank).  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        shards[r].append(i)
        loads[r] += costs[i]
    for s in shards:
        s.sort()
    return shards


def max_over_ranks(value: float, dist=None) -> float:
    """The maximum of `value` over all ranks of the default process group (or `value`
    itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return value
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def row_bands(height: int, world: int, halo: int):
    """Per rank (y0, y1, e0, e1): own rows [y0, y1) and extended rows [e0, e1) =
    [max(0, y0 - halo), min(height, y1 + halo)).  Bands differ by at most one row;
    ranks past the height get empty bands."""
    if world < 1 or height < 0 or halo < 0:
        raise ValueError("world >= 1, height >= 0, halo >= 0")
    out = []
    for r in range(world):
        y0 = (height * r) // world
        y1 = (height * (r + 1)) // world
        e0, e1 = (max(0, y0 - halo), min(height, y1 + halo)) if y1 > y0 else (y0, y0)
        out.append((y0, y1, e0, e1))
    return out


def exchange_halos(ext, bands, rank: int, dist, group=None):
    """Fill the halo rows of this rank's extended band `ext` (rows [e0, e1) of the image,
    own rows already in place) from the ranks that own them, and send the rows of mine
    that other ranks' halos cover.  Usually the two neighbours; more when bands are
    thinner than the halo.  Every rank calls it.  Blocking.

    All sends and receives of the call are posted together as one batch of
    point-to-point operations (``batch_isend_irecv``).  NCCL runs such a batch as one
    group, so a pair of ranks that each receive from and send to the other cannot block
    one another: posted one at a time, each rank's receive would wait on a send that
    sits behind the other rank's receive on the pair's stream."""
    y0, y1, e0, e1 = bands[rank]
    ops, recvs = [], []
    for nb, (n0, n1, ne0, ne1) in enumerate(bands):
        if nb == rank:
            continue
        r0, r1 = max(n0, e0), min(n1, e1)          # its own rows inside my extended band
        if r1 > r0 and y1 > y0:
            buf = ext.new_empty((r1 - r0,) + tuple(ext.shape[1:]))
            ops.append(dist.P2POp(dist.irecv, buf, nb, group))
            recvs.append((buf, r0, r1))
    for nb, (n0, n1, ne0, ne1) in enumerate(bands):
        if nb == rank:
            continue
        s0, s1 = max(y0, ne0), min(y1, ne1)        # my own rows inside its extended band
        if s1 > s0 and n1 > n0:
            ops.append(dist.P2POp(dist.isend, ext[s0 - e0:s1 - e0].contiguous(), nb, group))
    if ops:
        for rq in dist.batch_isend_irecv(ops):
            rq.wait()
    for buf, r0, r1 in recvs:
        ext[r0 - e0:r1 - e0].copy_(buf)
    return ext
