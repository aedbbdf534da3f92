"""Host-side work partitioning across ranks (one process per GPU).

The stencil operators have no exchange step: independent images shard across ranks with
no collective on the data path (weak scaling).  ``lpt_shards`` assigns images to ranks
longest-processing-time first, so the busiest rank carries at most the lightest rank's
load plus one image.  ``max_over_ranks`` is the timing reduction the benchmark uses.
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
