"""Independent games over several ranks (one process per GPU).

The games of a batch or of a request stream are independent problems, so
they shard with no collective on the data path: each rank loads and solves
its own games. Collectives are used only around that, to agree on timings
(the slowest rank's time) and to bring results or counts to one rank for
reporting. The games of a batch are assigned largest first to the rank with
the least work so far (greedy LPT), with the vertex count as the work of a
game; the arrivals of a stream go, in arrival order, to the rank with the
least work submitted so far. Ties go to the lower rank, so every rank
computes the same assignment on its own.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_assign(weights, world):
    """Index arrays (ascending) of the games of each of ``world`` ranks."""
    w = np.asarray(weights, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be at least 1")
    order = np.argsort(-w, kind="stable")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(w.size, dtype=np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(w[i]), r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def shard_of(weights, world, rank):
    """The games of ``rank`` (ascending indices)."""
    return lpt_assign(weights, world)[rank]


def stream_assign(weights, world):
    """Owner rank of each arrival of a request stream, in arrival order: each
    arrival goes to the rank with the least work submitted so far (its
    vertices), ties to the lower rank. Unlike lpt_assign it looks at no later
    arrival, so a rank can decide on each request as it comes; every rank
    that sees the same arrivals computes the same owners, with no message."""
    w = np.asarray(weights, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be at least 1")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(w.size, dtype=np.int64)
    for i in range(w.size):
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(w[i]), r))
    return owner


def _dist():
    try:
        import torch.distributed as dist
    except ImportError:  # pragma: no cover
        return None
    return dist if dist.is_available() and dist.is_initialized() else None


def _reduce(x, op):
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op(dist))
    return float(t.item())


def max_over_ranks(x):
    """The maximum of ``x`` over all ranks (``x`` itself without a process group)."""
    return _reduce(x, lambda d: d.ReduceOp.MAX)


def sum_over_ranks(x):
    """The sum of ``x`` over all ranks (``x`` itself without a process group)."""
    return _reduce(x, lambda d: d.ReduceOp.SUM)


def gather_to_all(obj):
    """Every rank's ``obj``, in rank order ([obj] without a process group)."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def barrier():
    dist = _dist()
    if dist is not None and dist.get_world_size() > 1:
        dist.barrier()
