"""Host-side sharding of a batch of independent boxes (lambda windows or trajectory frames) across ranks.

Each box is evaluated whole on one GPU (the single-box evaluation does not split across GPUs without
halo exchanges); boxes are assigned to ranks by the longest-processing-time rule on an estimated cost,
every rank evaluates its share with its own batch, and the per-box FP64 results are gathered on the host
of rank 0 in the original box order.  There is no device collective on the data path.
"""
from __future__ import annotations

import numpy as np


def box_cost(N: int, depth: int | None = None) -> float:
    """Estimated cost of one box: the evaluation is linear in the charge count (fixed charges per leaf),
    plus a fixed per-box latency worth about 20,000 charges (the coarse levels' launches)."""
    return float(N) + 2.0e4


def partition_boxes(costs, world: int) -> list[list[int]]:
    """Longest processing time first: boxes in descending cost, each to the currently lightest rank
    (ties to the lower rank).  Returns, per rank, its box indices in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def gather_box_results(local: dict[str, np.ndarray], mine: list[int], nbox: int, group=None):
    """Gather per-box FP64 arrays (same keys on every rank, one entry per box of `mine`) to rank 0 and
    place them at their box indices.  Returns the full arrays on rank 0 and None elsewhere.  Host
    memory only (torch.distributed gather_object over the process group)."""
    import torch.distributed as dist
    payload = {"idx": list(mine), **{k: np.asarray(v, dtype=np.float64).tolist() for k, v in local.items()}}
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        parts = [payload]
    else:
        parts = [None] * dist.get_world_size(group) if dist.get_rank(group) == 0 else None
        dist.gather_object(payload, parts, dst=0, group=group)
        if dist.get_rank(group) != 0:
            return None
    out = {k: np.full(nbox, np.nan) for k in local}
    seen = np.zeros(nbox, dtype=bool)
    for p in parts:
        for j, i in enumerate(p["idx"]):
            if seen[i]:
                raise ValueError("box %d reported by two ranks" % i)
            seen[i] = True
            for k in local:
                out[k][i] = p[k][j]
    if not seen.all():
        raise ValueError("boxes %s were not reported" % np.flatnonzero(~seen).tolist())
    return out
