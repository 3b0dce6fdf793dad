"""A batch of independent checks split over ranks, one GPU each.

The items of a batch (a host-loop sweep of one kernel, Sec. 4 class (4); a
corpus of kernels) are independent: no witness of one item depends on
another.  So a batch shards with no data-path exchange: each rank checks its
own share on its own GPU, and only the per-item verdicts travel, gathered on
the host once at the end.  Shares are cut by longest-processing-time-first
list scheduling (Graham, 1969) on the items' instance counts, the cost the
check's work grows with: items in decreasing cost, each to the rank with the
least assigned cost so far (ties to the lowest rank).
"""
from __future__ import annotations

import heapq


def lpt_partition(costs, world: int) -> list:
    """Item indices per rank (each share in increasing index order)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def gather(local: dict, n: int, dist=None) -> list:
    """Every rank's {item index: result} merged into one list of n results,
    in item order, on every rank (a host-side gather of the verdicts)."""
    parts = [local]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
    out = [None] * n
    for p in parts:
        for i, r in p.items():
            if out[i] is not None:
                raise RuntimeError(f"item {i} checked by two ranks")
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"items {missing[:8]} checked by no rank")
    return out


def check_sharded(kernels, costs=None, dist=None, checker=None, **batch_opts) -> list:
    """Check `kernels` (bound) split over the ranks of `dist` (or alone):
    this rank's LPT share runs as one batch (hgrd_batch_*), or through
    `checker(share_kernels) -> results`, and the verdicts of all ranks come
    back in item order.  `costs` default to the instance counts."""
    rank, world = 0, 1
    if dist is not None and dist.is_initialized():
        rank, world = dist.get_rank(), dist.get_world_size()
    if costs is None:
        costs = [k.info()[0] for k in kernels]
    share = lpt_partition(costs, world)[rank]
    mine = [kernels[i] for i in share]
    if checker is None:
        from . import Batch
        checker = lambda ks: Batch(ks, **batch_opts).check() if ks else []
    res = checker(mine)
    return gather(dict(zip(share, res)), len(kernels), dist)
