"""Partition of independent RVEs over ranks (one GPU per rank).

RVEs share nothing during a solve (the paper's strong-scaling argument,
Sec. 5.2), so ranks take contiguous RVE ranges with no data-path
collective; the only exchange is gathering the results.  Ranges are
balanced by expected cost, e.g. active fibers x expected DR iterations.
"""
from __future__ import annotations

import numpy as np


def partition(costs, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, end) ranges, one per rank, splitting the cumulative
    cost as evenly as whole RVEs allow; every RVE in exactly one range."""
    costs = np.asarray(costs, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = costs.shape[0]
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(np.maximum(costs, 0.0))])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left"))
        k = min(max(k, cuts[-1]), n)
        # move the cut to whichever neighbour is closer to the target
        if 0 < k <= n and abs(cum[k - 1] - target) < abs(cum[k] - target) and k - 1 >= cuts[-1]:
            k -= 1
        cuts.append(k)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]
