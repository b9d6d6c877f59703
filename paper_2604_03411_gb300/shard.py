"""Assignment of independent specimens to ranks, one process per GPU.

Specimens of a batch share nothing (each is its own boundary-value problem with
its own networks and load path), so a multi-GPU run splits the list of
specimens and every rank solves its share in one batched handle; there is no
exchange on the data path.  The split balances the estimated work of a rank:
element-kernel work per specimen is proportional to its quadrature points times
its load steps.  The split is the longest-processing-time rule: specimens in
decreasing cost, each to the rank with the least work so far (ties: the lower
rank), which keeps the largest rank within 4/3 of the best possible split.
Every rank computes the same split from the same list, so no rank has to send
it to another.
"""
from __future__ import annotations

from typing import List, Sequence


def specimen_cost(problem) -> float:
    """Estimated work of one specimen: quadrature points x load steps."""
    m = problem.mesh
    return float(m.n_elems * m.nq * max(int(problem.load.size), 1))


def partition(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """Indices of the specimens of every rank (each list ascending)."""
    if world_size < 1:
        raise ValueError("world_size must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world_size
    out: List[List[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(x) for x in out]


def shard(problems: Sequence, rank: int, world_size: int) -> List[int]:
    """This rank's specimen indices."""
    if not 0 <= rank < world_size:
        raise ValueError("rank out of range")
    return partition([specimen_cost(p) for p in problems], world_size)[rank]
