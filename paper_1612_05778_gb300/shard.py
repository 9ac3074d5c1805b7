"""Splitting a list of independent products across GPUs (one process per
GPU, no data-path collective).

The products of a batched call share nothing, so N GPUs can each run a
subset of them in one ipm_mul_batched call of their own.  The split is
balanced by an estimate of each product's cost: the analytic planner's
transform volume, r Y 2K points, weighted by the butterfly levels and the
per-point constant work of the three passes,

    cost = r Y 2K (3 (log2 Y + log2 K + 1) + 2 r + 4),

the same figure the planner minimises when it picks (K, M, r).  Products
are assigned largest first, each to the least-loaded rank (the LPT rule of
R. Graham, "Bounds on multiprocessing timing anomalies", SIAM J. Appl.
Math. 17, 1969): the most-loaded rank exceeds the least-loaded one by at
most the largest single cost, and the makespan is within 4/3 of the best
split.  Every rank computes the same split from the same shapes, so no
message is needed to agree on it.
"""
from __future__ import annotations

import heapq
import math


def product_cost(info: dict) -> float:
    """Cost estimate of one product from its plan info (ipm.choose)."""
    if info.get("school"):
        # schoolbook family: limb products
        return float(info["na"] * info["nb"] * info["la"] * info["lb"])
    r, Y, K = info["r"], info["Y"], info["K"]
    return float(r * Y * 2 * K * (3 * (math.log2(Y) + math.log2(K) + 1) + 2 * r + 4))


def shape_costs(shapes) -> list[float]:
    """Cost of every (na, nb, bits_a, bits_b) shape under the analytic
    planner (host-only: the planner runs on the CPU)."""
    import paper_1612_05778_gb300 as ipm
    return [product_cost(ipm.choose(*s)) for s in shapes]


def partition(costs, world: int) -> list[list[int]]:
    """Indices of the products each of `world` ranks runs (each list in
    increasing order).  Deterministic: ties in cost go to the lower index,
    ties in load to the lower rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, rank) for rank in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, rank = heapq.heappop(heap)
        parts[rank].append(i)
        heapq.heappush(heap, (load + costs[i], rank))
    return [sorted(p) for p in parts]


def loads(costs, parts) -> list[float]:
    """Total cost per rank."""
    return [sum(costs[i] for i in p) for p in parts]
