"""Sharding of independent geometries across ranks (one process per GPU).

The geometries of a bond scan are independent ground-state problems, so a job of
several scans or a long scan splits across GPUs with no exchange on the data path:
every rank builds and solves only the geometries assigned to it, and the one
collective is the final gather of the energies (a few doubles per geometry).  The
assignment is longest-processing-time first over an estimate of each geometry's
sigma cost, so ranks finish close together although subspace sizes are uneven.

Host logic only: the solves themselves run through the C ABI on each rank's GPU.
"""
from __future__ import annotations

import heapq


def geometry_cost(n_alpha_strings: int, n_beta_strings: int) -> float:
    """Relative sigma cost of one geometry from its string counts (the work of the
    row products and the opposite-spin term grows with N = N_alpha * N_beta)."""
    return float(n_alpha_strings) * float(n_beta_strings)


def lpt_assign(costs, world: int):
    """Longest-processing-time assignment: geometry indices per rank (each list in
    the order the rank should solve them, longest first).  Deterministic: ties go to
    the lower rank and the lower geometry index."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda g: (-float(costs[g]), g))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        out[r].append(g)
        heapq.heappush(heap, (load + float(costs[g]), r))
    return out


def solve_sharded(costs, solve_one, rank: int, world: int, group=None):
    """Solve this rank's share and gather every geometry's result on all ranks.

    costs      per-geometry cost estimates (same list on every rank)
    solve_one  callable(g) -> (energy, status) for geometry g, run locally
    Returns (energies, statuses) over all geometries, in geometry order.  With
    world == 1 no collective is made."""
    mine = lpt_assign(costs, world)[rank]
    local = {g: solve_one(g) for g in mine}
    if world == 1:
        gathered = [local]
    else:
        import torch.distributed as dist

        gathered = [None] * world
        dist.all_gather_object(gathered, local, group=group)
    energies = [None] * len(costs)
    statuses = [None] * len(costs)
    for part in gathered:
        for g, (e, st) in part.items():
            energies[g] = e
            statuses[g] = st
    if any(e is None for e in energies):
        raise RuntimeError("a geometry was not solved by any rank")
    return energies, statuses
