"""Sharding of a batch of independent systems over the processes of a job.

A single triangular solve does not shard across GPUs (every level, or every
flag hop of the synchronisation-free solve, would need a cross-GPU
exchange), so multi-GPU work is a batch of independent systems split over
the ranks: no collective in the data path, one host-side gather of the
per-system reports at the end.  This module holds that host logic; it does
no GPU work and needs no particular process-group backend (the tests run it
over gloo on CPU, a GPU job over NCCL).
"""
from __future__ import annotations

import heapq
from typing import Sequence

__all__ = ["system_cost", "partition", "local_share", "gather_reports"]


def system_cost(n: int, nnz: int, nrhs: int) -> int:
    """Work of one system: its nonzeros and right-hand-side entries, each
    touched once per right-hand side (the bytes of a forward solve grow with
    nnz + n per column)."""
    return (int(nnz) + int(n)) * max(1, int(nrhs))


def partition(costs: Sequence[int], world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of systems over `world`
    ranks: systems in decreasing cost order, each to the least-loaded rank
    (ties: lowest rank).  Deterministic, so every rank computes the same
    partition without communicating.  Returns, per rank, its system indices
    in increasing order.  The largest load is at most the mean load plus the
    largest single cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda m: (-int(costs[m]), m))
    heap = [(0, r) for r in range(world)]
    share: list[list[int]] = [[] for _ in range(world)]
    for m in order:
        load, r = heapq.heappop(heap)
        share[r].append(m)
        heapq.heappush(heap, (load + int(costs[m]), r))
    return [sorted(s) for s in share]


def local_share(costs: Sequence[int], rank: int, world: int) -> list[int]:
    """This rank's systems under `partition`."""
    return partition(costs, world)[rank]


def gather_reports(report: dict, dist=None, dst: int = 0):
    """Host-side gather of one report (a picklable dict: per-system status,
    timings) from every rank to `dst`.  Returns the list of reports on
    `dst`, None elsewhere; with no initialised process group, [report]."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return [report]
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(report, out, dst=dst)
    return out
