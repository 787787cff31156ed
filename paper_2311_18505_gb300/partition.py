"""Splitting one batch of strings across ranks (one GPU each) by cost.

Strings are independent, so a batch shards with no exchange step.  A rank's
work is the sum over its strings of (N_t + N_l) x steps (the grid points a
step updates; forced strings, whose steps also solve for the unit-force
response, weigh 1.5 times), and the shards are balanced by greedy
longest-processing-time: strings in decreasing cost, each to the rank with
the least work so far.  The result is a function of the batch and the rank
count only, so every rank computes the same split without communicating.

This balances throughput-bound batches (more strings than the GPU has warp
schedulers).  A small batch is latency-bound: it takes as long as its
slowest string whichever rank holds it, so it is better run whole on each
rank (weak scaling) than split.

Grid sizes come from the library's host-side grid rule (`sfd_grid`, no
device needed); this module holds no arithmetic of the scheme.
"""

from __future__ import annotations

import heapq
from typing import Sequence

from . import sfd


def string_cost(d: dict) -> float:
    """(N_t + N_l) x samples, times 1.5 for a hammer or a bow."""
    n_t, n_l = sfd.sfd_grid(sfd.params_from_dict(d))
    forced = d["excitation"]["kind"] != "pluck"
    return (n_t + n_l) * float(d["n_samples"]) * (1.5 if forced else 1.0)


def partition_lpt(costs: Sequence[float], world: int) -> list[list[int]]:
    """Indices of the items each of `world` ranks takes: greedy longest
    processing time (ties broken by index and rank, so deterministic)."""
    if world <= 0:
        raise ValueError("world must be > 0")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def shard(strings: Sequence[dict], rank: int, world: int) -> list[int]:
    """Indices of `strings` that rank `rank` of `world` renders."""
    return partition_lpt([string_cost(d) for d in strings], world)[rank]
