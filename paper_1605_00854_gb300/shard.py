"""Trajectory-id sharding across ranks.

Trajectories are independent and every draw is keyed by the global trajectory id, so
any split of the id range reproduces one run exactly; no data exchange is needed
beyond adding the five pooled counts of a query (a host-side sum).
"""
from __future__ import annotations


def weak_range(rank: int, world: int, per_rank: int):
    """(traj_begin, n_traj) of `rank` when every rank simulates per_rank trajectories."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    return rank * per_rank, per_rank


def strong_range(rank: int, world: int, total: int):
    """(traj_begin, n_traj) of `rank` for a contiguous split of `total` trajectories."""
    if not (0 <= rank < world) or total < 0:
        raise ValueError("bad rank/world/total")
    lo = total * rank // world
    hi = total * (rank + 1) // world
    return lo, hi - lo


def pool(counts_per_rank):
    """Sum the pooled [V, n00, n01, n10, n11] counts of several ranks."""
    out = [0, 0, 0, 0, 0]
    for c in counts_per_rank:
        for i in range(5):
            out[i] += int(c[i])
    return out
