"""Trajectory-id sharding across ranks, and recovery of the ranges of failed ranks.

Trajectories are independent and every draw is keyed by the global trajectory id, so
any split of the id range reproduces one run exactly; no data exchange is needed
beyond adding the five pooled counts of a query (a host-side sum).  For the same
reason a range whose rank failed can be recomputed by any other process and gives
the same bits: ranks publish their results to a key-value store, the collector waits
for each with a time limit and reports the ranges that never arrived.
"""
from __future__ import annotations

import io
import time

import numpy as np


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


def missing_ranges(done, total: int):
    """Sub-ranges of [0, total) not covered by the (traj_begin, n_traj) pairs in done."""
    out, cur = [], 0
    for b, n in sorted(done):
        if b > cur:
            out.append((cur, b - cur))
        cur = max(cur, b + n)
    if cur < total:
        out.append((cur, total - cur))
    return out


def publish(store, rank: int, traj_begin: int, n_traj: int, arrays: dict):
    """Store a rank's results (named numpy arrays) under its rank."""
    buf = io.BytesIO()
    np.savez(buf, traj_begin=np.int64(traj_begin), n_traj=np.int64(n_traj), **arrays)
    store.set(f"pbn/rank/{rank}", buf.getvalue())


def collect(store, ranks, timeout_s: float):
    """Results published by the given ranks within timeout_s seconds in total:
    {rank: (traj_begin, n_traj, arrays)}; ranks that did not publish are left out."""
    import datetime
    got = {}
    deadline = time.monotonic() + timeout_s
    for r in ranks:
        left = deadline - time.monotonic()
        try:
            store.wait([f"pbn/rank/{r}"], datetime.timedelta(seconds=max(0.01, left)))
        except Exception:  # the rank never published (failed, exited or too slow)
            continue
        z = np.load(io.BytesIO(store.get(f"pbn/rank/{r}")))
        arrays = {k: z[k] for k in z.files if k not in ("traj_begin", "n_traj")}
        got[r] = (int(z["traj_begin"]), int(z["n_traj"]), arrays)
    return got
