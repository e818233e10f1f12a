"""Steady-state query serving with continuous batching.

A query asks for the steady-state probability of a meta-state of a PBN with
precision r at confidence s (Sec. 4.2: the two-state Markov chain approach).  The
server:

* prepares queries on host worker threads (pbn_load, pbn_reduce on the meta nodes,
  pbn_group, plan image upload, device buffers for the query's trajectories);
* admits prepared queries while the device bytes they need (plan image, states,
  counts) fit under the memory cap, in arrival order;
* runs rounds: one persistent batched launch (pbn_batch_run) advances every active
  query by `chunk_steps` steps, then one copy brings back every query's pooled
  counts [V, n00, n01, n10, n11];
* after each round applies the two-state Markov chain stopping rule to each query:
  if the burn-in m* exceeds the start of its counting window, the window restarts
  at the current step (counts cleared); if the counted states reach N*, the query
  completes with pi = V / L; otherwise it continues.

Each query's draws are keyed by its own seed and trajectory ids and every query
advances by the same chunk in every round, so a query's result does not depend on
the other queries in flight.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import _lib, api


@dataclass
class Query:
    qid: int
    text: str
    meta_ids: list
    seed: int
    r: float = 0.01
    s: float = 0.95
    eps: float = 1e-3
    meta_vals: list | None = None
    arrival: float = 0.0


@dataclass
class Result:
    qid: int
    pi: float
    n_star: int
    m_star: int
    L: int
    steps: int
    rounds: int
    latency: float
    prep_s: float
    node_updates: float
    alpha: float
    beta: float
    counts: list = field(default_factory=list)


class _Active:
    def __init__(self, q: Query, plan, bufs, n, prep_s, nbytes, count_from):
        self.q = q
        self.plan = plan
        self.bufs = bufs
        self.n = n
        self.prep_s = prep_s
        self.nbytes = nbytes
        self.step = 0              # steps simulated so far
        self.count_from = count_from
        self.rounds = 0
        self.node_updates = 0.0


class Server:
    """Continuous-batching server for steady-state queries on one GPU."""

    def __init__(self, n_traj: int = 512, chunk_steps: int = 256, burn_in0: int = 64,
                 min_pairs: int = 4096, mem_cap_bytes: float = 100e9, workers: int = 8,
                 max_steps: int = 1 << 20, device="cuda"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.n_traj = n_traj
        self.chunk = chunk_steps
        self.burn_in0 = burn_in0
        self.min_pairs = min_pairs
        self.cap = mem_cap_bytes
        self.max_steps = max_steps
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.prepared: "queue.Queue" = queue.Queue()
        self.waiting = []          # prepared, not yet admitted (arrival order)
        self.active = []
        self.done = []
        self.rejected = []         # queries needing more bytes than the cap
        self.failed = []           # (qid, error) of queries whose preparation failed
        self.in_use = 0
        self.stream = torch.cuda.Stream(self.dev)
        self.pending = 0
        self.lock = threading.Lock()
        self.node_updates = 0.0
        # host-side time split of the rounds (seconds): batch build, launch + wait, decisions
        self.stats = {"rounds": 0, "build_s": 0.0, "device_s": 0.0, "decide_s": 0.0}

    # -- preparation (host worker threads) -------------------------------------------
    def _prepare(self, q: Query):
        try:
            t0 = time.perf_counter()
            net = api.Net.load(q.text)
            red, _ = net.reduce(q.meta_ids)
            plan = api.Plan(red)
            n = net.info().n
            with self.torch.cuda.stream(self.stream):
                plan.device_image(self.dev)
                bufs = api.alloc_buffers(plan, self.n_traj, self.dev)
            nbytes = query_bytes(plan, self.n_traj)
            self.prepared.put((q, plan, bufs, n, time.perf_counter() - t0, nbytes))
        except Exception as exc:  # a query that cannot be prepared fails alone
            with self.lock:
                self.failed.append((q.qid, repr(exc)))
                self.pending -= 1

    def submit(self, q: Query):
        if not q.arrival:
            q.arrival = time.perf_counter()
        with self.lock:
            self.pending += 1
        self.pool.submit(self._prepare, q)

    # -- admission ----------------------------------------------------------------------
    def _admit(self):
        while True:
            try:
                item = self.prepared.get_nowait()
            except queue.Empty:
                break
            self.waiting.append(item)
        self.waiting.sort(key=lambda it: it[0].arrival)
        keep = []
        for item in self.waiting:
            q, plan, bufs, n, prep_s, nbytes = item
            if nbytes > self.cap:
                self.rejected.append(q.qid)
                with self.lock:
                    self.pending -= 1
                continue
            if self.in_use + nbytes <= self.cap:
                self.in_use += nbytes
                self.active.append(_Active(q, plan, bufs, n, prep_s, nbytes, self.burn_in0))
            else:
                keep.append(item)
        self.waiting = keep

    # -- one round --------------------------------------------------------------------
    def _round(self):
        torch = self.torch
        entries = []
        for a in self.active:
            entries.append(dict(plan=a.plan, bufs=a.bufs, seed=a.q.seed, meta_ids=a.q.meta_ids,
                                meta_vals=a.q.meta_vals, step_begin=a.step, count_from=a.count_from,
                                init=_lib.PBN_INIT_KEYED if a.step == 0 else _lib.PBN_INIT_STATE))
        t0 = time.perf_counter()
        with torch.cuda.stream(self.stream):
            B = api.Batch(entries, device=self.dev)
            t1 = time.perf_counter()
            B.run(self.chunk, step_offset=0, stream=self.stream)
            pooled = torch.stack([a.bufs.pooled for a in self.active]).to("cpu", non_blocking=True)
        self.stream.synchronize()
        if int(B.status.item()) != 0:
            raise RuntimeError("batch kernel reported an error status")
        t2 = time.perf_counter()
        pooled = pooled.numpy().view(np.uint64)
        finished = []
        for a, c in zip(self.active, pooled):
            a.step += self.chunk
            a.rounds += 1
            nu = float(a.n) * self.n_traj * self.chunk
            a.node_updates += nu
            self.node_updates += nu
            if self._decide(a, c):
                finished.append(a)
        for a in finished:
            self.active.remove(a)
            self.in_use -= a.nbytes
            with self.lock:
                self.pending -= 1
        st = self.stats
        st["rounds"] += 1
        st["build_s"] += t1 - t0
        st["device_s"] += t2 - t1
        st["decide_s"] += time.perf_counter() - t2
        return finished

    def _decide(self, a: _Active, c) -> bool:
        """Two-state chain stopping rule on the query's pooled counts."""
        pairs = int(c[1] + c[2] + c[3] + c[4])
        if pairs < self.min_pairs and a.step < self.max_steps:
            return False
        est = api.estimate(c, self.n_traj, a.q.r, a.q.s, a.q.eps, burn_in_used=a.count_from)
        if not est.defined or est.m_star == 2**64 - 1:
            if a.step >= self.max_steps:
                self._finish(a, est, c)
                return True
            return False
        if est.m_star > a.count_from:
            if a.step >= est.m_star:
                # restart the counting window after the burn-in (ordered before the
                # next round on the server's stream)
                a.count_from = a.step
                with self.torch.cuda.stream(self.stream):
                    a.bufs.counts.zero_()
                    a.bufs.pooled.zero_()
            return False
        if est.L >= est.n_star or a.step >= self.max_steps:
            self._finish(a, est, c)
            return True
        return False

    def _finish(self, a: _Active, est, c):
        self.done.append(Result(
            qid=a.q.qid, pi=est.pi, n_star=int(est.n_star), m_star=int(est.m_star), L=int(est.L),
            steps=a.step, rounds=a.rounds, latency=time.perf_counter() - a.q.arrival, prep_s=a.prep_s,
            node_updates=a.node_updates, alpha=est.alpha, beta=est.beta, counts=[int(x) for x in c]))

    def step(self) -> list:
        """Admit what is ready and run one round (if anything is active)."""
        self._admit()
        if not self.active:
            return []
        return self._round()

    def drain(self, timeout: float = 600.0):
        """Run rounds until every submitted query has completed."""
        t_end = time.perf_counter() + timeout
        while time.perf_counter() < t_end:
            with self.lock:
                left = self.pending
            if left == 0:
                return
            if not self.step():
                time.sleep(0.001)
        raise TimeoutError("queries still pending")

    def close(self):
        self.pool.shutdown(wait=True)


def query_bytes(plan, n_traj: int) -> int:
    """Device bytes a query holds while admitted: plan image, states, counts, pooled."""
    return int(plan.info.image_bytes + n_traj * (plan.info.state_words * 8 + 5 * 8) + 5 * 8)


def latency_summary(results) -> dict:
    lat = np.array([r.latency for r in results])
    if lat.size == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()), "count": int(lat.size)}
