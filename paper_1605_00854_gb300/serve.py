"""Steady-state query serving with continuous batching.

A query asks for the steady-state probability of a meta-state of a PBN with
precision r at confidence s (Sec. 4.2: the two-state Markov chain approach).  The
server:

* prepares queries on host worker threads (pbn_load, pbn_reduce on the meta nodes,
  pbn_group, plan image upload, device buffers for the query's trajectories);
* admits prepared queries while the device bytes they may need (plan image,
  states and counts at the largest trajectory count they may grow to) fit under the
  memory cap, in arrival order;
* runs rounds: one persistent batched launch (pbn_batch_run) advances every active
  query by `chunk_steps` steps, then one copy brings back every query's pooled
  counts [V, n00, n01, n10, n11]; with kernel="auto" the trajectory blocks of
  queries whose plan compiled (pbn_plan_compile) and that hold at least
  `compiled_min_traj` trajectories run as their own compiled-plan launches on a
  few side streams instead, the rest in the batched launch;
* after each round applies the two-state Markov chain stopping rule to each query:
  if the burn-in m* exceeds the start of its counting window, the window restarts
  at the current step (counts cleared); if the counted states reach N*, the query
  completes with pi = V / L; otherwise it continues;
* grows a query that would need many more rounds: when the states still to count
  exceed `grow_rounds` rounds at its current trajectory count, it gets a new block
  of as many trajectories again (the next trajectory ids, their own burn-in), up to
  `max_traj`.

Each query's draws are keyed by its own seed and trajectory ids, every query
advances by the same chunk in every round, and the growth rule reads only the
query's own counts, so a query's result does not depend on the other queries in
flight.
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
    n_traj: int = 0
    n_eff: int = 0          # trajectories whose counting window had started (the estimate's n_traj)
    restarts: int = 0       # counting-window restarts by the burn-in rule
    # per trajectory block: traj_begin, n_traj, count_from, steps (and, with
    # Server(record_blocks=True), its final "state" [state_words, n_traj] and per-trajectory
    # "counts" [5, n_traj] as uint64 host arrays)
    blocks: list = field(default_factory=list)


class _Block:
    """A range of a query's trajectories with its own buffers and counting window."""

    def __init__(self, bufs, traj_begin: int, n_traj: int, count_from: int):
        self.bufs = bufs
        self.traj_begin = traj_begin
        self.n_traj = n_traj
        self.step = 0              # steps simulated so far
        self.count_from = count_from


class _Active:
    def __init__(self, q: Query, plan, bufs, n, prep_s, nbytes, count_from, n_traj, compiled=False):
        self.q = q
        self.plan = plan
        self.compiled = compiled
        self.compiling = None      # future of a background compilation
        self.blocks = [_Block(bufs, 0, n_traj, count_from)]
        self.n = n
        self.prep_s = prep_s
        self.nbytes = nbytes
        self.rounds = 0
        self.node_updates = 0.0
        self.restarts = 0

    @property
    def step(self) -> int:
        return self.blocks[0].step

    @property
    def n_traj(self) -> int:
        return sum(b.n_traj for b in self.blocks)


class Server:
    """Continuous-batching server for steady-state queries on one GPU."""

    def __init__(self, n_traj: int = 512, chunk_steps: int = 256, burn_in0: int = 64,
                 min_pairs: int = 4096, mem_cap_bytes: float = 100e9, workers: int = 8,
                 max_steps: int = 1 << 20, grow_rounds: int = 4, max_traj: int = 1 << 16, device="cuda",
                 kernel: str = "batch", sampler: int = _lib.PBN_PERT_BITSLICED,
                 compile_flags: int = _lib.PBN_COMPILE_INTERLEAVED, compiled_min_traj: int = 4096,
                 side_streams: int = 4, record_blocks: bool = False):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.n_traj = n_traj
        self.chunk = chunk_steps
        self.burn_in0 = burn_in0
        self.min_pairs = min_pairs
        self.cap = mem_cap_bytes
        self.max_steps = max_steps
        self.grow_rounds = grow_rounds
        self.max_traj = max(max_traj, n_traj)
        if kernel not in ("batch", "auto"):
            raise ValueError("kernel must be 'batch' or 'auto'")
        self.kernel = kernel
        self.sampler = sampler
        self.compile_flags = compile_flags
        self.compiled_min_traj = compiled_min_traj
        self.record_blocks = record_blocks
        self.side = [torch.cuda.Stream(self.dev) for _ in range(side_streams)] if kernel == "auto" else []
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.prepared: "queue.Queue" = queue.Queue()
        self.waiting = []          # prepared, not yet admitted (arrival order)
        self.active = []
        self.done = []
        self.rejected = []         # queries needing more bytes than the cap
        self.failed = []           # (qid, error) of queries whose preparation failed
        self.cancelled = []        # qids cancelled before completing
        self._cancel = set()
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
            plan = api.Plan(red, sampler=self.sampler)
            # compile now only if the query starts large enough to use it; otherwise
            # it is compiled in the background once it grows
            compiled = self.kernel == "auto" and self.n_traj >= self.compiled_min_traj and self._compile(plan)
            n = net.info().n
            # admission reserves the device bytes of the largest size the query may
            # grow to, so that growth never waits for memory and results stay
            # independent of the other queries; nothing is allocated on the device
            # before admission
            nbytes = query_bytes(plan, self.max_traj)
            self.prepared.put((q, plan, None, n, time.perf_counter() - t0, nbytes, compiled))
        except Exception as exc:  # a query that cannot be prepared fails alone
            with self.lock:
                self.failed.append((q.qid, repr(exc)))
                self.pending -= 1

    def _compile(self, plan) -> bool:
        try:
            plan.compile(self.compile_flags)
            return True
        except _lib.PbnError:  # too wide to compile: the batched interpreter runs it
            return False

    def submit(self, q: Query):
        if not q.arrival:
            q.arrival = time.perf_counter()
        with self.lock:
            self.pending += 1
        self.pool.submit(self._prepare, q)

    def cancel(self, qid: int):
        """Cancel a query: it is dropped before its next round (or when its
        preparation finishes) and its device bytes are released.  Other queries'
        results are unaffected (their draws are keyed by their own ids)."""
        with self.lock:
            self._cancel.add(qid)

    def _drop_cancelled(self):
        with self.lock:
            if not self._cancel:
                return
            # a query that already completed or failed is not cancelled
            over = {r.qid for r in self.done} | {f[0] for f in self.failed}
            self._cancel -= over
            cancel = set(self._cancel)
        keep = []
        for item in self.waiting:
            if item[0].qid in cancel:
                self._retire(item[0].qid)
            else:
                keep.append(item)
        self.waiting = keep
        for a in [a for a in self.active if a.q.qid in cancel]:
            self.active.remove(a)
            self.in_use -= a.nbytes
            self._retire(a.q.qid)

    def _retire(self, qid: int):
        self.cancelled.append(qid)
        with self.lock:
            self._cancel.discard(qid)
            self.pending -= 1

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
            q, plan, bufs, n, prep_s, nbytes, compiled = item
            if nbytes > self.cap:
                self.rejected.append(q.qid)
                with self.lock:
                    self.pending -= 1
                continue
            if self.in_use + nbytes <= self.cap:
                self.in_use += nbytes
                with self.torch.cuda.stream(self.stream):
                    plan.device_image(self.dev)
                    bufs = api.alloc_buffers(plan, self.n_traj, self.dev)
                self.active.append(_Active(q, plan, bufs, n, prep_s, nbytes, self.burn_in0, self.n_traj, compiled))
            else:
                keep.append(item)
        self.waiting = keep

    # -- one round --------------------------------------------------------------------
    def _round(self):
        torch = self.torch
        entries, owner, direct, blocks = [], [], [], []
        for a in self.active:
            if a.compiling is not None and a.compiling.done():
                a.compiled = a.compiling.result()
                a.compiling = None
        for qi, a in enumerate(self.active):
            for b in a.blocks:
                init = _lib.PBN_INIT_KEYED if b.step == 0 else _lib.PBN_INIT_STATE
                if a.compiled and b.n_traj >= self.compiled_min_traj:
                    direct.append((a, b, init))
                else:
                    entries.append(dict(plan=a.plan, bufs=b.bufs, seed=a.q.seed, meta_ids=a.q.meta_ids,
                                        meta_vals=a.q.meta_vals, traj_begin=b.traj_begin, step_begin=b.step,
                                        count_from=b.count_from, init=init))
                owner.append(qi)
                blocks.append(b)
        t0 = time.perf_counter()
        B = None
        with torch.cuda.stream(self.stream):
            if direct:
                # compiled-plan launches on side streams, after the server stream's
                # pending work (count resets, new buffers), joined back before the copy
                ready = self.stream.record_event()
                for i, (a, b, init) in enumerate(direct):
                    st = self.side[i % len(self.side)]
                    st.wait_event(ready)
                    api.simulate(a.plan, b.bufs, seed=a.q.seed, n_steps=self.chunk, meta_ids=a.q.meta_ids,
                                 meta_vals=a.q.meta_vals, traj_begin=b.traj_begin, step_begin=b.step,
                                 count_from=b.count_from, init=init, stream=st, kernel=_lib.PBN_KERNEL_COMPILED)
            if entries:
                B = api.Batch(entries, device=self.dev)
            t1 = time.perf_counter()
            if B is not None:
                B.run(self.chunk, step_offset=0, stream=self.stream)
            for st in self.side[: len(direct)]:
                self.stream.wait_event(st.record_event())
            pooled = torch.stack([b.bufs.pooled for b in blocks]).to("cpu", non_blocking=True)
            if direct:
                status = torch.stack([b.bufs.status for _, b, _ in direct]).to("cpu", non_blocking=True)
        self.stream.synchronize()
        if B is not None and int(B.status.item()) != 0:
            raise RuntimeError("batch kernel reported an error status")
        if direct and int(status.abs().sum()) != 0:
            raise RuntimeError("a compiled-plan launch reported an error status")
        t2 = time.perf_counter()
        pooled = pooled.numpy().view(np.uint64)
        per_query = np.zeros((len(self.active), 5), dtype=np.uint64)
        for qi, c in zip(owner, pooled):
            per_query[qi] += c
        finished = []
        for a, c in zip(self.active, per_query):
            for b in a.blocks:
                b.step += self.chunk
            a.rounds += 1
            nu = float(a.n) * a.n_traj * self.chunk
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
        # trajectories whose window has started (each contributes its first counted state)
        n_eff = sum(b.n_traj for b in a.blocks if b.step >= b.count_from)
        burn = min(b.count_from for b in a.blocks)
        est = api.estimate(c, max(1, n_eff), a.q.r, a.q.s, a.q.eps, burn_in_used=burn)
        if not est.defined or est.m_star == 2**64 - 1:
            # the meta-state was never (or always) seen, so the chain's switching rates
            # are not estimable: stop at the worst-case sample size of a proportion,
            # (z / r)^2 / 4, and report pi = V / L
            n_min = math.ceil(0.25 * (est.z / a.q.r) ** 2)
            if a.step >= self.max_steps or (est.L >= n_min and (int(c[0]) == 0 or int(c[0]) == est.L)):
                self._finish(a, est, c, n_eff)
                return True
            return False
        if est.m_star > burn:
            # restart the windows that began before the burn-in: at the next state to
            # be produced or at m*, whichever is later (the current state was counted
            # by the discarded window; ordered before the next round on the server's
            # stream)
            if a.step >= est.m_star:
                a.restarts += 1
                with self.torch.cuda.stream(self.stream):
                    for b in a.blocks:
                        if b.count_from < est.m_star:
                            b.count_from = max(b.step + 1, int(est.m_star))
                            b.bufs.counts.zero_()
                            b.bufs.pooled.zero_()
            return False
        if est.L >= est.n_star or a.step >= self.max_steps:
            self._finish(a, est, c, n_eff)
            return True
        self._maybe_grow(a, est)
        return False

    def _maybe_grow(self, a: _Active, est):
        """Double the query's trajectories when the states still to count exceed
        grow_rounds rounds at its current size (reads only the query's own counts)."""
        per_round = a.n_traj * self.chunk
        if est.n_star - est.L <= self.grow_rounds * per_round or 2 * a.n_traj > self.max_traj:
            return
        nb = a.n_traj
        with self.torch.cuda.stream(self.stream):
            bufs = api.alloc_buffers(a.plan, nb, self.dev)
        # new trajectories take the next ids and count after the query's burn-in
        burn = max(min(b.count_from for b in a.blocks), int(est.m_star))
        a.blocks.append(_Block(bufs, a.n_traj, nb, burn))
        if (self.kernel == "auto" and not a.compiled and a.compiling is None
                and max(b.n_traj for b in a.blocks) >= self.compiled_min_traj):
            a.compiling = self.pool.submit(self._compile, a.plan)
        self.stats["grown"] = self.stats.get("grown", 0) + 1

    def _finish(self, a: _Active, est, c, n_eff: int):
        latency = time.perf_counter() - a.q.arrival
        blocks = []
        for b in a.blocks:
            rec = {"traj_begin": b.traj_begin, "n_traj": b.n_traj, "count_from": b.count_from, "steps": b.step}
            if self.record_blocks:
                # this round's launches have completed (the round synchronised its stream)
                rec["state"] = b.bufs.state.cpu().numpy().view(np.uint64).copy()
                rec["counts"] = b.bufs.counts.cpu().numpy().view(np.uint64).copy()
            blocks.append(rec)
        self.done.append(Result(
            qid=a.q.qid, pi=est.pi, n_star=int(est.n_star), m_star=int(est.m_star), L=int(est.L),
            steps=a.step, rounds=a.rounds, latency=latency, prep_s=a.prep_s,
            node_updates=a.node_updates, alpha=est.alpha, beta=est.beta, counts=[int(x) for x in c],
            n_traj=a.n_traj, n_eff=int(n_eff), restarts=a.restarts, blocks=blocks))

    def step(self) -> list:
        """Admit what is ready and run one round (if anything is active)."""
        self._admit()
        self._drop_cancelled()
        if not self.active:
            return []
        nvtx = self.torch.cuda.nvtx
        nvtx.range_push(f"pbn serve round {self.stats['rounds']}: {len(self.active)} queries")
        try:
            return self._round()
        finally:
            nvtx.range_pop()

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
