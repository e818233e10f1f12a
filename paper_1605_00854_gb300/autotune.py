"""Autotuner: group size, kernel, lanes per trajectory and steps per launch.

For one network it builds plans with several caps on the inputs of a merged group
(the group size of Sec. 3.3; larger groups mean fewer table lookups but bigger
tables), and for each plan times short launches of the candidate kernels on the
caller's trajectory count: the compiled plan (when the plan can be compiled, with
each code-shape flag), the interpreter with 1 to 32 lanes per trajectory and the
team interpreter (warps sharing 32 trajectories, for states of 8 rows or more),
with the tables in shared or in global memory.  The fastest configuration is returned and cached by the shape of
the problem.  For batches it times CUDA-graph replays of the persistent launch with
several steps per launch.

Every candidate simulates the same keyed trajectories, so the choice changes speed
only, never results.
"""
from __future__ import annotations

import json
import os
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import asdict, dataclass

from . import _lib, api

_CACHE: dict = {}
_LOCK = threading.Lock()


@dataclass
class Choice:
    max_inputs: int
    kernel: int            # _lib.PBN_KERNEL_COMPILED or _lib.PBN_KERNEL_INTERP
    lanes_per_traj: int
    smem_budget: int       # 0 = default (tables staged when they fit)
    node_updates_per_s: float
    compile_flags: int = 0  # pbn_plan_compile flags of the compiled kernel
    team_warps: int = 0     # _lib.PBN_KERNEL_TEAM: warps per team (0 = the library's choice)


def _shape_key(net: api.Net, meta, n_traj: int) -> str:
    import torch
    info = net.info()
    tb = max(0, n_traj.bit_length() - 1)
    gpu = torch.cuda.get_device_name().replace(" ", "_") if torch.cuda.is_available() else "cpu"
    return f"{gpu}-n{info.n}-f{info.n_functions}-m{len(meta)}-p{info.P}-t{tb}"


def _time(plan, bufs, seed, steps, meta, kernel, lanes, team_warps=0) -> float:
    import torch
    kw = dict(kernel=kernel, lanes_per_traj=lanes, team_warps=team_warps)
    api.simulate(plan, bufs, seed=seed, n_steps=8, meta_ids=meta, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.simulate(plan, bufs, seed=seed, n_steps=steps, meta_ids=meta, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def tune_network(text: str, meta, n_traj: int, *, steps: int = 256, seed: int = 1,
                 max_inputs_options=(4, 6, 8, 12), lanes_options=(1, 2, 4, 8, 16, 32),
                 compile_flags_options=(0, _lib.PBN_COMPILE_INTERLEAVED, _lib.PBN_COMPILE_PIPELINED,
                                        _lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_COMPILE_MAGIC_GATHER,
                                        _lib.PBN_COMPILE_PIPELINED | _lib.PBN_COMPILE_MAGIC_GATHER),
                 try_compiled: bool = True, cache_file: str | None = None, log=None,
                 sampler: int = _lib.PBN_PERT_BITSLICED,
                 warp_split_options=(_lib.PBN_COMPILE_WARPS(2) | _lib.PBN_COMPILE_WS_BATCH(1),
                                     _lib.PBN_COMPILE_WARPS(2),
                                     _lib.PBN_COMPILE_WARPS(4)),
                 warp_split_max_inputs: int = 8, team_warps_options=(0, 8)) -> Choice:
    """Pick the fastest (group size, kernel and its compile flags, lanes, table
    placement) for simulating n_traj trajectories of this network."""
    net = api.Net.load(text)
    key = _shape_key(net, meta, n_traj) + f"-s{sampler}"
    with _LOCK:
        if key in _CACHE:
            return _CACHE[key]
    if cache_file and os.path.exists(cache_file):
        try:
            with open(cache_file) as f:
                saved = json.load(f)
            if key in saved:
                ch = Choice(**saved[key])
                with _LOCK:
                    _CACHE[key] = ch
                return ch
        except (OSError, ValueError, TypeError):
            pass
    red, _ = net.reduce(list(meta))
    n = net.info().n
    best = None
    for mi in max_inputs_options:
        default_staged = None
        for budget in (0, 1024, 220 * 1024):
            try:
                plan = api.Plan(red, max_inputs=mi, smem_budget=budget, sampler=sampler) if budget \
                    else api.Plan(red, max_inputs=mi, sampler=sampler)
            except _lib.PbnError:
                continue
            if budget == 0:
                default_staged = bool(plan.info.tables_in_smem)
            # the small budget moves the tables to global memory, the large one into
            # shared memory: skip them when they give the default plan again
            if budget == 1024 and plan.info.tables_in_smem:
                continue
            if budget > 1024 and (default_staged or not plan.info.tables_in_smem):
                continue
            bufs = api.alloc_buffers(plan, n_traj)
            cands = []
            if try_compiled and budget == 0:
                cands += [(_lib.PBN_KERNEL_COMPILED, 1, f, plan, 0) for f in compile_flags_options]
                # plans too wide for the default forms: the wide register form, while its
                # code stays small (it compiles for minutes at thousands of nodes)
                if plan.info.n_sel_blocks > 24 and plan.info.n_groups <= 512 and plan.info.n <= 1024:
                    cands.append((_lib.PBN_KERNEL_COMPILED, 1, _lib.PBN_COMPILE_WIDE, plan, 0))
                # wide states: the warp-split form in a few warp counts and occupancies,
                # each on its own plan object (a plan holds one compiled kernel), compiled
                # in parallel
                # (each of these compiles for tens of seconds on wide plans, so only at
                # one group size)
                if (warp_split_options and mi == warp_split_max_inputs
                        and (plan.info.state_words >= 4 or plan.info.n_sel_blocks > 24)):
                    # (on the scale-free network: 2 warps per CTA, ptxas -O3 and groups in
                    # batches of 4 ran 1.29x the interpreter; 4 or more warps, or -O1,
                    # ran slower than it)
                    ws = []
                    for extra in warp_split_options:
                        pw = api.Plan(red, max_inputs=mi, sampler=sampler)
                        ws.append((_lib.PBN_COMPILE_WARP_SPLIT | extra, pw))

                    def _compile(fp):
                        try:
                            fp[1].compile(fp[0])
                            return True
                        except _lib.PbnError:
                            return False
                    with ThreadPoolExecutor(max_workers=len(ws)) as ex:
                        ok = list(ex.map(_compile, ws))
                    cands += [(_lib.PBN_KERNEL_COMPILED, 1, f, pw, 0) for (f, pw), good in zip(ws, ok) if good]
            # at most about one lane per state word
            cands += [(_lib.PBN_KERNEL_INTERP, lg, 0, plan, 0) for lg in lanes_options
                      if lg == 1 or lg <= 2 * plan.info.state_words]
            if 2 * plan.info.state_words >= 8 and plan.info.semantics == _lib.PBN_SEM_EQ1:
                cands += [(_lib.PBN_KERNEL_TEAM, 0, 0, plan, k) for k in team_warps_options]
            for kern, lg, cf, pl, tw in cands:
                try:
                    if kern == _lib.PBN_KERNEL_COMPILED and not (cf & _lib.PBN_COMPILE_WARP_SPLIT):
                        pl.compile(cf)
                    dt = _time(pl, bufs, seed, steps, list(meta), kern, lg, tw)
                except _lib.PbnError:
                    continue
                rate = n * n_traj * steps / dt
                if log is not None:
                    log.append(dict(max_inputs=mi, smem_budget=budget, kernel=kern, lanes=lg, flags=cf, team_warps=tw,
                                    rate=rate,
                                    groups=int(plan.info.n_groups), tables_in_smem=int(plan.info.tables_in_smem)))
                if best is None or rate > best.node_updates_per_s:
                    best = Choice(max_inputs=mi, kernel=kern, lanes_per_traj=lg, smem_budget=budget,
                                  node_updates_per_s=rate, compile_flags=cf, team_warps=tw)
            del bufs
    if best is None:
        raise RuntimeError("no configuration could run this network")
    with _LOCK:
        _CACHE[key] = best
    if cache_file:
        try:
            saved = {}
            if os.path.exists(cache_file):
                with open(cache_file) as f:
                    saved = json.load(f)
            saved[key] = asdict(best)
            with open(cache_file, "w") as f:
                json.dump(saved, f, indent=1)
        except (OSError, ValueError):
            pass
    return best


def plan_for_choice(text: str, meta, ch: Choice, sampler: int = _lib.PBN_PERT_BITSLICED) -> api.Plan:
    red, _ = api.Net.load(text).reduce(list(meta))
    plan = api.Plan(red, max_inputs=ch.max_inputs, smem_budget=ch.smem_budget, sampler=sampler) if ch.smem_budget \
        else api.Plan(red, max_inputs=ch.max_inputs, sampler=sampler)
    if ch.kernel == _lib.PBN_KERNEL_COMPILED:
        plan.compile(ch.compile_flags)
    return plan


def tune_chunk(batch: api.Batch, total_steps: int, options=(250, 500, 1000, 2000), trial_steps: int = 2000):
    """Steps per persistent launch for a batch: time a CUDA-graph replay of
    trial_steps steps cut into chunks of each size (the batch's state advances; the
    caller re-initialises it afterwards if needed).  Returns (best chunk, timings)."""
    import torch
    timings = {}
    off = batch.steps_done
    for c in options:
        if c > total_steps:
            continue
        n = max(1, trial_steps // c)
        g = batch.capture([c] * n, step_offset=off)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        timings[c] = e0.elapsed_time(e1) / 1e3 / (n * c)
        off += n * c
    batch.steps_done = off
    best = min(timings, key=timings.get) if timings else options[0]
    return best, timings
