"""Benchmark: PBN node-updates/s of the reduced + grouped CUDA simulation.

Workload (one bench step = one pass of the whole hot path): the paper-scale network
(n = 100, 70% single-function nodes, in-degree 1-5, 25% sinks, p = 1e-4, meta-state
= nodes 0,1,2 ON), reduced and grouped (the autotuner picks the group input cap, the
kernel and its code shape, e.g. 12 inputs and the compiled interleaved plan with
multiply gathers), 2^16 trajectories x 10^6 steps per GPU from the keyed initial
state, with per-trajectory and pooled meta-state counts.  node-updates = n x
trajectories x steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n-steps S] [--n-traj T] [--sampler bitsliced|geometric]
                  [--workload paper100|scalefree2000|batch|serve|apoptosis]

Under torchrun each rank simulates its own trajectory-id range (weak scaling); the
timed region is bracketed by a barrier and device synchronisation and the maximum
over ranks is reported.  --impl reference times the CPU oracle (the plain Eq. 1
simulator of the unreduced network) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1605_00854_gb300 import _lib, api, autotune, shard, synth  # noqa: E402

SEED = 20160503
META = [0, 1, 2]
WORKLOAD = "paper-scale PBN n=100 (70% 1 function, 30% 2-3; in-degree 1-5; 25% sinks; p=1e-4), reduced+grouped"


# ------------------------------------------------------------------ helpers ----
def captured_traffic(src_hash: str, n_traj: int):
    """(DRAM bytes per launch, source file) of an ncu capture listed in profiles/*.md
    as `ncu-traffic: source-sha256=<hash> n_traj=<T> dram-bytes-per-launch=<bytes>`
    for this kernel source and trajectory count, else (None, None)."""
    import glob
    pat = re.compile(r"ncu-traffic: source-sha256=([0-9a-f]{64}) n_traj=(\d+) dram-bytes-per-launch=(\d+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == src_hash and int(m.group(2)) == n_traj:
                    return float(m.group(3)), f"ncu dram__bytes_read+write of this kernel source, {os.path.relpath(path, ROOT)}"
    return None, None


def captured_instructions(src_hash: str):
    """(warp instructions per warp-step, thread instructions per trajectory-step) of
    an ncu capture listed in profiles/*.md as `ncu-inst: source-sha256=<hash>
    warp-inst-per-warp-step=<w> thread-inst-per-traj-step=<t>`, else None."""
    import glob
    pat = re.compile(r"ncu-inst: source-sha256=([0-9a-f]{64}) warp-inst-per-warp-step=(\d+) "
                     r"thread-inst-per-traj-step=(\d+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == src_hash:
                    return float(m.group(2)), float(m.group(3))
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def expected_blocks(k: int) -> float:
    """Expected Philox blocks (2 levels each) to decide every lane of a k-lane
    perturbation word under early exit: a lane is undecided after L levels with
    probability 2^-L, independently, so E = sum_h P(some lane undecided after 2h levels)."""
    return sum(1.0 - (1.0 - 2.0 ** (-2 * h)) ** k for h in range(16))


def ops_per_traj_step(info, n: int, P: int) -> float:
    """Algorithmic 32-bit integer operations of one trajectory-step of the method
    (the per-unit figure of the roofline): Philox blocks at 56 ops (9 full rounds of
    2 mul.hi + 2 mul.lo + 2 xor3; round 1's products are shared per step), 12 ops per
    bit-sliced level pair, and in non-perturbed steps the SEL blocks, 2 ops per
    threshold compare-accumulate and 1 per multi node, 3 ops per group input
    (load, rotate, insert) and 5 per group (index, load, extract, shift, or; a split
    node adds 5 for its function record and reads its selected function's inputs),
    plus 8 ops of counting."""
    pe = P / 2**32
    W = (n + 63) // 64
    blocks = sum(expected_blocks(64 if w < W - 1 or n % 64 == 0 else n % 64) for w in range(W)) if P else 0.0
    pert = blocks * (56 + 12) + 4
    if info.sampler == _lib.PBN_PERT_GEOMETRIC:  # one block per word pair, a 64-bit compare per word
        pert = 56 * ((W + 1) // 2) + 4 * W + 4 if P else 4
    nonpert = (info.n_sel_blocks * 56 + 2 * info.total_thresholds + info.n_multi
               + 3 * info.total_inputs + 5 * (info.n_groups + info.n_split) + 2 * info.state_words)
    return pert + (1.0 - pe) ** n * nonpert + 8


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------- CPU oracle ----
def oracle_rate(text: str, n: int, target_s: float, meta=META):
    """Time the oracle on the host cores over a bounded sample: nthreads trajectories
    (one per core) for a number of steps calibrated to take about target_s."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    steps = 200
    t0 = time.perf_counter()
    oracle.simulate(text, SEED, 0, cores, steps, meta_ids=meta, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    steps = max(200, int(steps * target_s / dt))
    t0 = time.perf_counter()
    oracle.simulate(text, SEED, 0, cores, steps, meta_ids=meta, nthreads=cores)
    dt = time.perf_counter() - t0
    return n * cores * steps / dt, cores, f"{cores} trajectories x {steps} steps of the same network (unreduced, ungrouped Eq. 1 simulator)", dt


def oracle_rate_single(text: str, n: int, target_s: float, meta=META):
    """The same oracle on one host core (one trajectory)."""
    from oracle import oracle
    steps = 200
    t0 = time.perf_counter()
    oracle.simulate(text, SEED, 0, 1, steps, meta_ids=meta, nthreads=1)
    dt = max(time.perf_counter() - t0, 1e-3)
    steps = max(200, int(steps * target_s / dt))
    t0 = time.perf_counter()
    oracle.simulate(text, SEED, 0, 1, steps, meta_ids=meta, nthreads=1)
    return n * steps / (time.perf_counter() - t0), steps


def workload_network(args):
    """(network, meta nodes, description) of the single-network workloads."""
    if args.workload == "scalefree2000":
        return (synth.scalefree2000(seed=3), [0, 1, 2, 3],
                "scale-free PBN n=2000 (power-law out-degree 2.5; in-degree 1-6; 1-3 functions; p=1e-5), "
                "reduced+grouped")
    return synth.paper100(seed=2), META, WORKLOAD


KERNEL_NAMES = {_lib.PBN_KERNEL_COMPILED: "compiled", _lib.PBN_KERNEL_INTERP: "interpreter",
                _lib.PBN_KERNEL_TEAM: "team"}
SAMPLERS = {"bitsliced": _lib.PBN_PERT_BITSLICED, "geometric": _lib.PBN_PERT_GEOMETRIC}


# ------------------------------------------------------------------- ours ----
def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    net_obj, meta, workload = workload_network(args)
    text = net_obj.to_text()
    n = net_obj.n
    T = args.n_traj if args.n_traj else (1 << 16 if args.workload == "paper100" else 1 << 14)
    S = args.n_steps if args.n_steps else (10**6 if args.workload == "paper100" else 10**5)
    args.n_traj, args.n_steps = T, S
    lanes, team_warps = 0, 0
    tune_s = 0.0
    if args.compile_flags is not None or args.max_inputs:
        args.autotune = False  # a pinned configuration (for profiling runs)
    if args.autotune:
        # group size, kernel and lanes per trajectory picked by timing short passes
        t0 = time.perf_counter()
        choice = autotune.tune_network(text, meta, T, steps=2000 if args.workload == "paper100" else 200,
                                       sampler=SAMPLERS[args.sampler])
        tune_s = time.perf_counter() - t0
        max_inputs, lanes, team_warps = choice.max_inputs, choice.lanes_per_traj, choice.team_warps
        budget, cflags = choice.smem_budget, choice.compile_flags
        args.kernel = KERNEL_NAMES[choice.kernel]
    else:
        max_inputs, budget, cflags = args.max_inputs or 8, 0, args.compile_flags or 0
        lanes = args.lanes
    t_prep = time.perf_counter()
    red, retained = api.Net.load(text).reduce(meta)
    sampler = SAMPLERS[args.sampler]
    plan = api.Plan(red, max_inputs=max_inputs, smem_budget=budget, sampler=sampler) if budget \
        else api.Plan(red, max_inputs=max_inputs, sampler=sampler)
    compile_ms = 0.0
    kattrs = None
    if args.kernel == "compiled":
        try:
            compile_ms = plan.compile(cflags)
            kattrs = plan.compiled_attrs()
        except _lib.PbnError:
            args.kernel = "interpreter"  # plan too wide to compile: the interpreter runs it
    prep_s = time.perf_counter() - t_prep
    kern = {"compiled": _lib.PBN_KERNEL_COMPILED, "team": _lib.PBN_KERNEL_TEAM}.get(args.kernel, _lib.PBN_KERNEL_INTERP)
    P = api.Net.load(text).info().P
    info = plan.info
    T, S = args.n_traj, args.n_steps
    traj_begin, _ = shard.weak_range(rank, ws, T)
    d_img = plan.device_image(dev)
    bufs = api.alloc_buffers(plan, T, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def one_step():
        api.simulate(plan, bufs, seed=SEED, n_steps=S, meta_ids=meta, traj_begin=traj_begin,
                     stream=stream, d_image=d_img, kernel=kern, lanes_per_traj=lanes, team_warps=team_warps)

    for _ in range(args.warmup):
        bufs.counts.zero_(); bufs.pooled.zero_()
        one_step()
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0, "kernel status word set"

    times = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if ws == 1 else local) as clk:
        for _ in range(args.steps):
            bufs.counts.zero_(); bufs.pooled.zero_()
            flush.fill_(1)  # write 256 MiB (> L2) between timed steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total = sum(times)
    if ws > 1:
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    node_updates = n * T * S * ws * args.steps
    value = node_updates / total
    kernel_s = total / args.steps

    # end to end through the public API with host buffers: H2D of the plan image,
    # the simulation, D2H of states, counts and pooled counts, per step
    img_host = torch.from_numpy(plan.image()).pin_memory()
    st_h = torch.empty_like(bufs.state, device="cpu").pin_memory()
    cnt_h = torch.empty_like(bufs.counts, device="cpu").pin_memory()
    pool_h = torch.empty_like(bufs.pooled, device="cpu").pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    e_times = []
    for _ in range(e2e_steps):
        bufs.counts.zero_(); bufs.pooled.zero_()
        flush.fill_(1)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        d_img.copy_(img_host, non_blocking=True)
        one_step()
        st_h.copy_(bufs.state, non_blocking=True)
        cnt_h.copy_(bufs.counts, non_blocking=True)
        pool_h.copy_(bufs.pooled, non_blocking=True)
        torch.cuda.synchronize()
        e_times.append(time.perf_counter() - w0)
    e2e_total = sum(e_times)
    if ws > 1:
        t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = n * T * S * ws * e2e_steps / e2e_total

    compare = {}
    if rank == 0 and args.compare_steps > 0 and args.workload == "paper100":
        # the same workload on shorter passes: interpreter and the unmerged method
        # K0: unreduced, one node per group; K1: reduced, one node per group
        plain_plan = api.Plan(api.Net.load(text), mode=_lib.PBN_PLAN_PLAIN)
        reduced_plain = api.Plan(red, mode=_lib.PBN_PLAN_PLAIN)
        variants = [("interpreter_grouped", plan, _lib.PBN_KERNEL_INTERP),
                    ("compiled_plain_unreduced", plain_plan, _lib.PBN_KERNEL_COMPILED),
                    ("interpreter_plain_unreduced", plain_plan, _lib.PBN_KERNEL_INTERP),
                    ("compiled_plain_reduced", reduced_plain, _lib.PBN_KERNEL_COMPILED),
                    ("interpreter_plain_reduced", reduced_plain, _lib.PBN_KERNEL_INTERP)]
        # the same grouped plan compiled with each code-shape flag
        for fname, fl in (("rolled", 0), ("unrolled", _lib.PBN_COMPILE_PERT_UNROLLED),
                          ("interleaved", _lib.PBN_COMPILE_INTERLEAVED), ("pipelined", _lib.PBN_COMPILE_PIPELINED),
                          ("interleaved_magic_gather", _lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_COMPILE_MAGIC_GATHER)):
            pf = api.Plan(red, max_inputs=max_inputs)
            try:
                pf.compile(fl)
            except _lib.PbnError:
                continue
            variants.append((f"compiled_grouped_{fname}", pf, _lib.PBN_KERNEL_COMPILED))
        # the second perturbation sampler (a different draw contract, same law)
        pg = api.Plan(red, max_inputs=max_inputs, sampler=_lib.PBN_PERT_GEOMETRIC)
        try:
            pg.compile(_lib.PBN_COMPILE_INTERLEAVED)
            variants.append(("compiled_grouped_interleaved_geometric_sampler", pg, _lib.PBN_KERNEL_COMPILED))
        except _lib.PbnError:
            pass
        for name, pl, kk in variants:
            b2 = api.alloc_buffers(pl, T, dev)
            img2 = pl.device_image(dev)
            try:
                api.simulate(pl, b2, seed=SEED, n_steps=1000, meta_ids=meta, stream=stream, d_image=img2, kernel=kk)
            except _lib.PbnError as ex:  # a plan the compiled form does not take
                compare[name] = {"unavailable": str(ex)}
                continue
            torch.cuda.synchronize()
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            api.simulate(pl, b2, seed=SEED, n_steps=args.compare_steps, meta_ids=meta, stream=stream,
                         d_image=img2, kernel=kk)
            e1.record(stream)
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            compare[name] = {"value": n * T * args.compare_steps / dt, "unit": "node-updates/s",
                             "n_steps": args.compare_steps, "groups": int(pl.info.n_groups),
                             "achieved_tops": pl.info.ops_per_step * T * args.compare_steps / dt / 1e12}
            del b2

    out = None
    if rank == 0:
        pk, src = peaks()
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ops = ops_per_traj_step(info, n, P)
        achieved = ops * T * S / kernel_s / 1e12
        peak = sms * 128 * sm_max * 1e6 / 1e12
        clk_sum = clk.summary()
        # DRAM bytes per launch from an ncu capture of this very kernel (matched by the
        # SHA-256 of its generated source; a 2,000-step launch of the same trajectories:
        # the traffic is the state, counts and plan image, which does not grow with the
        # number of steps), else null
        traffic, traffic_note, issue = None, None, None
        if args.kernel == "compiled":
            src_hash = hashlib.sha256(plan.source(cflags).encode()).hexdigest()
            traffic, traffic_note = captured_traffic(src_hash, T)
            inst = captured_instructions(src_hash)
            if inst is not None:
                # issue slots: ncu's executed warp instructions per warp-step of this
                # kernel source x the warp-steps this launch ran, against every
                # scheduler issuing one warp instruction per clock
                wpi, tpi = inst
                warp_steps = math.ceil(T / 32) * S
                issued = wpi * warp_steps / kernel_s
                issue_peak = sms * 4 * sm_max * 1e6
                issue = {"warp_inst_per_warp_step": wpi, "thread_inst_per_traj_step": tpi,
                         "achieved_warp_inst_per_s": issued, "peak_warp_inst_per_s": issue_peak,
                         "frac": issued / issue_peak,
                         "note": "instruction counts from the ncu capture of this kernel source"}
        pooled = bufs.pooled.cpu().numpy().view(np.uint64)
        est = api.estimate(pooled, T, 0.01, 0.95)
        out = {
            "metric": "PBN node-updates/s (reduced+grouped kernel, bit-exact keyed draws)",
            "value": value, "unit": "node-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": kernel_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload, "n": n, "n_retained": int(info.n_retained),
                       "groups": int(info.n_groups), "n_traj_per_gpu": T, "n_steps": S,
                       "seed": SEED, "meta": meta, "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas{ws} (disjoint trajectory ids)",
                       "host_prep_s": round(prep_s, 4), "compile_ms": round(compile_ms, 1),
                       "kernel": args.kernel, "max_inputs_per_group": max_inputs,
                       "compile_flags": cflags if args.kernel == "compiled" else None,
                       "perturbation_sampler": args.sampler,
                       "compiled_kernel": kattrs,
                       "split_nodes": int(info.n_split),
                       "lanes_per_traj": lanes or "auto", "autotune_s": round(tune_s, 2)},
            "compare": compare,
            "traj_steps_per_s": T * S * ws * args.steps / total,
            "retained_node_updates_per_s": int(info.n_retained) * T * S * ws * args.steps / total,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "ops_per_traj_step": ops,
                         "peak_note": f"{sms} SMs x 128 int32 lanes x {sm_max:.0f} MHz ({src} max SM clock)",
                         "issue_slots": issue,
                         # the HBM side, for context: state, counts and plan image per launch
                         "hbm": None if traffic is None else {
                             "achieved_gbs": traffic / kernel_s / 1e9, "peak_gbs": float(pk.get("hbm_gbs", 6800.0)),
                             "frac": traffic / kernel_s / 1e9 / float(pk.get("hbm_gbs", 6800.0))}},
            "e2e": {"value": e2e_value, "unit": "node-updates/s",
                    "h2d_bytes_per_step": int(img_host.numel()),
                    "d2h_bytes_per_step": int(st_h.numel() * 8 + cnt_h.numel() * 8 + pool_h.numel() * 8)},
            "gpu_launches": args.steps,
            "clocks": clk_sum,
            "estimate": {"pi": est.pi, "alpha": est.alpha, "beta": est.beta, "n_star": est.n_star,
                         "L": est.L},
        }
    if ws > 1:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------- batched form ----
def _progress(msg: str):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def _timed(stream, fn):
    """CUDA-event seconds of fn() on `stream` after an L2 flush (a 256 MiB write)."""
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=stream.device)
    flush.fill_(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def measure_batch(args):
    """256 networks of the paper-scale generator with n log-uniform in [20, 4000],
    trajectories log-uniform in [1024, 65536] and p log-uniform in [1e-5, 1e-2],
    10^4 steps: the batched persistent launch (device work queue, chunks replayed from
    a CUDA graph; the autotuner picks the interpreted or compiled batch and the steps
    per launch) against one launch per network of the grouped plans (K2) and of the
    plain method (K0: unreduced, one node per group), each compiled where its plan
    compiles and interpreted otherwise, and both interpreted only."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    shapes = synth.batch_shapes(seed=4, count=args.batch_count)
    S = args.batch_steps
    S_each = min(S, args.batch_compare_steps)
    sampler = SAMPLERS[args.sampler]
    t0 = time.perf_counter()
    texts, entries, nu_step, ops_step = [], [], 0, 0.0
    for i, (n, T, p) in enumerate(shapes):
        text = synth.batch_network(seed=5000 + i, n=n, p=p).to_text()
        red, _ = api.Net.load(text).reduce(META)
        plan = api.Plan(red, sampler=sampler)
        entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, T, dev), seed=SEED + i, meta_ids=META))
        texts.append(text)
        nu_step += n * T
        ops_step += plan.info.ops_per_step * T
    prep_s = time.perf_counter() - t0
    _progress(f"batch: {len(shapes)} plans in {prep_s:.1f} s")

    def reset():
        for e in entries:
            e["bufs"].counts.zero_(); e["bufs"].pooled.zero_()

    # the two batched forms on a short trial; the faster one runs the workload
    forms = {}
    # the batched forms: the interpreter in CTAs of 512 or 1,024 threads, the compiled
    # batch (one module: compiled networks' functions and the interpreter) and the
    # split compiled batch (two persistent launches per chunk: the compiled networks,
    # then the rest in 1,024-thread CTAs)
    # (wide interpreted networks as teams of warps; the split batch also with lane
    # groups, for comparison)
    for form, flags, threads, lg in (
            ("interpreted", None, 512, False), ("interpreted_1024", None, 1024, False),
            ("compiled", _lib.PBN_COMPILE_INTERLEAVED, 512, False),
            ("compiled_split", _lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_BATCH_SPLIT, 512, False),
            ("compiled_split_lane_groups", _lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_BATCH_SPLIT, 512, True)):
        t0 = time.perf_counter()
        B = api.Batch(entries, device=dev, compile_flags=flags, threads=threads, lane_groups=lg)
        build_s = time.perf_counter() - t0
        B.run(20, step_offset=0)
        torch.cuda.synchronize()
        trial = min(S, args.batch_trial_steps)
        dt = _timed(stream, lambda: B.run(trial, step_offset=0))
        forms[form] = dict(batch=B, trial_rate=nu_step * trial / dt, build_s=build_s,
                           n_compiled=int(B.info.n_compiled), n_team=int(B.info.n_team),
                           work_items=int(B.info.n_items))
        _progress(f"batch: {form} form built in {build_s:.1f} s, trial {nu_step * trial / dt:.3e}")
    best = max(forms, key=lambda f: forms[f]["trial_rate"])
    B = forms[best]["batch"]
    # steps per launch: CUDA-graph replays of one trial length cut into chunks
    chunk, chunk_t = autotune.tune_chunk(B, S, options=tuple(c for c in (250, 500, 1000, 2500) if c <= S),
                                         trial_steps=min(S, args.batch_trial_steps))
    reset()
    chunks = [chunk] * (S // chunk) + ([S % chunk] if S % chunk else [])
    g = B.capture(chunks, step_offset=0)
    _progress(f"batch: chunk {chunk} steps")
    t_batch = _timed(stream, g.replay)
    _progress(f"batch: timed {S} steps in {t_batch:.1f} s")
    assert int(B.status.item()) == 0, "batch kernel status word set"
    value = nu_step * S / t_batch

    # one launch per network: grouped (K2) and plain (K0) plans, compiled where they
    # compile (compilation before the timed region), else the interpreter
    plain = []
    for i, (n, T, p) in enumerate(shapes):
        try:
            pp = api.Plan(api.Net.load(texts[i]), mode=_lib.PBN_PLAN_PLAIN, sampler=sampler)
        except _lib.PbnError:  # plain specs that exceed shared memory: left out
            pp = None
        plain.append(pp)

    def try_compile(pl):
        if pl is None:
            return False
        try:
            pl.compile(_lib.PBN_COMPILE_INTERLEAVED)
            return True
        except _lib.PbnError:
            return False
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        k2_ok = list(ex.map(try_compile, [e["plan"] for e in entries]))
        k0_ok = list(ex.map(try_compile, plain))
    compile_each_s = time.perf_counter() - t0
    _progress(f"batch: per-network plans compiled in {compile_each_s:.1f} s")
    plain_bufs = [api.alloc_buffers(pp, T, dev) if pp is not None else None for pp, (n, T, p) in zip(plain, shapes)]

    def each(plans, bufs, kernels):
        """One launch per network with its kernel; a team launch that does not fit
        the network (its records and one team beyond shared memory) falls back to the
        lane-group interpreter during the warm-up."""
        nu = 0
        launches = []
        for i, (pl, bf, kk) in enumerate(zip(plans, bufs, kernels)):
            if pl is None:
                continue
            nu += shapes[i][0] * shapes[i][1] * S_each
            launches.append([pl, bf, kk, entries[i]["seed"]])
        for ln in launches:  # warm (first launches, shape queries)
            try:
                api.simulate(ln[0], ln[1], seed=ln[3], n_steps=8, meta_ids=META, stream=stream, kernel=ln[2])
            except _lib.PbnError:
                if ln[2] != _lib.PBN_KERNEL_TEAM:
                    raise
                ln[2] = _lib.PBN_KERNEL_INTERP
                api.simulate(ln[0], ln[1], seed=ln[3], n_steps=8, meta_ids=META, stream=stream, kernel=ln[2])

        def go(steps):
            for pl, bf, kk, sd in launches:
                api.simulate(pl, bf, seed=sd, n_steps=steps, meta_ids=META, stream=stream, kernel=kk)
        torch.cuda.synchronize()
        dt = _timed(stream, lambda: go(S_each))
        _progress(f"batch: per-network leg {dt:.1f} s")
        return {"value": nu / dt, "unit": "node-updates/s", "seconds": dt, "networks": len(launches),
                "n_steps": S_each, "team_networks": sum(1 for ln in launches if ln[2] == _lib.PBN_KERNEL_TEAM)}
    C, I, TM = _lib.PBN_KERNEL_COMPILED, _lib.PBN_KERNEL_INTERP, _lib.PBN_KERNEL_TEAM

    def interp(pl):
        """The interpreter a network runs best: teams for states of 8 rows or more
        (Eq. 1 semantics), lane groups otherwise."""
        if pl is None:
            return I
        wide = 2 * pl.info.state_words >= 8 and pl.info.semantics == _lib.PBN_SEM_EQ1
        return TM if wide else I
    grouped = [e["plan"] for e in entries]
    gbufs = [e["bufs"] for e in entries]
    legs = {
        "compiled_grouped": each(grouped, gbufs, [C if ok else interp(pl) for ok, pl in zip(k2_ok, grouped)]),
        "interpreted_grouped": each(grouped, gbufs, [interp(pl) for pl in grouped]),
        "interpreted_grouped_lane_groups": each(grouped, gbufs, [I] * len(grouped)),
        "compiled_plain": each(plain, plain_bufs, [C if ok else interp(pl) for ok, pl in zip(k0_ok, plain)]),
        "interpreted_plain": each(plain, plain_bufs, [interp(pl) for pl in plain]),
    }
    legs["compiled_grouped"]["compiled_networks"] = int(sum(k2_ok))
    legs["compiled_plain"]["compiled_networks"] = int(sum(k0_ok))
    best_plain = max(legs["compiled_plain"]["value"], legs["interpreted_plain"]["value"])
    best_grouped = max(legs[k]["value"] for k in ("compiled_grouped", "interpreted_grouped",
                                                  "interpreted_grouped_lane_groups"))
    pk, _ = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = ops_step * S / t_batch / 1e12
    return {
        "metric": "PBN node-updates/s, batched persistent launch vs one launch per network",
        "value": value, "unit": "node-updates/s", "seconds": t_batch,
        "workload": f"batch of {len(shapes)} paper-scale PBNs, n log-uniform [20,4000], trajectories log-uniform "
                    "[1024,65536], p log-uniform [1e-5,1e-2]",
        "n_steps": S, "form": best, "chunk_steps": chunk, "launches": len(chunks),
        "autotune": {"forms": {f: {k: v for k, v in d.items() if k != "batch"} for f, d in forms.items()},
                     "chunk_seconds_per_step": {str(k): v for k, v in chunk_t.items()}},
        "threads_per_cta": int(B.info.threads), "smem_per_cta": int(B.info.smem_bytes),
        "graph": "chunk launches captured in one CUDA graph", "host_prep_s": round(prep_s, 2),
        "per_network": legs, "per_network_compile_s": round(compile_each_s, 2),
        "speedup_vs_plain_per_network": value / best_plain,
        "speedup_vs_grouped_per_network": value / best_grouped,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s", "frac": achieved / peak,
                     "ops_per_step": ops_step, "traffic": None,
                     "note": "algorithmic ops of every network's plan x trajectories x steps / CUDA-event time"},
    }


def run_batch(args):
    out = measure_batch(args)
    line = {"metric": out["metric"], "value": out["value"], "unit": out["unit"], "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": out["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": {"workload": out["workload"]},
            "batch": out}
    print(json.dumps(line), flush=True)


def measure_serve(args):
    """Poisson query arrivals (rate per second for a duration), each a fresh PBN of the
    paper-scale generator with n log-uniform in [30, 3000] and a meta-state of 1-4
    nodes, precision r = 0.01 at 95% confidence, served with continuous batching."""
    import multiprocessing
    from paper_1605_00854_gb300 import serve
    rng = np.random.default_rng(5)
    n_q = int(args.serve_rate * args.serve_seconds)
    gaps = rng.exponential(1.0 / args.serve_rate, size=n_q)
    shapes, metas = [], []
    for i in range(n_q):
        n = int(round(math.exp(rng.uniform(math.log(30), math.log(3000)))))
        k = int(rng.integers(1, 5))
        metas.append(sorted(int(x) for x in rng.choice(4, size=k, replace=False)))
        shapes.append((9000 + i, n, float(10 ** rng.uniform(-4, -2))))
    # the client: query networks written by worker processes (spawned, so they hold
    # no CUDA state) ahead of the arrival clock, in arrival order
    ctx = multiprocessing.get_context("spawn")
    gen = ctx.Pool(processes=max(2, min(8, (os.cpu_count() or 4) // 2)))
    texts = gen.imap(synth.query_text_args, shapes, chunksize=8)
    ahead = [next(texts) for _ in range(min(n_q, int(2 * args.serve_rate)))]  # two seconds of arrivals
    _progress(f"serve: {n_q} queries, generation under way")

    def query(i):
        text = ahead[i] if i < len(ahead) else next(texts)
        return serve.Query(qid=i, text=text, meta_ids=metas[i], seed=SEED + i, r=0.01, s=0.95)
    srv = serve.Server(n_traj=args.serve_traj, chunk_steps=args.serve_chunk, mem_cap_bytes=100e9,
                       workers=os.cpu_count() or 8, max_traj=args.serve_max_traj, kernel=args.serve_kernel,
                       sampler=SAMPLERS[args.sampler])
    t_start = time.perf_counter()
    due = t_start + np.cumsum(gaps)
    k = 0
    # arrivals for serve_seconds, then at most 60 s more to finish what is in flight;
    # queries still open then are reported as unfinished
    t_limit = t_start + args.serve_seconds + 60
    last = t_start
    while (k < n_q or srv.pending) and time.perf_counter() < t_limit:
        now = time.perf_counter()
        while k < n_q and due[k] <= now:
            q = query(k)
            q.arrival = due[k]
            srv.submit(q)
            k += 1
        if not srv.step():
            time.sleep(0.0005)
        if time.perf_counter() - last > 30:
            last = time.perf_counter()
            _progress(f"serve: {k} submitted, {len(srv.done)} done, {len(srv.active)} active, "
                      f"{len(srv.waiting)} waiting")
    makespan = time.perf_counter() - t_start
    srv.close()
    gen.terminate()
    lat = serve.latency_summary(srv.done)
    st = dict(srv.stats)
    return {"metric": "served steady-state queries: p50/p99 latency, queries/s, node-updates/s",
            "workload": "Poisson queries, n log-uniform [30,3000], meta 1-4 nodes, r=0.01, s=0.95 "
                        "(each a fresh paper-scale network, synth.query_text)",
            "rate_per_s": args.serve_rate, "seconds": args.serve_seconds, "queries": n_q,
            "trajectories_per_query": args.serve_traj, "max_trajectories_per_query": args.serve_max_traj,
            "chunk_steps": args.serve_chunk, "memory_cap_bytes": 100e9, "kernel": args.serve_kernel,
            "p50_s": lat.get("p50_s"), "p99_s": lat.get("p99_s"), "latency": lat,
            "queries_per_s": len(srv.done) / makespan, "node_updates_per_s": srv.node_updates / makespan,
            "makespan_s": makespan, "device_busy_frac": st.get("device_s", 0.0) / makespan,
            "completed": len(srv.done), "rejected": len(srv.rejected), "failed": len(srv.failed),
            "unfinished": n_q - len(srv.done) - len(srv.rejected) - len(srv.failed) - len(srv.cancelled),
            "rounds": st, "mean_prep_s": float(np.mean([r.prep_s for r in srv.done])) if srv.done else None}


def run_serve(args):
    out = measure_serve(args)
    line = {"metric": out["metric"], "value": out["p99_s"], "unit": "s (p99 latency)", "higher_is_better": False,
            "n_gpus": 1, "dtype": "u32", "data": "synthetic", "config": {"workload": out["workload"]}, "serve": out}
    print(json.dumps(line), flush=True)


def measure_scalefree(args):
    """One pass of the scale-free network (n = 2000, 2^14 trajectories x 10^5 steps)
    in the autotuner's configuration, with its roofline."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    net = synth.scalefree2000(seed=3)
    text, meta, n = net.to_text(), [0, 1, 2, 3], net.n
    T, S = 1 << 14, args.scalefree_steps
    t0 = time.perf_counter()
    ch = autotune.tune_network(text, meta, T, steps=200, sampler=SAMPLERS[args.sampler])
    tune_s = time.perf_counter() - t0
    plan = autotune.plan_for_choice(text, meta, ch, sampler=SAMPLERS[args.sampler])
    bufs = api.alloc_buffers(plan, T, dev)
    img = plan.device_image(dev)
    run = lambda steps: api.simulate(plan, bufs, seed=SEED, n_steps=steps, meta_ids=meta, stream=stream,
                                     d_image=img, kernel=ch.kernel, lanes_per_traj=ch.lanes_per_traj,
                                     team_warps=ch.team_warps)
    run(200)
    torch.cuda.synchronize()
    bufs.counts.zero_(); bufs.pooled.zero_()
    dt = _timed(stream, lambda: run(S))
    assert int(bufs.status.item()) == 0
    P = api.Net.load(text).info().P
    ops = ops_per_traj_step(plan.info, n, P)
    pk, _ = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = ops * T * S / dt / 1e12
    return {"workload": "scale-free PBN n=2000 (power-law out-degree 2.5; in-degree 1-6; 1-3 functions; "
                        "p=1e-5), reduced+grouped", "n_traj": T, "n_steps": S,
            "value": n * T * S / dt, "unit": "node-updates/s", "seconds": dt,
            "kernel": KERNEL_NAMES[ch.kernel], "team_warps": ch.team_warps,
            "lanes_per_traj": ch.lanes_per_traj, "max_inputs_per_group": ch.max_inputs,
            "compile_flags": ch.compile_flags, "groups": int(plan.info.n_groups),
            "n_retained": int(plan.info.n_retained), "autotune_s": round(tune_s, 1),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                         "frac": achieved / peak, "ops_per_traj_step": ops, "traffic": None}}


def apoptosis_queries():
    """The seven meta-states of the apoptosis-shaped workload: for a core node X with
    three parents A, B, C (the shape of the paper's analysis of one node and its three
    parents), P(A), P(B), P(C), P(X and A), P(X and B), P(X and C) and P(X), all ON."""
    net = synth.apoptosis96()
    core = 60
    for X in range(core):
        par = sorted({a for f in net.funcs[X] for a in f.parents if a != X and a < core})
        if len(par) >= 3:
            A, B, C = par[:3]
            break
    metas = [[A], [B], [C], [X, A], [X, B], [X, C], [X]]
    return net, X, (A, B, C), metas


def run_apoptosis(args):
    """Seven steady-state probabilities of the apoptosis-shaped network at precision
    r = 1e-5 and confidence 0.95 (Sec. 4.2's setting), estimated together by the
    two-state Markov chain stopping rule through the serving loop."""
    from paper_1605_00854_gb300 import serve
    net, X, par, metas = apoptosis_queries()
    text = net.to_text()
    srv = serve.Server(n_traj=args.apo_traj, chunk_steps=args.apo_chunk, burn_in0=256,
                       mem_cap_bytes=100e9, workers=8, max_steps=1 << 24, max_traj=args.apo_max_traj,
                       kernel=args.serve_kernel, sampler=SAMPLERS[args.sampler])
    t0 = time.perf_counter()
    for i, m in enumerate(metas):
        srv.submit(serve.Query(qid=i, text=text, meta_ids=m, seed=SEED + 17 * i, r=1e-5, s=0.95, eps=1e-3))
    srv.drain(timeout=args.apo_timeout)
    wall = time.perf_counter() - t0
    srv.close()
    res = sorted(srv.done, key=lambda r: r.qid)
    samples = sum(r.L for r in res)
    line = {"metric": "apoptosis-shaped network: 7 steady-state probabilities at r=1e-5, s=0.95 (wall time)",
            "value": wall, "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "u32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "apoptosis-shaped PBN: n=96, 37.5% leaves, density 1.78, p=1e-4",
                       "node_X": X, "parents_ABC": list(par), "trajectories_per_query": args.apo_traj,
                       "max_trajectories_per_query": args.apo_max_traj, "kernel": args.serve_kernel,
                       "perturbation_sampler": args.sampler,
                       "chunk_steps": args.apo_chunk, "r": 1e-5, "s": 0.95, "eps": 1e-3},
            "queries": [{"meta": metas[r.qid], "pi": r.pi, "n_star": r.n_star, "samples": r.L, "m_star": r.m_star,
                         "steps": r.steps, "rounds": r.rounds, "trajectories": r.n_traj, "latency_s": r.latency}
                        for r in res],
            "total_samples": samples, "node_updates_per_s": srv.node_updates / wall, "rounds": srv.stats,
            "completed": len(res), "failed": len(srv.failed),
            "paper_context": "Sec. 4.2: 7 probabilities, 50-452 million samples each, about 10 minutes "
                             "in total for the structure-based method on the paper's CPU (other hardware)"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-traj", type=int, default=0, help="trajectories per GPU (default per workload)")
    ap.add_argument("--n-steps", type=int, default=0, help="steps per pass (default per workload)")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default="compiled", choices=["compiled", "interpreter", "team"])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use group size 8 and the default launch shape instead of the autotuner")
    ap.add_argument("--max-inputs", type=int, default=0, help="pin the group input cap (skips the autotuner)")
    ap.add_argument("--compile-flags", type=int, default=None, help="pin pbn_plan_compile flags (skips the autotuner)")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per trajectory when the autotuner is skipped")
    ap.add_argument("--workload", default="paper100",
                    choices=["paper100", "scalefree2000", "batch", "serve", "apoptosis"])
    ap.add_argument("--apo-traj", type=int, default=1 << 14)
    ap.add_argument("--apo-max-traj", type=int, default=1 << 17)
    ap.add_argument("--apo-chunk", type=int, default=4096)
    ap.add_argument("--apo-timeout", type=float, default=600.0)
    ap.add_argument("--extras", default="batch,serve,scalefree2000",
                    help="sub-measurements added to the default line at N=1 (comma list, or 'none')")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=10**4)
    ap.add_argument("--batch-compare-steps", type=int, default=2000,
                    help="steps of each per-network comparison leg")
    ap.add_argument("--batch-trial-steps", type=int, default=1000,
                    help="steps of the autotuner's trials (batched form, steps per launch)")
    ap.add_argument("--scalefree-steps", type=int, default=10**5)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=300.0)
    ap.add_argument("--serve-traj", type=int, default=2048)
    ap.add_argument("--serve-kernel", default="auto", choices=["batch", "auto"],
                    help="serving rounds: batched interpreter only, or compiled plans for large blocks")
    ap.add_argument("--sampler", default="bitsliced", choices=["bitsliced", "geometric"],
                    help="perturbation sampler (draw contract) of the plans")
    ap.add_argument("--serve-chunk", type=int, default=128)
    ap.add_argument("--serve-max-traj", type=int, default=1 << 16)
    ap.add_argument("--compare-steps", type=int, default=100000,
                    help="steps of the comparison passes (interpreter, plain method); 0 = skip")
    args = ap.parse_args()
    ws, rank, _ = dist_env()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "apoptosis":
        return run_apoptosis(args)

    net_obj = synth.paper100(seed=2)
    text = net_obj.to_text()
    n = net_obj.n

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        last = None
        for i in range(args.warmup + args.steps):
            rate, cores, sample, dt = oracle_rate(text, n, args.oracle_seconds / 2)
            if i >= args.warmup:
                vals.append((rate, dt))
            last = (cores, sample)
        total_t = sum(d for _, d in vals)
        value = sum(r * d for r, d in vals) / total_t
        line = {"metric": "PBN node-updates/s (reduced+grouped kernel, bit-exact keyed draws)",
                "value": value, "unit": "node-updates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(vals),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD, "n": n, "n_traj_per_gpu": args.n_traj or (1 << 16),
                           "n_steps": args.n_steps or 10**6, "seed": SEED, "meta": META,
                           "parallelism": "host cores (trajectories split over threads)"},
                "cpu_baseline": {"value": value, "unit": "node-updates/s", "cores": last[0],
                                 "kind": "oracle", "sample": last[1]},
                "e2e": {"value": value, "unit": "node-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    t_run = time.perf_counter()
    out = run_ours(args)
    if rank == 0:
        print(f"[bench] headline: {time.perf_counter() - t_run:.1f} s", file=sys.stderr, flush=True)
    if rank == 0 and out is not None:
        extras = [] if args.extras in ("", "none") else args.extras.split(",")
        measures = {"batch": measure_batch, "serve": measure_serve, "scalefree2000": measure_scalefree}
        for name in extras if ws == 1 else []:
            # the batched / served forms and the scale-free network, measured after the
            # headline's timed region (one GPU; under torchrun only the headline runs)
            t_leg = time.perf_counter()
            try:
                out[name] = measures[name](args)
            except Exception as exc:  # a leg that cannot run reports why
                out[name] = {"error": f"{type(exc).__name__}: {exc}"}
            out[name]["leg_wall_s"] = round(time.perf_counter() - t_leg, 1)
            print(f"[bench] {name}: {out[name]['leg_wall_s']} s", file=sys.stderr, flush=True)
        if not args.no_cpu_baseline and ws == 1:
            rate, cores, sample, dt = oracle_rate(text, n, args.oracle_seconds)
            r1, s1 = oracle_rate_single(text, n, min(3.0, args.oracle_seconds / 4))
            out["cpu_baseline"] = {"value": rate, "unit": "node-updates/s", "cores": cores,
                                   "kind": "oracle", "sample": sample, "seconds": round(dt, 2),
                                   "single_core": {"value": r1, "sample": f"1 trajectory x {s1} steps"}}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
