"""Parity of the CUDA path with the CPU oracle: bit-exact states and counts.

The oracle simulates the unreduced, ungrouped network by Eq. 1; the kernels run the
reduced, grouped plan (or the plain one-node-per-group plan).  Because every draw is
keyed by (trajectory, step, original node), every retained node's bit at every step
and every meta-state count must agree exactly.
"""
import os

import numpy as np
import pytest

from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare(gpu, orc, ids, trace=True):
    assert gpu["status"] == 0
    assert np.array_equal(gpu["final"][:, ids], orc["final"][:, ids])
    assert np.array_equal(gpu["counts"], orc["counts"])
    assert np.array_equal(gpu["pooled"], orc["counts"].sum(axis=0).astype(np.uint64))
    if trace:
        assert np.array_equal(gpu["trace"][:, :, ids], orc["trace"][:, :, ids])


@pytest.mark.parametrize("mode,reduce", [(0, True), (1, False), (1, True), (0, False)])
def test_tiny12_full_run_every_step(oracle_mod, mode, reduce):
    """n = 12, 64 trajectories x 10^4 steps, meta = nodes 0,1,2 ON: every state of
    every trajectory and every count equals the oracle's."""
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, mode=mode, reduce=reduce)
    orc = oracle_mod.simulate(text, 1, 0, 64, 10000, meta_ids=meta, trace=True, nthreads=NCPU)
    gpu = run(plan, seed=1, n_traj=64, n_steps=10000, meta=meta, trace=True)
    _compare(gpu, orc, ids)


@pytest.mark.parametrize("lanes,tpb", [(1, 32), (1, 96), (2, 16), (2, 64), (4, 8), (4, 40), (8, 4), (8, 64),
                                       (16, 2), (16, 10), (32, 1), (32, 16), (0, 0)])
def test_launch_shape_invariance(oracle_mod, lanes, tpb):
    """Lanes per trajectory and trajectories per CTA change nothing (ragged last CTA)."""
    net = synth.paper100(seed=2, p=2e-3)
    text = net.to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta)
    T, S = 333, 600
    orc = oracle_mod.simulate(text, 77, 1000, T, S, meta_ids=meta, count_from=13, nthreads=NCPU)
    gpu = run(plan, seed=77, traj_begin=1000, n_traj=T, n_steps=S, meta=meta, count_from=13,
              lanes=lanes, tpb=tpb)
    _compare(gpu, orc, ids, trace=False)


def test_resume_in_chunks_and_split_ranges(oracle_mod):
    """Chunked launches resumed from the device state, and disjoint trajectory ranges,
    reproduce one oracle run (checkpoint / resume and sharding by trajectory id)."""
    net = synth.paper100(seed=4, n=90, p=5e-3)
    text = net.to_text()
    meta = [0, 2]
    plan, ids = plan_for(text, meta)
    T, S = 200, 900
    orc = oracle_mod.simulate(text, 5, 0, T, S, meta_ids=meta, count_from=250, trace=True, nthreads=NCPU)
    a = run(plan, seed=5, n_traj=T, n_steps=S, meta=meta, count_from=250, chunks=[100, 150, 1, 649],
            trace=True)
    _compare(a, orc, ids)
    lo = run(plan, seed=5, n_traj=120, n_steps=S, meta=meta, count_from=250)
    hi = run(plan, seed=5, traj_begin=120, n_traj=80, n_steps=S, meta=meta, count_from=250)
    assert np.array_equal(np.concatenate([lo["final"], hi["final"]])[:, ids], orc["final"][:, ids])
    assert np.array_equal(np.concatenate([lo["counts"], hi["counts"]]), orc["counts"])


@pytest.mark.parametrize("mode", [0, 1])
def test_paper100_against_oracle(oracle_mod, mode):
    """Paper-scale network (n = 100, 25% sinks, p = 1e-4) grouped and plain."""
    text = synth.paper100(seed=2).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, mode=mode)
    T, S = 384, 4000
    orc = oracle_mod.simulate(text, 11, 0, T, S, meta_ids=meta, nthreads=NCPU)
    gpu = run(plan, seed=11, n_traj=T, n_steps=S, meta=meta)
    _compare(gpu, orc, ids, trace=False)


@pytest.mark.parametrize("lanes", [0, 32])
def test_scalefree2000_against_oracle(oracle_mod, lanes):
    """Large scale-free network (n = 2000, p = 1e-5, meta = 4 nodes)."""
    text = synth.scalefree2000(seed=3).to_text()
    meta = [0, 1, 2, 3]
    plan, ids = plan_for(text, meta)
    T, S = 64, 150
    orc = oracle_mod.simulate(text, 3, 0, T, S, meta_ids=meta, trace=True, nthreads=NCPU)
    gpu = run(plan, seed=3, n_traj=T, n_steps=S, meta=meta, trace=True, lanes=lanes)
    _compare(gpu, orc, ids)


def test_tables_in_global_memory(oracle_mod):
    """A plan whose tables exceed the shared-memory budget reads them from global
    memory and gives the same bits."""
    text = synth.paper100(seed=6, p=1e-3).to_text()
    meta = [1]
    import imgdecode
    base, _ = plan_for(text, meta)
    specs = imgdecode.decode(base.image())["H"]["off_tables"]
    plan, ids = plan_for(text, meta, smem_budget=max(1024, specs))
    assert plan.info.tables_in_smem == 0 and plan.info.stage_bytes == specs
    orc = oracle_mod.simulate(text, 8, 0, 256, 800, meta_ids=meta, nthreads=NCPU)
    gpu = run(plan, seed=8, n_traj=256, n_steps=800, meta=meta)
    _compare(gpu, orc, ids, trace=False)


@pytest.mark.parametrize("lanes", [1, 2, 8])
@pytest.mark.parametrize("tables", ["smem", "global"])
def test_split_nodes(oracle_mod, lanes, tables):
    """Multi-function nodes whose inputs exceed the merge cap keep one table per
    function (split nodes); only the selected function is evaluated."""
    text = synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11))).to_text()
    meta = [0, 1]
    kw = dict(max_inputs=3)
    if tables == "global":
        import imgdecode
        base, _ = plan_for(text, meta, **kw)
        kw["smem_budget"] = max(1024, imgdecode.decode(base.image())["H"]["off_tables"])
    plan, ids = plan_for(text, meta, **kw)
    assert plan.info.n_split > 0
    assert plan.info.tables_in_smem == (tables == "smem")
    orc = oracle_mod.simulate(text, 21, 0, 160, 400, meta_ids=meta, trace=True, nthreads=NCPU)
    gpu = run(plan, seed=21, n_traj=160, n_steps=400, meta=meta, trace=True, lanes=lanes,
              kernel=_lib.PBN_KERNEL_INTERP)
    _compare(gpu, orc, ids)


@pytest.mark.parametrize("kernel", [_lib.PBN_KERNEL_INTERP, _lib.PBN_KERNEL_COMPILED])
def test_reach_reduced_plan(oracle_mod, kernel):
    """The reachability rule (which also drops cycles that reach no meta node)
    gives the same bits on the kept nodes and the same counts as the oracle's
    unreduced simulation."""
    from paper_1605_00854_gb300 import api
    net = synth.random_pbn(4, 60, 0.01, k_choices=(1, 2, 3), sinks=0.2, protect=(0, 1, 2))
    # two extra nodes in a cycle that no other node reads: Definition 1 keeps them
    net.funcs.append([synth.Function(c=0.5, parents=[61, 5], tt=0b0110), synth.Function(c=0.5, parents=[61], tt=0b01)])
    net.funcs.append([synth.Function(c=1.0, parents=[60, 7], tt=0b1000)])
    net.n = 62
    text = net.to_text()
    meta = [0, 1, 2]
    red, ids = api.Net.load(text).reduce(meta, rule=_lib.PBN_REDUCE_REACH)
    _, ids_leaf = api.Net.load(text).reduce(meta)
    assert len(ids) < len(ids_leaf)
    plan = api.Plan(red)
    orc = oracle_mod.simulate(text, 5, 0, 128, 600, meta_ids=meta, trace=True, nthreads=NCPU)
    _compare(run(plan, seed=5, n_traj=128, n_steps=600, meta=meta, trace=True, kernel=kernel), orc, ids)


@pytest.mark.parametrize("p", [0.0, 0.05, 0.3, 0.75])
def test_perturbation_regimes(oracle_mod, p):
    """No perturbation, frequent, mostly and almost always perturbed steps."""
    text = synth.paper100(seed=9, n=70, p=p).to_text()
    meta = [0, 1]
    plan, ids = plan_for(text, meta)
    orc = oracle_mod.simulate(text, 2, 0, 96, 300, meta_ids=meta, trace=True, nthreads=NCPU)
    gpu = run(plan, seed=2, n_traj=96, n_steps=300, meta=meta, trace=True)
    _compare(gpu, orc, ids)


def test_edge_cases(oracle_mod):
    # one node, one trajectory
    text = "pbn 1 0x1p-3\nf 0 0x1p-1 1 0 2\nf 0 0x1p-1 1 0 1\n"
    plan, ids = plan_for(text, [0])
    orc = oracle_mod.simulate(text, 1, 0, 1, 500, meta_ids=[0], trace=True)
    _compare(run(plan, seed=1, n_traj=1, n_steps=500, meta=[0], trace=True), orc, ids)
    # zero steps: s(0) and the count of the first state only
    text = synth.tiny12(3).to_text()
    plan, ids = plan_for(text, [0, 1, 2])
    orc = oracle_mod.simulate(text, 4, 0, 50, 0, meta_ids=[0, 1, 2])
    _compare(run(plan, seed=4, n_traj=50, n_steps=0, meta=[0, 1, 2]), orc, ids, trace=False)
    # counting window beyond the end; meta values 0/1 mixed
    orc = oracle_mod.simulate(text, 4, 0, 50, 100, meta_ids=[0, 1, 2], meta_vals=[0, 1, 0],
                              count_from=1000)
    g = run(plan, seed=4, n_traj=50, n_steps=100, meta=[0, 1, 2], meta_vals=[0, 1, 0], count_from=1000)
    _compare(g, orc, ids, trace=False)
    assert int(g["counts"].sum()) == 0
    # large trajectory ids and step indices above 2^32, resumed from given states
    rng = np.random.default_rng(0)
    init = rng.integers(0, 2, size=(40, 12)).astype(np.uint8)
    tb, sb = 2**40 + 17, 2**33 + 5
    orc = oracle_mod.simulate(text, 2**63 + 9, tb, 40, 200, meta_ids=[1], step_begin=sb,
                              init_states=init, count_from=sb + 3, trace=True)
    g = run(plan, seed=2**63 + 9, traj_begin=tb, n_traj=40, n_steps=200, meta=[1], step_begin=sb,
            init_bits=init, count_from=sb + 3, trace=True)
    _compare(g, orc, ids)


def test_status_and_argument_errors():
    import torch
    from paper_1605_00854_gb300 import _lib, api
    text = synth.tiny12(1).to_text()
    plan, ids = plan_for(text, [0, 1, 2])
    bufs = api.alloc_buffers(plan, 64)
    with pytest.raises(_lib.PbnError):          # removed meta node
        removed = [i for i in range(12) if i not in set(ids.tolist())]
        if not removed:
            raise _lib.PbnError(-1, "skip")
        api.simulate(plan, bufs, seed=1, n_steps=10, meta_ids=[removed[0]])
    with pytest.raises(_lib.PbnError):          # keyed init needs step_begin == 0
        api.simulate(plan, bufs, seed=1, n_steps=10, meta_ids=[0], step_begin=5, init=0)
    with pytest.raises(_lib.PbnError):          # bad lanes
        api.simulate(plan, bufs, seed=1, n_steps=10, meta_ids=[0], lanes_per_traj=3)
    api.simulate(plan, bufs, seed=1, n_steps=10, meta_ids=[0])
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0


def test_apoptosis_stand_in_against_oracle(oracle_mod):
    """The apoptosis-shaped network (n = 96, 36 leaves) with a two-node meta-state:
    bit-exact against the oracle."""
    text = synth.apoptosis96().to_text()
    meta = [1, 37]
    plan, ids = plan_for(text, meta)
    assert len(ids) == 60
    orc = oracle_mod.simulate(text, 13, 0, 256, 2000, meta_ids=meta, count_from=100, nthreads=NCPU)
    for kernel in (_lib.PBN_KERNEL_INTERP, _lib.PBN_KERNEL_COMPILED):
        _compare(run(plan, seed=13, n_traj=256, n_steps=2000, meta=meta, count_from=100, kernel=kernel),
                 orc, ids, trace=False)



@pytest.mark.parametrize("lanes", [1, 4, 32])
@pytest.mark.parametrize("which", ["tiny12", "paper100"])
def test_nodewise_semantics(oracle_mod, lanes, which):
    """Node-wise perturbation semantics: every step applies the functions and the
    perturbed nodes negate; bit-exact against the oracle's node-wise simulator."""
    if which == "tiny12":
        text, meta = synth.tiny12(1).to_text(), [0, 1, 2]
    else:
        text, meta = synth.paper100(seed=2, p=5e-3).to_text(), [0, 1, 2]
    plan, ids = plan_for(text, meta, semantics=_lib.PBN_SEM_NODEWISE)
    orc = oracle_mod.simulate(text, 31, 0, 96, 700, meta_ids=meta, trace=True, nthreads=NCPU, semantics=1)
    gpu = run(plan, seed=31, n_traj=96, n_steps=700, meta=meta, trace=True, lanes=lanes,
              kernel=_lib.PBN_KERNEL_INTERP)
    _compare(gpu, orc, ids)
    # and it differs from Eq. 1 on the same draws
    eq1 = oracle_mod.simulate(text, 31, 0, 96, 700, meta_ids=meta, nthreads=NCPU)
    assert not np.array_equal(eq1["final"], orc["final"])



@pytest.mark.parametrize("lanes", [1, 4, 32])
@pytest.mark.parametrize("p", [0.0, 0.01, 0.3, 0.75])
def test_geometric_sampler(oracle_mod, lanes, p):
    """The geometric perturbation sampler: bit-exact against the oracle's
    geometric sampler (the rare path of several perturbed lanes per word runs
    often at large p); a partial last word (n = 150)."""
    text = synth.paper100(seed=12, n=150, p=p).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, sampler=_lib.PBN_PERT_GEOMETRIC)
    orc = oracle_mod.simulate(text, 41, 5, 96, 400, meta_ids=meta, trace=True, nthreads=NCPU, sampler=1)
    gpu = run(plan, seed=41, traj_begin=5, n_traj=96, n_steps=400, meta=meta, trace=True, lanes=lanes,
              kernel=_lib.PBN_KERNEL_INTERP)
    _compare(gpu, orc, ids)


def test_geometric_sampler_nodewise(oracle_mod):
    text = synth.tiny12(2).to_text()
    meta = [0, 1]
    plan, ids = plan_for(text, meta, sampler=_lib.PBN_PERT_GEOMETRIC, semantics=_lib.PBN_SEM_NODEWISE)
    orc = oracle_mod.simulate(text, 8, 0, 64, 800, meta_ids=meta, trace=True, semantics=1, sampler=1)
    _compare(run(plan, seed=8, n_traj=64, n_steps=800, meta=meta, trace=True, kernel=_lib.PBN_KERNEL_INTERP),
             orc, ids)


@pytest.mark.parametrize("kernel", [_lib.PBN_KERNEL_INTERP, _lib.PBN_KERNEL_COMPILED])
def test_trace_snapshots_with_a_stride(kernel):
    """Snapshots every 7th step equal every 7th row of the full trace."""
    import torch
    from paper_1605_00854_gb300 import api
    text = synth.paper100(seed=2, p=3e-3).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta)
    T, S, k = 96, 300, 7
    full = torch.zeros((S, plan.info.state_words, T), dtype=torch.int64, device="cuda")
    snap = torch.zeros((S // k, plan.info.state_words, T), dtype=torch.int64, device="cuda")
    for tr, st in ((full, 1), (snap, k)):
        bufs = api.alloc_buffers(plan, T)
        api.simulate(plan, bufs, seed=3, n_steps=S, meta_ids=meta, trace=tr, trace_stride=st, kernel=kernel)
    torch.cuda.synchronize()
    assert torch.equal(snap, full[k - 1:: k][: S // k])


@pytest.mark.parametrize("kernel", [_lib.PBN_KERNEL_INTERP, _lib.PBN_KERNEL_COMPILED])
@pytest.mark.parametrize("count_from", [0, 99, 100, 101, 250, 300])
def test_chain_cut_at_the_window_start(oracle_mod, kernel, count_from):
    """Launches chained from the device state count what one oracle run counts when
    the cuts fall just before, at and just after the start of the counting window
    (a meta-state that is ON at the cuts in some trajectories)."""
    text = synth.tiny12(1).to_text()
    meta = [11]
    plan, ids = plan_for(text, meta)
    if kernel == _lib.PBN_KERNEL_COMPILED:
        plan.compile(_lib.PBN_COMPILE_INTERLEAVED)
    T, S = 96, 300
    orc = oracle_mod.simulate(text, 21, 0, T, S, meta_ids=meta, count_from=count_from, nthreads=NCPU)
    got = run(plan, seed=21, n_traj=T, n_steps=S, meta=meta, count_from=count_from, chunks=[100, 150, 50],
              kernel=kernel)
    _compare(got, orc, ids, trace=False)


def test_first_launch_at_exactly_48_kb_of_dynamic_shared_memory():
    """A kernel's first launch asking for exactly 48 KB of dynamic shared memory
    (here a 104-node plan in CTAs of 480 trajectory slots) needs its opt-in raised,
    since the kernel's static shared memory comes on top of the dynamic part.  Run
    in a fresh process, where no earlier launch raised the limit, and compared with
    the oracle."""
    import subprocess
    import sys
    from conftest import ROOT
    code = """
import sys, numpy as np
sys.path.insert(0, %r)
sys.path.insert(0, %r)
from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import synth
from oracle import oracle
oracle.build()
text = synth.paper100(seed=2, n=104, p=1e-3).to_text()
plan, ids = plan_for(text, [0, 1, 2])
i = plan.info
per = 4 * (2 * (2 * i.state_words + 1) + (i.n_sel_blocks | 1))
assert (i.stage_bytes + 127) // 128 * 128 + per * 480 == 49152
got = run(plan, seed=6, n_traj=1000, n_steps=50, meta=[0, 1, 2], lanes=1, tpb=480, kernel=1)
orc = oracle.simulate(text, 6, 0, 1000, 50, meta_ids=[0, 1, 2])
assert got["status"] == 0
assert np.array_equal(got["final"][:, ids], orc["final"][:, ids])
assert np.array_equal(got["counts"], orc["counts"])
print("OK")
""" % (ROOT, os.path.join(ROOT, "tests"))
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0 and "OK" in p.stdout, (p.stdout + p.stderr)[-3000:]
