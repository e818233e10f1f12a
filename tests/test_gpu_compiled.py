"""Parity of compiled plans (the plan's own kernel, generated and built with NVRTC)
with the CPU oracle and with the interpreter kernel: bit-exact states and counts."""
import os

import numpy as np
import pytest

from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
COMPILED = _lib.PBN_KERNEL_COMPILED
INTERP = _lib.PBN_KERNEL_INTERP


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


@pytest.mark.parametrize("mode,reduce", [(0, True), (1, False)])
def test_tiny12_compiled_every_step(oracle_mod, mode, reduce):
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, mode=mode, reduce=reduce)
    ms = plan.compile()
    assert ms > 0
    orc = oracle_mod.simulate(text, 1, 0, 64, 10000, meta_ids=meta, trace=True, nthreads=NCPU)
    _compare(run(plan, seed=1, n_traj=64, n_steps=10000, meta=meta, trace=True, kernel=COMPILED), orc, ids)


@pytest.mark.parametrize("mode,flags", [(0, 0), (1, 0), (0, 4)])
def test_paper100_compiled_matches_oracle_and_interpreter(oracle_mod, mode, flags):
    text = synth.paper100(seed=2).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, mode=mode)
    plan.compile(flags)
    T, S = 1000, 3000
    orc = oracle_mod.simulate(text, 11, 77, T, S, meta_ids=meta, count_from=100, nthreads=NCPU)
    c = run(plan, seed=11, traj_begin=77, n_traj=T, n_steps=S, meta=meta, count_from=100, kernel=COMPILED)
    i = run(plan, seed=11, traj_begin=77, n_traj=T, n_steps=S, meta=meta, count_from=100, kernel=INTERP)
    _compare(c, orc, ids, trace=False)
    _compare(i, orc, ids, trace=False)


@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_PIPELINED])
def test_compiled_resume_and_keyed_init(oracle_mod, flags):
    text = synth.paper100(seed=4, n=90, p=5e-3).to_text()
    meta = [0, 2]
    plan, ids = plan_for(text, meta)
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 5, 0, 200, 900, meta_ids=meta, count_from=250, trace=True, nthreads=NCPU)
    a = run(plan, seed=5, n_traj=200, n_steps=900, meta=meta, count_from=250, chunks=[100, 150, 1, 649],
            trace=True, kernel=COMPILED)
    _compare(a, orc, ids)


@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_PERT_UNROLLED, _lib.PBN_COMPILE_INTERLEAVED,
                                   _lib.PBN_COMPILE_PIPELINED])
@pytest.mark.parametrize("p", [0.0, 0.05, 0.3, 0.75])
def test_compiled_perturbation_regimes(oracle_mod, p, flags):
    text = synth.paper100(seed=9, n=170, p=p).to_text()
    meta = [0, 1]
    plan, ids = plan_for(text, meta)
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 2, 0, 96, 300, meta_ids=meta, trace=True, nthreads=NCPU)
    _compare(run(plan, seed=2, n_traj=96, n_steps=300, meta=meta, trace=True, kernel=COMPILED), orc, ids)


@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_PIPELINED])
def test_compiled_edge_cases(oracle_mod, flags):
    text = "pbn 1 0x1p-3\nf 0 0x1p-1 1 0 2\nf 0 0x1p-1 1 0 1\n"
    plan, ids = plan_for(text, [0])
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 1, 0, 1, 500, meta_ids=[0], trace=True)
    _compare(run(plan, seed=1, n_traj=1, n_steps=500, meta=[0], trace=True, kernel=COMPILED), orc, ids)
    text = synth.tiny12(3).to_text()
    plan, ids = plan_for(text, [0, 1, 2])
    plan.compile(flags)
    rng = np.random.default_rng(0)
    init = rng.integers(0, 2, size=(40, 12)).astype(np.uint8)
    tb, sb = 2**40 + 17, 2**33 + 5
    orc = oracle_mod.simulate(text, 2**63 + 9, tb, 40, 200, meta_ids=[1], meta_vals=[0], step_begin=sb,
                              init_states=init, count_from=sb + 3, trace=True)
    g = run(plan, seed=2**63 + 9, traj_begin=tb, n_traj=40, n_steps=200, meta=[1], meta_vals=[0],
            step_begin=sb, init_bits=init, count_from=sb + 3, trace=True, kernel=COMPILED)
    _compare(g, orc, ids)
    orc = oracle_mod.simulate(text, 4, 0, 50, 0, meta_ids=[0, 1, 2])
    _compare(run(plan, seed=4, n_traj=50, n_steps=0, meta=[0, 1, 2], kernel=COMPILED), orc, ids, trace=False)


def test_compiled_global_tables(oracle_mod):
    """A network whose merged tables exceed 48 KiB reads them from global memory."""
    text = synth.paper100(seed=7, n=300, p=1e-3).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, max_inputs=12)
    assert plan.info.table_bytes > 48 * 1024
    plan.compile()
    orc = oracle_mod.simulate(text, 3, 0, 128, 400, meta_ids=meta, nthreads=NCPU)
    _compare(run(plan, seed=3, n_traj=128, n_steps=400, meta=meta, kernel=COMPILED), orc, ids, trace=False)


@pytest.mark.parametrize("kmax", [5, 10])
def test_compiled_split_nodes(oracle_mod, kmax):
    """Split nodes in a compiled plan: function tables as immediates (k <= 6) or one
    lookup at the selected function's table."""
    text = synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, kmax + 1))).to_text()
    meta = [0, 1]
    plan, ids = plan_for(text, meta, max_inputs=3)
    assert plan.info.n_split > 0
    plan.compile()
    orc = oracle_mod.simulate(text, 21, 0, 160, 400, meta_ids=meta, trace=True, nthreads=NCPU)
    _compare(run(plan, seed=21, n_traj=160, n_steps=400, meta=meta, trace=True, kernel=COMPILED), orc, ids)



@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_INTERLEAVED, _lib.PBN_COMPILE_PIPELINED])
def test_compiled_nodewise_semantics(oracle_mod, flags):
    text = synth.paper100(seed=2, p=5e-3).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, semantics=_lib.PBN_SEM_NODEWISE)
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 32, 0, 160, 600, meta_ids=meta, trace=True, nthreads=NCPU, semantics=1)
    _compare(run(plan, seed=32, n_traj=160, n_steps=600, meta=meta, trace=True, kernel=COMPILED), orc, ids)



@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_INTERLEAVED, _lib.PBN_COMPILE_PIPELINED])
def test_compiled_kernel_attributes(flags):
    text = synth.paper100(seed=2).to_text()
    plan, _ = plan_for(text, [0, 1, 2])
    plan.compile(flags)
    a = plan.compiled_attrs()
    assert a["flags"] == flags and 16 <= a["regs"] <= 255



@pytest.mark.parametrize("flags", [0, _lib.PBN_COMPILE_INTERLEAVED, _lib.PBN_COMPILE_PIPELINED])
@pytest.mark.parametrize("p", [0.01, 0.3])
def test_compiled_geometric_sampler(oracle_mod, flags, p):
    text = synth.paper100(seed=12, n=150, p=p).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, sampler=_lib.PBN_PERT_GEOMETRIC)
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 41, 0, 128, 400, meta_ids=meta, trace=True, nthreads=NCPU, sampler=1)
    _compare(run(plan, seed=41, n_traj=128, n_steps=400, meta=meta, trace=True, kernel=COMPILED), orc, ids)



@pytest.mark.parametrize("which", ["tiny12", "paper100", "paper100_mi12", "nodewise", "geometric", "split"])
@pytest.mark.parametrize("flags", [_lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_COMPILE_MAGIC_GATHER,
                                   _lib.PBN_COMPILE_PIPELINED | _lib.PBN_COMPILE_MAGIC_GATHER])
def test_compiled_magic_gather(oracle_mod, which, flags):
    """Multiply gathers with rebuilt tables: bit-exact against the oracle."""
    kw, sem, samp = {}, 0, 0
    if which == "tiny12":
        text, meta = synth.tiny12(1).to_text(), [0, 1, 2]
    elif which == "split":
        text, meta = synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11))).to_text(), [0, 1]
        kw = dict(max_inputs=6)
    else:
        text, meta = synth.paper100(seed=2, p=3e-3).to_text(), [0, 1, 2]
        if which == "paper100_mi12":
            kw = dict(max_inputs=12)
        if which == "nodewise":
            kw, sem = dict(semantics=_lib.PBN_SEM_NODEWISE), 1
        if which == "geometric":
            kw, samp = dict(sampler=_lib.PBN_PERT_GEOMETRIC), 1
    plan, ids = plan_for(text, meta, **kw)
    plan.compile(flags)
    orc = oracle_mod.simulate(text, 51, 0, 160, 500, meta_ids=meta, trace=True, nthreads=NCPU,
                              semantics=sem, sampler=samp)
    _compare(run(plan, seed=51, n_traj=160, n_steps=500, meta=meta, trace=True, kernel=COMPILED), orc, ids)



@pytest.mark.parametrize("sampler", [0, 1])
def test_compiled_wide_plan(oracle_mod, sampler):
    """A plan with more than 24 SEL blocks compiles only in the wide form (SEL
    blocks drawn lazily in group order); bit-exact against the oracle."""
    text = synth.paper100(seed=21, n=400, p=1e-3).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta, sampler=sampler)
    assert plan.info.n_sel_blocks > 24
    plan.compile(_lib.PBN_COMPILE_WIDE)
    orc = oracle_mod.simulate(text, 61, 0, 96, 300, meta_ids=meta, trace=True, nthreads=NCPU, sampler=sampler)
    _compare(run(plan, seed=61, n_traj=96, n_steps=300, meta=meta, trace=True, kernel=COMPILED), orc, ids)
