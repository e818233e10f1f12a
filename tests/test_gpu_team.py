"""The team interpreter (PBN_KERNEL_TEAM): K warps share 32 x TPL trajectories (TPL =
1 or 2 per lane), splitting each step's perturbation words, SEL blocks and groups.
Bit-exact against the CPU oracle (every step's state, the counts, the pooled counts)
over warps per team from 1 to 32 and several teams per CTA, ragged trajectory counts,
chained launches cut where the counting window starts, initial states loaded from
memory, split nodes, the geometric sampler, p = 0, tables in shared and in global
memory, and the 2,000-node scale-free network (sampled trajectories)."""
import os

import numpy as np
import pytest

from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
TEAM = _lib.PBN_KERNEL_TEAM


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


@pytest.mark.parametrize("warps,tpb,tpl", [(1, 0, 1), (3, 0, 1), (32, 32, 1), (2, 96, 1), (1, 0, 2), (3, 128, 2),
                                           (16, 64, 2), (5, 0, 0)])
def test_tiny12_every_step(oracle_mod, warps, tpb, tpl):
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta)
    orc = oracle_mod.simulate(text, 1, 0, 70, 3000, meta_ids=meta, trace=True, nthreads=NCPU)
    got = run(plan, seed=1, n_traj=70, n_steps=3000, meta=meta, trace=True, kernel=TEAM, team_warps=warps, tpb=tpb,
              team_tpl=tpl)
    _compare(got, orc, ids)


@pytest.mark.parametrize("n,warps,tpb,tables,tpl", [(100, 0, 0, "default", 0), (300, 4, 64, "default", 1),
                                                    (700, 7, 0, "default", 1), (700, 0, 0, "global", 0),
                                                    (1500, 16, 32, "default", 1), (1500, 0, 0, "default", 0),
                                                    (300, 8, 128, "default", 2), (700, 0, 0, "global", 2),
                                                    (1500, 32, 64, "default", 2)])
def test_wide_plans_against_oracle(oracle_mod, n, warps, tpb, tables, tpl):
    """Paper-scale networks up to 1,500 nodes, a ragged trajectory count, chained
    launches cut where the window starts; tables staged or read from global memory."""
    text = synth.paper100(seed=40 + n, n=n, p=2e-3).to_text()
    meta = [0, 1, 2]
    kw = {}
    if tables == "global":
        import imgdecode
        base, _ = plan_for(text, meta)
        kw["smem_budget"] = max(1024, imgdecode.decode(base.image())["H"]["off_tables"])
    plan, ids = plan_for(text, meta, **kw)
    if tables == "global":
        assert plan.info.tables_in_smem == 0
    T, S = 150, 600
    orc = oracle_mod.simulate(text, 3, 500, T, S, meta_ids=meta, count_from=200, nthreads=NCPU)
    got = run(plan, seed=3, traj_begin=500, n_traj=T, n_steps=S, meta=meta, count_from=200, chunks=[200, 250, 150],
              kernel=TEAM, team_warps=warps, tpb=tpb, team_tpl=tpl)
    _compare(got, orc, ids, trace=False)


@pytest.mark.parametrize("tpl", [1, 2])
def test_loaded_initial_state_and_meta_values(oracle_mod, tpl):
    """A stored initial state, trajectory ids and step indices above 2^32, meta
    values other than 1."""
    text = synth.paper100(seed=77, n=240, p=5e-3).to_text()
    meta, vals = [0, 5, 9], [1, 0, 1]
    plan, ids = plan_for(text, meta)
    rng = np.random.default_rng(5)
    T, S = 45, 300
    tb, sb = 2**40 + 17, 2**33 + 5
    init = (rng.random((T, 240)) < 0.5).astype(np.uint8)
    orc = oracle_mod.simulate(text, 2**63 + 9, tb, T, S, meta_ids=meta, meta_vals=vals, step_begin=sb,
                              init_states=init, count_from=sb + 3, trace=True, nthreads=NCPU)
    got = run(plan, seed=2**63 + 9, traj_begin=tb, n_traj=T, n_steps=S, meta=meta, meta_vals=vals, step_begin=sb,
              count_from=sb + 3, init_bits=init, trace=True, kernel=TEAM, team_warps=5, team_tpl=tpl)
    _compare(got, orc, ids)


@pytest.mark.parametrize("tpl", [1, 2])
def test_split_nodes_geometric_and_p0(oracle_mod, tpl):
    """Split nodes (tables per function), the geometric sampler and a network without
    perturbations, each against its oracle path, with traces."""
    cases = [
        (synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11))).to_text(), [0, 1], dict(max_inputs=3), {}),
        (synth.paper100(seed=2, n=150).to_text(), [0, 1, 2], dict(sampler=_lib.PBN_PERT_GEOMETRIC), dict(sampler=1)),
        (synth.paper100(seed=9, n=70, p=0.0).to_text(), [0, 1], {}, {}),
        (synth.paper100(seed=11, n=90, p=0.3).to_text(), [0, 1], {}, {}),
    ]
    for text, meta, kw, okw in cases:
        plan, ids = plan_for(text, meta, **kw)
        orc = oracle_mod.simulate(text, 8, 0, 40, 400, meta_ids=meta, trace=True, nthreads=NCPU, **okw)
        _compare(run(plan, seed=8, n_traj=40, n_steps=400, meta=meta, trace=True, kernel=TEAM, team_warps=3,
                     team_tpl=tpl), orc, ids)


def test_scalefree_sampled_against_oracle(oracle_mod):
    """The 2,000-node scale-free network: trajectories sampled from a launch of 1,000,
    each equal to the oracle's; the whole launch equal to the interpreter's."""
    text = synth.scalefree2000(seed=3).to_text()
    meta = [0, 1, 2, 3]
    plan, ids = plan_for(text, meta)
    T, S = 1000, 300
    got = run(plan, seed=5, n_traj=T, n_steps=S, meta=meta, count_from=50, kernel=TEAM)
    assert got["status"] == 0
    ref = run(plan, seed=5, n_traj=T, n_steps=S, meta=meta, count_from=50, kernel=_lib.PBN_KERNEL_INTERP)
    assert np.array_equal(got["final"], ref["final"])
    assert np.array_equal(got["counts"], ref["counts"])
    for t in (0, 31, 32, 517, 999):
        orc = oracle_mod.simulate(text, 5, t, 1, S, meta_ids=meta, count_from=50)
        assert np.array_equal(got["final"][t, ids], orc["final"][0, ids]), t
        assert np.array_equal(got["counts"][t], orc["counts"][0]), t


def test_refusals():
    """Node-wise plans, more than 32 warps and ragged CTA sizes are refused."""
    import torch
    text = synth.paper100(seed=9, n=70).to_text()
    red, _ = api.Net.load(text).reduce([0, 1])
    nw = api.Plan(red, semantics=_lib.PBN_SEM_NODEWISE)
    bufs = api.alloc_buffers(nw, 64, "cuda")
    with pytest.raises(_lib.PbnError):
        api.simulate(nw, bufs, seed=1, n_steps=4, meta_ids=[0, 1], kernel=TEAM)
    plan = api.Plan(red)
    bufs = api.alloc_buffers(plan, 64, "cuda")
    for kw in (dict(team_warps=33), dict(trajs_per_block=48), dict(trajs_per_block=64, team_warps=17, team_trajs_per_lane=1),
               dict(trajs_per_block=128, team_warps=17, team_trajs_per_lane=2),
               dict(team_trajs_per_lane=3), dict(team_trajs_per_lane=2, trajs_per_block=32)):
        with pytest.raises(_lib.PbnError):
            api.simulate(plan, bufs, seed=1, n_steps=4, meta_ids=[0, 1], kernel=TEAM, **kw)
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0
