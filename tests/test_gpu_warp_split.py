"""The warp-split compiled form (PBN_COMPILE_WARP_SPLIT): a CTA of K warps runs 32
trajectories, each warp its own share of the perturbation words and state rows, the
states in shared memory.  Bit-exact against the CPU oracle (every step's state, the
counts, the pooled counts) on small and wide plans, ragged trajectory counts, chained
launches cut at the window start, split nodes, the geometric sampler and p = 0, with
the selection choices in registers and in shared memory (PBN_COMPILE_WS_SELSMEM)."""
import os

import numpy as np
import pytest

from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
COMPILED = _lib.PBN_KERNEL_COMPILED
WS = _lib.PBN_COMPILE_WARP_SPLIT
SELSMEM = _lib.PBN_COMPILE_WS_SELSMEM


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


@pytest.mark.parametrize("warps,extra", [(1, 0), (2, 0), (1, SELSMEM), (2, SELSMEM)])
def test_tiny12_every_step(oracle_mod, warps, extra):
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta)
    plan.compile(WS | _lib.PBN_COMPILE_WARPS(warps) | extra)
    orc = oracle_mod.simulate(text, 1, 0, 70, 3000, meta_ids=meta, trace=True, nthreads=NCPU)
    _compare(run(plan, seed=1, n_traj=70, n_steps=3000, meta=meta, trace=True, kernel=COMPILED), orc, ids)


@pytest.mark.parametrize("n,warps,minctas,extra", [(100, 0, 0, 0), (300, 4, 0, 0), (300, 3, 3, 0), (700, 0, 2, 0),
                                                   (1500, 8, 0, 0), (300, 2, 0, SELSMEM), (1500, 3, 0, SELSMEM)])
def test_wide_plans_against_oracle(oracle_mod, n, warps, minctas, extra):
    """Paper-scale networks up to 1,500 nodes (beyond the register-state forms), a
    ragged trajectory count, chained launches cut where the window starts."""
    text = synth.paper100(seed=40 + n, n=n, p=2e-3).to_text()
    meta = [0, 1, 2]
    plan, ids = plan_for(text, meta)
    plan.compile(WS | _lib.PBN_COMPILE_WARPS(warps) | _lib.PBN_COMPILE_MINCTAS(minctas) | extra)
    T, S = 150, 600
    orc = oracle_mod.simulate(text, 3, 500, T, S, meta_ids=meta, count_from=200, nthreads=NCPU)
    got = run(plan, seed=3, traj_begin=500, n_traj=T, n_steps=S, meta=meta, count_from=200, chunks=[200, 250, 150],
              kernel=COMPILED)
    _compare(got, orc, ids, trace=False)


@pytest.mark.parametrize("extra", [0, SELSMEM])
def test_split_nodes_geometric_and_p0(oracle_mod, extra):
    """Split nodes (tables per function, some looked up), the geometric sampler and a
    network without perturbations, each against its oracle path, with traces."""
    cases = [
        (synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11))).to_text(), [0, 1], dict(max_inputs=3), {}),
        (synth.paper100(seed=2, n=150).to_text(), [0, 1, 2], dict(sampler=_lib.PBN_PERT_GEOMETRIC), dict(sampler=1)),
        (synth.paper100(seed=9, n=70, p=0.0).to_text(), [0, 1], {}, {}),
    ]
    for text, meta, kw, okw in cases:
        plan, ids = plan_for(text, meta, **kw)
        plan.compile(WS | _lib.PBN_COMPILE_WARPS(2) | extra)
        orc = oracle_mod.simulate(text, 8, 0, 40, 400, meta_ids=meta, trace=True, nthreads=NCPU, **okw)
        _compare(run(plan, seed=8, n_traj=40, n_steps=400, meta=meta, trace=True, kernel=COMPILED), orc, ids)


@pytest.mark.parametrize("extra", [0, SELSMEM | _lib.PBN_COMPILE_WS_BATCH(1)])
def test_scalefree_sampled_against_oracle(oracle_mod, extra):
    """The 2,000-node scale-free network: trajectories sampled from a launch of 1,024,
    each equal to the oracle's."""
    text = synth.scalefree2000(seed=3).to_text()
    meta = [0, 1, 2, 3]
    plan, ids = plan_for(text, meta)
    plan.compile(WS | extra)
    T, S = 1024, 300
    got = run(plan, seed=5, n_traj=T, n_steps=S, meta=meta, count_from=50, kernel=COMPILED)
    assert got["status"] == 0
    for t in (0, 31, 32, 517, 1023):
        orc = oracle_mod.simulate(text, 5, t, 1, S, meta_ids=meta, count_from=50)
        assert np.array_equal(got["final"][t, ids], orc["final"][0, ids]), t
        assert np.array_equal(got["counts"][t], orc["counts"][0]), t
