"""Full-size parity at the benchmark configuration: the paper-scale network, 2^16
trajectories x 10^6 steps in one launch with the default (autotuned) launch shape,
exactly as bench.py runs it.  The oracle recomputes sampled trajectories at full
length; every trajectory is checked against the count invariants."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1605_00854_gb300 import api, synth

pytestmark = pytest.mark.gpu

SEED = 20160503  # the benchmark's seed
META = [0, 1, 2]


def test_paper100_full_size_sampled_trajectories(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    text = synth.paper100(seed=2).to_text()
    red, ids = api.Net.load(text).reduce(META)
    plan = api.Plan(red)
    T, S = 1 << 16, 10**6
    bufs = api.alloc_buffers(plan, T)
    api.simulate(plan, bufs, seed=SEED, n_steps=S, meta_ids=META)
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0
    counts = bufs.counts.cpu().numpy().view(np.uint64).T          # [T, 5]
    final = plan.unpack(bufs.state.cpu().numpy().view(np.uint64))  # [T, n]
    pooled = bufs.pooled.cpu().numpy().view(np.uint64)
    # invariants for every trajectory: S pairs; V = visits over S + 1 states
    pairs = counts[:, 1:].sum(axis=1)
    assert np.all(pairs == S)
    z_first_last = counts[:, 0].astype(np.int64) - (counts[:, 3] + counts[:, 4]).astype(np.int64)
    assert np.all((z_first_last >= 0) & (z_first_last <= 1))   # V - (n10 + n11) = z_last
    assert np.array_equal(pooled, counts.sum(axis=0))
    # sampled trajectories recomputed by the oracle at full length
    sample = [0, 1, 12345, 40000, 65535, 31337, 777, 50001]
    def one(t):
        return oracle_mod.simulate(text, SEED, t, 1, S, meta_ids=META)
    with ThreadPoolExecutor(max_workers=min(len(sample), os.cpu_count() or 1)) as ex:
        outs = list(ex.map(one, sample))
    for t, o in zip(sample, outs):
        assert np.array_equal(final[t, ids], o["final"][0, ids]), t
        assert np.array_equal(counts[t], o["counts"][0]), t


def test_scalefree2000_full_size_sampled_trajectories(oracle_mod):
    """Large network at its benchmark size: n = 2000, 2^14 trajectories x 10^5 steps,
    default launch shape; sampled trajectories recomputed by the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    text = synth.scalefree2000(seed=3).to_text()
    meta = [0, 1, 2, 3]
    red, ids = api.Net.load(text).reduce(meta)
    plan = api.Plan(red)
    T, S = 1 << 14, 10**5
    bufs = api.alloc_buffers(plan, T)
    api.simulate(plan, bufs, seed=SEED, n_steps=S, meta_ids=meta)
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0
    counts = bufs.counts.cpu().numpy().view(np.uint64).T
    final = plan.unpack(bufs.state.cpu().numpy().view(np.uint64))
    assert np.all(counts[:, 1:].sum(axis=1) == S)
    assert np.array_equal(bufs.pooled.cpu().numpy().view(np.uint64), counts.sum(axis=0))
    sample = [0, 16383, 4242, 9999]
    def one(t):
        return oracle_mod.simulate(text, SEED, t, 1, S, meta_ids=meta)
    with ThreadPoolExecutor(max_workers=min(len(sample), os.cpu_count() or 1)) as ex:
        outs = list(ex.map(one, sample))
    for t, o in zip(sample, outs):
        assert np.array_equal(final[t, ids], o["final"][0, ids]), t
        assert np.array_equal(counts[t], o["counts"][0]), t


def test_paper100_full_size_geometric_sampler(oracle_mod):
    """The benchmark size with the geometric perturbation sampler and its compiled
    kernel: sampled trajectories recomputed by the oracle's geometric sampler."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00854_gb300 import _lib
    text = synth.paper100(seed=2).to_text()
    red, ids = api.Net.load(text).reduce(META)
    plan = api.Plan(red, max_inputs=12, sampler=_lib.PBN_PERT_GEOMETRIC)
    plan.compile(_lib.PBN_COMPILE_INTERLEAVED)
    T, S = 1 << 16, 10**6
    bufs = api.alloc_buffers(plan, T)
    api.simulate(plan, bufs, seed=SEED, n_steps=S, meta_ids=META, kernel=_lib.PBN_KERNEL_COMPILED)
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0
    counts = bufs.counts.cpu().numpy().view(np.uint64).T
    final = plan.unpack(bufs.state.cpu().numpy().view(np.uint64))
    assert np.all(counts[:, 1:].sum(axis=1) == S)
    sample = [3, 65534, 20000, 47011]
    def one(t):
        return oracle_mod.simulate(text, SEED, t, 1, S, meta_ids=META, sampler=1)
    with ThreadPoolExecutor(max_workers=min(len(sample), os.cpu_count() or 1)) as ex:
        outs = list(ex.map(one, sample))
    for t, o in zip(sample, outs):
        assert np.array_equal(final[t, ids], o["final"][0, ids]), t
        assert np.array_equal(counts[t], o["counts"][0]), t


@pytest.mark.parametrize("workload", ["paper100", "scalefree2000"])
def test_full_size_in_the_bench_launch_configuration(oracle_mod, workload):
    """The configuration bench.py times: the autotuner's choice of group size,
    kernel, code shape and lanes per trajectory, at the benchmark size; sampled
    trajectories recomputed by the oracle, count invariants for all of them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00854_gb300 import autotune
    if workload == "paper100":
        text, meta, T, S, steps = synth.paper100(seed=2).to_text(), META, 1 << 16, 10**6, 2000
        sample = [5, 65000, 33333]
    else:
        text, meta, T, S, steps = synth.scalefree2000(seed=3).to_text(), [0, 1, 2, 3], 1 << 14, 10**5, 200
        sample = [7, 16000]
    ch = autotune.tune_network(text, meta, T, steps=steps)
    plan = autotune.plan_for_choice(text, meta, ch)
    _, ids = api.Net.load(text).reduce(meta)
    bufs = api.alloc_buffers(plan, T)
    api.simulate(plan, bufs, seed=SEED, n_steps=S, meta_ids=meta, kernel=ch.kernel, lanes_per_traj=ch.lanes_per_traj)
    torch.cuda.synchronize()
    assert int(bufs.status.item()) == 0
    counts = bufs.counts.cpu().numpy().view(np.uint64).T
    final = plan.unpack(bufs.state.cpu().numpy().view(np.uint64))
    assert np.all(counts[:, 1:].sum(axis=1) == S)
    assert np.array_equal(bufs.pooled.cpu().numpy().view(np.uint64), counts.sum(axis=0))
    def one(t):
        return oracle_mod.simulate(text, SEED, t, 1, S, meta_ids=meta)
    with ThreadPoolExecutor(max_workers=min(len(sample), os.cpu_count() or 1)) as ex:
        outs = list(ex.map(one, sample))
    for t, o in zip(sample, outs):
        assert np.array_equal(final[t, ids], o["final"][0, ids]), (t, ch)
        assert np.array_equal(counts[t], o["counts"][0]), (t, ch)
