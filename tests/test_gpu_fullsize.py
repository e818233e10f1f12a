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
