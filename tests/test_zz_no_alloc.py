"""The allocation-free batch entry point (pbn_batch_run_static).

Callers that cannot allocate device memory when they run a batch -- a serving loop
whose allocator owns the device, code recording a CUDA graph, a latency-critical loop
that must not call cudaMalloc/cudaFree because they can synchronise the device --
use this entry point: its work-queue scratch is a small static array inside the
library.  Its results must equal those of pbn_batch_run (caller-provided scratch)
exactly, on consecutive calls that reuse the array.  This file is collected last so
that a stop-at-first-failure run has already run every other test."""

import numpy as np
import pytest

from paper_1605_00854_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu


def _entries(seed=11, count=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(20, 300))
        T = int(rng.integers(40, 700))
        text = synth.paper100(seed=300 + i, n=n, p=float(10 ** rng.uniform(-4, -2))).to_text()
        red, ids = api.Net.load(text).reduce([0, 1, 2])
        plan = api.Plan(red)
        out.append(dict(plan=plan, bufs=api.alloc_buffers(plan, T), seed=int(rng.integers(0, 2**62)),
                        meta_ids=[0, 1, 2], traj_begin=i * 100000, count_from=5, ids=ids))
    return out


def _snapshot(entries):
    import torch
    torch.cuda.synchronize()
    return [(e["bufs"].state.cpu().numpy().copy(), e["bufs"].counts.cpu().numpy().copy(),
             e["bufs"].pooled.cpu().numpy().copy()) for e in entries]


def test_static_scratch_entry_point_matches_allocating_one():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ref_entries, got_entries = _entries(), _entries()
    ref = api.Batch([{k: v for k, v in e.items() if k != "ids"} for e in ref_entries])
    got = api.Batch([{k: v for k, v in e.items() if k != "ids"} for e in got_entries])
    # two calls in a row: the second reuses the static queue the first left behind
    for n_steps, slot in [(120, 0), (77, 0), (50, 5)]:
        ref.run(n_steps)
        got.run_static(n_steps, slot=slot)
        a, b = _snapshot(ref_entries), _snapshot(got_entries)
        for (sa, ca, pa), (sb, cb, pb) in zip(a, b):
            assert np.array_equal(sa, sb) and np.array_equal(ca, cb) and np.array_equal(pa, pb)
    assert int(got.status.item()) == 0
    # slots beyond the static array are rejected with a clear error
    with pytest.raises(_lib.PbnError) as e:
        got.run_static(10, slot=_lib.PBN_STATIC_QUEUE_SLOTS)
    assert e.value.status == -1 and "static slots" in str(e.value)


def _sized_entries(n, count, seed):
    """Batch entries of `count` paper-scale networks of n nodes (fresh buffers)."""
    out = []
    for i in range(count):
        text = synth.paper100(seed=seed + i, n=n, p=1e-3).to_text()
        red, _ = api.Net.load(text).reduce([0, 1, 2])
        plan = api.Plan(red)
        out.append(dict(plan=plan, bufs=api.alloc_buffers(plan, 600), seed=seed * 7 + i, meta_ids=[0, 1, 2],
                        traj_begin=1000 * i))
    return out


def test_static_and_allocating_calls_mix_across_shared_memory_sizes():
    """Two batches whose kernels need different dynamic shared memory (one between
    the 48 KB default and 100 KB, one above 100 KB), advanced by alternating calls of
    the allocating and the allocation-free entry points: every call launches (neither
    entry point lowers the limit the other raised) and every result equals a batch
    advanced by pbn_batch_run alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mid_ref, mid_got = _sized_entries(200, 3, 40), _sized_entries(200, 3, 40)
    big_ref, big_got = _sized_entries(600, 2, 60), _sized_entries(600, 2, 60)
    mk = lambda es: api.Batch([dict(e) for e in es])
    mid_r, mid_g, big_r, big_g = mk(mid_ref), mk(mid_got), mk(big_ref), mk(big_got)
    assert 48 * 1024 < mid_g.info.smem_bytes <= 100 * 1024 < big_g.info.smem_bytes
    # the big batch first through the allocating call, then the mid-sized one through
    # the static call, then the big one again through both
    plan = [(big_g, "run", 60), (mid_g, "static", 70), (big_g, "run", 40), (big_g, "static", 30),
            (mid_g, "run", 20), (mid_g, "static", 25)]
    for b, how, steps in plan:
        if how == "run":
            b.run(steps)
        else:
            b.run_static(steps, slot=3)
        (big_r if b is big_g else mid_r).run(steps)
    for ref_es, got_es in ((mid_ref, mid_got), (big_ref, big_got)):
        for (sa, ca, pa), (sb, cb, pb) in zip(_snapshot(ref_es), _snapshot(got_es)):
            assert np.array_equal(sa, sb) and np.array_equal(ca, cb) and np.array_equal(pa, pb)
    assert int(mid_g.status.item()) == 0 and int(big_g.status.item()) == 0
