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
