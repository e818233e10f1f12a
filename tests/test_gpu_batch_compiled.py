"""Compiled batches (pbn_batch_compile): networks whose plans compile run their own
generated device functions and the others the interpreter, in one persistent launch
per chunk.  Every network's states and counts equal those of the uncompiled batch,
of its own single-network launch and of the CPU oracle, whatever the mix, chunking,
graph replay or queue entry point."""
import os

import numpy as np
import pytest

from gpu_helpers import plan_for, run
from paper_1605_00854_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mix(seed, sizes, T_max):
    """Networks of the given sizes: sizes above 1,024 nodes (or with more than 24
    selection blocks) do not compile and stay with the interpreter."""
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        T = int(rng.integers(40, T_max))
        p = float(10 ** rng.uniform(-4, -2))
        text = synth.paper100(seed=seed * 100 + i, n=n, p=p).to_text()
        k = int(rng.integers(1, 4))
        meta = sorted(int(x) for x in rng.choice(3, size=k, replace=False))
        vals = [int(v) for v in rng.integers(0, 2, size=k)] if i % 2 else None
        out.append(dict(text=text, T=T, meta=meta, vals=vals, seed=int(rng.integers(0, 2**63)), n=n))
    return out


def _entries(nets, **plan_kw):
    entries, plans = [], []
    for k, d in enumerate(nets):
        plan, ids = plan_for(d["text"], d["meta"], **plan_kw)
        entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, d["T"]), seed=d["seed"], meta_ids=d["meta"],
                            meta_vals=d["vals"], traj_begin=k * 10**5, count_from=21))
        plans.append((plan, ids))
    return entries, plans


def _collect(plan, bufs):
    import torch
    torch.cuda.synchronize()
    return dict(final=plan.unpack(bufs.state.cpu().numpy().view(np.uint64)),
                counts=bufs.counts.cpu().numpy().view(np.uint64).T.copy(),
                pooled=bufs.pooled.cpu().numpy().view(np.uint64).copy())


SIZES = [20, 45, 90, 160, 300, 520, 1100]


@pytest.mark.parametrize("flags", [_lib.PBN_COMPILE_INTERLEAVED, 0, _lib.PBN_COMPILE_PERT_UNROLLED,
                                   _lib.PBN_COMPILE_PIPELINED])
def test_compiled_batch_equals_interpreted_batch_and_single_launches(flags):
    nets = _mix(51, SIZES, 900)
    ref_e, plans = _entries(nets)
    got_e, _ = _entries(nets)
    ref = api.Batch(ref_e)
    got = api.Batch(got_e, compile_flags=flags)
    assert 0 < got.info.n_compiled < len(nets)  # a mix of compiled and interpreted networks
    for c in [150, 1, 249]:
        ref.run(c)
        got.run(c)
    assert int(got.status.item()) == 0 and got.queue.cpu().tolist() == [0, 0]
    for k, (d, (plan, ids)) in enumerate(zip(nets, plans)):
        a, b = _collect(plan, ref_e[k]["bufs"]), _collect(plan, got_e[k]["bufs"])
        assert np.array_equal(a["final"][:, ids], b["final"][:, ids]), k
        assert np.array_equal(a["counts"], b["counts"]) and np.array_equal(a["pooled"], b["pooled"]), k
    # and one network's own launch
    k = 2
    d, (plan, ids) = nets[k], plans[k]
    one = run(plan, seed=d["seed"], traj_begin=k * 10**5, n_traj=d["T"], n_steps=400, meta=d["meta"],
              meta_vals=d["vals"], count_from=21, kernel=_lib.PBN_KERNEL_INTERP)
    b = _collect(plan, got_e[k]["bufs"])
    assert np.array_equal(b["final"][:, ids], one["final"][:, ids]) and np.array_equal(b["counts"], one["counts"])


def test_compiled_batch_against_oracle(oracle_mod):
    nets = _mix(52, [25, 70, 130, 1050], 160)
    entries, plans = _entries(nets)
    B = api.Batch(entries, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    assert B.info.n_compiled == 3
    B.run(300)
    B.run(200)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], k * 10**5, d["T"], 500, meta_ids=d["meta"],
                                  meta_vals=d["vals"], count_from=21, nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k
        assert np.array_equal(got["pooled"], orc["counts"].sum(axis=0, dtype=np.uint64)), k


@pytest.mark.parametrize("variant", ["geometric", "nodewise", "p0"])
def test_compiled_batch_variants_against_oracle(oracle_mod, variant):
    """The second perturbation sampler, the node-wise semantics and p = 0 in the
    batch functions, against their own oracle paths."""
    nets = _mix(53, [30, 80, 200], 140)
    kw, okw = {}, {}
    if variant == "geometric":
        kw, okw = dict(sampler=_lib.PBN_PERT_GEOMETRIC), dict(sampler=1)
    elif variant == "nodewise":
        kw, okw = dict(semantics=_lib.PBN_SEM_NODEWISE), dict(semantics=1)
    else:
        for k, d in enumerate(nets):
            d["text"] = synth.paper100(seed=900 + k, n=d["n"], p=0.0).to_text()
    entries, plans = _entries(nets, **kw)
    B = api.Batch(entries, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    assert B.info.n_compiled == len(nets)
    B.run(250)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], k * 10**5, d["T"], 250, meta_ids=d["meta"],
                                  meta_vals=d["vals"], count_from=21, nthreads=NCPU, **okw)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), (variant, k)
        assert np.array_equal(got["counts"], orc["counts"]), (variant, k)


def test_compiled_batch_graph_replay_and_static_queue():
    """Chunks captured in a CUDA graph and the allocation-free entry point give the
    same results as direct launches of the compiled batch."""
    import torch
    nets = _mix(54, [40, 110, 700, 1200], 500)
    e1, plans = _entries(nets)
    e2, _ = _entries(nets)
    e3, _ = _entries(nets)
    b1 = api.Batch(e1, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    b2 = api.Batch(e2, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    b3 = api.Batch(e3, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    for c in [100, 100, 57]:
        b1.run(c)
        b3.run_static(c, slot=2)
    b2.run(1)  # launch shape found outside the capture
    torch.cuda.synchronize()
    for e in e2:
        e["bufs"].counts.zero_(); e["bufs"].pooled.zero_(); e["bufs"].state.zero_()
    g = b2.capture([100, 100, 57], step_offset=0)
    g.replay()
    torch.cuda.synchronize()
    assert int(b1.status.item()) == int(b2.status.item()) == int(b3.status.item()) == 0
    for k, (plan, ids) in enumerate(plans):
        a, b, c = _collect(plan, e1[k]["bufs"]), _collect(plan, e2[k]["bufs"]), _collect(plan, e3[k]["bufs"])
        for x in (b, c):
            assert np.array_equal(a["final"], x["final"]) and np.array_equal(a["counts"], x["counts"]), k
            assert np.array_equal(a["pooled"], x["pooled"]), k


def test_compile_errors():
    nets = _mix(55, [30], 100)
    entries, _ = _entries(nets)
    B = api.Batch(entries, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    with pytest.raises(_lib.PbnError) as e:  # twice
        _lib.check(_lib.load().pbn_batch_compile(B._h, _lib.PBN_COMPILE_INTERLEAVED, None), "pbn_batch_compile")
    assert e.value.status == _lib.PBN_EINVAL
    wide = _mix(56, [1300], 100)
    we, _ = _entries(wide)
    with pytest.raises(_lib.PbnError) as e:  # nothing compiles
        api.Batch(we, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)
    assert e.value.status == _lib.PBN_EINVAL and "no network" in str(e.value)


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("count_from", [100, 250])
def test_batch_chain_cut_at_the_window_start(oracle_mod, compiled, count_from):
    """Batch launches cut exactly where the counting window starts count each state
    once (the oracle's one run), compiled or interpreted."""
    text = synth.tiny12(1).to_text()
    nets = [dict(text=text, T=90, meta=[11], vals=None, seed=31, n=12),
            dict(text=synth.paper100(seed=57, n=60, p=1e-2).to_text(), T=70, meta=[0], vals=None, seed=32, n=60)]
    entries, plans = _entries(nets)
    for e in entries:
        e["count_from"] = count_from
    B = api.Batch(entries, compile_flags=_lib.PBN_COMPILE_INTERLEAVED if compiled else None)
    for c in [100, 150, 50]:
        B.run(c)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], k * 10**5, d["T"], 300, meta_ids=d["meta"],
                                  count_from=count_from, nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k


def test_batch_of_1024_thread_ctas_against_oracle(oracle_mod):
    """The interpreted batch kernel with CTAs of 1,024 threads (wider lane groups per
    item) gives the oracle's states and counts; such a batch refuses compilation."""
    nets = _mix(57, [25, 90, 700, 1300, 2100], 200)
    entries, plans = _entries(nets)
    B = api.Batch(entries, threads=1024)
    assert B.info.threads == 1024
    for c in [150, 1, 149]:
        B.run(c)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], k * 10**5, d["T"], 300, meta_ids=d["meta"],
                                  meta_vals=d["vals"], count_from=21, nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k
    e2, _ = _entries(nets[:1])
    with pytest.raises(_lib.PbnError):
        api.Batch(e2, threads=1024, compile_flags=_lib.PBN_COMPILE_INTERLEAVED)


def test_split_batch_against_oracle_graph_and_static_queue(oracle_mod):
    """A split compiled batch (the compiled networks' items in the generated module,
    the others in the 1,024-thread interpreter kernel, two launches per chunk on one
    queue) gives the oracle's states and counts through direct runs, a CUDA graph
    and the allocation-free entry point."""
    import torch
    nets = _mix(58, [30, 75, 160, 900, 1400, 2200], 180)
    split = _lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_BATCH_SPLIT
    e1, plans = _entries(nets)
    e2, _ = _entries(nets)
    e3, _ = _entries(nets)
    b1, b2, b3 = (api.Batch(e, compile_flags=split) for e in (e1, e2, e3))
    assert 0 < b1.info.n_items_compiled < b1.info.n_items and b1.info.n_compiled == 3
    for c in [120, 1, 179]:
        b1.run(c)
        b3.run_static(c, slot=4)
    b2.run(1)
    torch.cuda.synchronize()
    for e in e2:
        e["bufs"].counts.zero_(); e["bufs"].pooled.zero_()
    g = b2.capture([120, 1, 179], step_offset=0)
    g.replay()
    torch.cuda.synchronize()
    assert int(b1.status.item()) == int(b2.status.item()) == int(b3.status.item()) == 0
    assert b1.queue.cpu().tolist() == [0, 0]
    for k, (d, (plan, ids)) in enumerate(zip(nets, plans)):
        orc = oracle_mod.simulate(d["text"], d["seed"], k * 10**5, d["T"], 300, meta_ids=d["meta"],
                                  meta_vals=d["vals"], count_from=21, nthreads=NCPU)
        for es in (e1, e2, e3):
            got = _collect(plan, es[k]["bufs"])
            assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
            assert np.array_equal(got["counts"], orc["counts"]), k
            assert np.array_equal(got["pooled"], orc["counts"].sum(axis=0, dtype=np.uint64)), k
