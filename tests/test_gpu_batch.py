"""The batched persistent kernel (device work queue, CUDA-graph step chunks):
every network's states and counts equal those of its own single-network launch and
of the CPU oracle, whatever the mix."""
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


def _networks(seed=40, count=10):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(20, 400))
        T = int(rng.integers(50, 1200))
        p = float(10 ** rng.uniform(-5, -2))
        text = synth.paper100(seed=1000 + i, n=n, p=p).to_text()
        meta = sorted(set(int(x) for x in rng.choice(3, size=int(rng.integers(1, 4)), replace=False)))
        out.append(dict(text=text, T=T, meta=meta, seed=int(rng.integers(0, 2**63)), n=n))
    return out


def _collect(plan, bufs):
    import torch
    torch.cuda.synchronize()
    return dict(final=plan.unpack(bufs.state.cpu().numpy().view(np.uint64)),
                counts=bufs.counts.cpu().numpy().view(np.uint64).T.copy(),
                pooled=bufs.pooled.cpu().numpy().view(np.uint64).copy())


@pytest.mark.parametrize("chunks", [[400], [150, 1, 249], [200, 200]])
def test_batch_equals_single_network_launches(chunks):
    nets = _networks()
    S = sum(chunks)
    entries, plans = [], []
    for k, d in enumerate(nets):
        plan, ids = plan_for(d["text"], d["meta"])
        bufs = api.alloc_buffers(plan, d["T"])
        entries.append(dict(plan=plan, bufs=bufs, seed=d["seed"], meta_ids=d["meta"],
                            traj_begin=k * 10**6, count_from=37))
        plans.append((plan, ids))
    B = api.Batch(entries)
    assert B.info.n_nets == len(nets) and B.info.n_items >= len(nets)
    for c in chunks:
        B.run(c)
    assert int(B.status.item()) == 0 and B.queue.cpu().tolist() == [0, 0]
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        ref = run(plan, seed=d["seed"], traj_begin=k * 10**6, n_traj=d["T"], n_steps=S, meta=d["meta"],
                  count_from=37, kernel=_lib.PBN_KERNEL_INTERP)
        assert np.array_equal(got["final"][:, ids], ref["final"][:, ids]), k
        assert np.array_equal(got["counts"], ref["counts"]), k
        assert np.array_equal(got["pooled"], ref["pooled"]), k


def test_batch_against_oracle(oracle_mod):
    nets = _networks(seed=7, count=4)
    entries, plans = [], []
    for d in nets:
        d["T"] = min(d["T"], 150)
        plan, ids = plan_for(d["text"], d["meta"])
        entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, d["T"]), seed=d["seed"], meta_ids=d["meta"]))
        plans.append((plan, ids))
    B = api.Batch(entries)
    B.run(300)
    B.run(200)
    for d, (plan, ids), e in zip(nets, plans, entries):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], 0, d["T"], 500, meta_ids=d["meta"], nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids])
        assert np.array_equal(got["counts"], orc["counts"])


def test_batch_graph_capture_replays_the_chunk_loop():
    import torch
    nets = _networks(seed=3, count=6)
    def build():
        entries, plans = [], []
        for d in nets:
            plan, ids = plan_for(d["text"], d["meta"])
            entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, d["T"]), seed=d["seed"], meta_ids=d["meta"]))
            plans.append((plan, ids))
        return api.Batch(entries), entries, plans
    B1, e1, p1 = build()
    for _ in range(4):
        B1.run(100)
    B2, e2, p2 = build()
    B2.run(1)                 # warm up (attribute setting) outside the capture
    for e in e2:
        e["bufs"].state.zero_(); e["bufs"].counts.zero_(); e["bufs"].pooled.zero_()
    g = B2.capture([100, 100, 100, 100])
    g.replay()
    torch.cuda.synchronize()
    assert int(B2.status.item()) == 0
    for (plan, ids), a, b in zip(p1, e1, e2):
        ga, gb = _collect(plan, a["bufs"]), _collect(plan, b["bufs"])
        assert np.array_equal(ga["final"], gb["final"]) and np.array_equal(ga["counts"], gb["counts"])


@pytest.mark.parametrize("lane_groups", [True, False])
def test_batch_wide_networks_use_lane_groups(lane_groups):
    """Wide networks get several lanes per trajectory (lane groups) or teams of warps
    on 32 trajectories inside the batch and still reproduce their single-network
    launches exactly."""
    rng = np.random.default_rng(12)
    entries, plans, refs = [], [], []
    for i, n in enumerate([1500, 2500, 60, 900]):
        text = synth.paper100(seed=2000 + i, n=n, p=float(10 ** rng.uniform(-4, -2))).to_text()
        plan, ids = plan_for(text, [0, 1, 2])
        T = int(rng.integers(100, 400))
        seed = int(rng.integers(0, 2**62))
        entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, T), seed=seed, meta_ids=[0, 1, 2]))
        plans.append((plan, ids))
        refs.append(run(plan, seed=seed, n_traj=T, n_steps=240, meta=[0, 1, 2], kernel=_lib.PBN_KERNEL_INTERP, lanes=1))
    B = api.Batch(entries, lane_groups=lane_groups)
    assert (B.info.n_team == 0) if lane_groups else (B.info.n_team == 3)
    B.run(100)
    B.run(140)
    assert int(B.status.item()) == 0
    for (plan, ids), e, ref in zip(plans, entries, refs):
        got = _collect(plan, e["bufs"])
        assert np.array_equal(got["final"][:, ids], ref["final"][:, ids])
        assert np.array_equal(got["counts"], ref["counts"])


def test_batch_warp_per_trajectory_on_a_wide_state(oracle_mod):
    """A network whose specs nearly fill shared memory and whose state spans 62 words
    runs with 16 lanes per trajectory inside the batch (32 trajectory slots x 16 lanes
    = the CTA's 512 threads) and equals the oracle, next to a small network."""
    big = synth.scalefree2000(seed=3).to_text()
    small = synth.paper100(seed=5).to_text()
    specs = [(big, [0, 1, 2, 3], 64, 8), (small, [0, 1, 2], 96, 12)]
    entries, plans = [], []
    for k, (text, meta, T, mi) in enumerate(specs):
        plan, ids = plan_for(text, meta, max_inputs=mi)
        entries.append(dict(plan=plan, bufs=api.alloc_buffers(plan, T), seed=31 + k, meta_ids=meta, count_from=5))
        plans.append((plan, ids))
    assert plans[0][0].info.state_words >= 16
    B = api.Batch(entries, lane_groups=True)
    assert B.info.max_lanes == 16
    B.run(50)
    B.run(30)
    assert int(B.status.item()) == 0
    for k, ((text, meta, T, _), (plan, ids), e) in enumerate(zip(specs, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(text, 31 + k, 0, T, 80, meta_ids=meta, count_from=5, nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k


def test_batch_with_split_nodes(oracle_mod):
    """Networks with split nodes in the batched kernel equal the oracle."""
    texts = [synth.random_pbn(50 + i, 30 + 7 * i, 1e-2, k_choices=tuple(range(1, 11))).to_text() for i in range(3)]
    entries, plans = [], []
    for k, text in enumerate(texts):
        plan, ids = plan_for(text, [0, 1], max_inputs=3)
        assert plan.info.n_split > 0
        bufs = api.alloc_buffers(plan, 100 + 50 * k)
        entries.append(dict(plan=plan, bufs=bufs, seed=9 + k, meta_ids=[0, 1]))
        plans.append((plan, ids))
    B = api.Batch(entries)
    B.run(300)
    assert int(B.status.item()) == 0
    for k, (text, (plan, ids), e) in enumerate(zip(texts, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(text, 9 + k, 0, 100 + 50 * k, 300, meta_ids=[0, 1], nthreads=NCPU)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k



def test_batch_mixes_semantics(oracle_mod):
    """A batch holding Eq. 1 and node-wise plans gives each network its own law."""
    nets = _networks(seed=11, count=4)
    entries, plans = [], []
    for k, d in enumerate(nets):
        sem = _lib.PBN_SEM_NODEWISE if k % 2 else _lib.PBN_SEM_EQ1
        plan, ids = plan_for(d["text"], d["meta"], semantics=sem)
        bufs = api.alloc_buffers(plan, d["T"])
        entries.append(dict(plan=plan, bufs=bufs, seed=d["seed"], meta_ids=d["meta"]))
        plans.append((plan, ids, sem))
    B = api.Batch(entries)
    B.run(250)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids, sem), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], 0, d["T"], 250, meta_ids=d["meta"], nthreads=NCPU,
                                  semantics=int(sem))
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k



def test_batch_geometric_sampler(oracle_mod):
    nets = _networks(seed=13, count=3)
    entries, plans = [], []
    for d in nets:
        plan, ids = plan_for(d["text"], d["meta"], sampler=_lib.PBN_PERT_GEOMETRIC)
        bufs = api.alloc_buffers(plan, d["T"])
        entries.append(dict(plan=plan, bufs=bufs, seed=d["seed"], meta_ids=d["meta"]))
        plans.append((plan, ids))
    B = api.Batch(entries)
    B.run(200)
    assert int(B.status.item()) == 0
    for k, (d, (plan, ids), e) in enumerate(zip(nets, plans, entries)):
        got = _collect(plan, e["bufs"])
        orc = oracle_mod.simulate(d["text"], d["seed"], 0, d["T"], 200, meta_ids=d["meta"], nthreads=NCPU, sampler=1)
        assert np.array_equal(got["final"][:, ids], orc["final"][:, ids]), k
        assert np.array_equal(got["counts"], orc["counts"]), k
