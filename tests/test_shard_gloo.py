"""World-size-2 gloo test of the trajectory sharding (CPU only).

Each rank simulates its own trajectory-id range with the oracle; gathering the
ranges reproduces one single-process run exactly, and the pooled counts add up."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1605_00854_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        text = synth.tiny12(1).to_text()
        if mode == "weak":
            tb, nt = shard.weak_range(rank, world, 24)
        else:
            tb, nt = shard.strong_range(rank, world, 37)
        r = oracle.simulate(text, 9, tb, nt, 400, meta_ids=[0, 1, 2])
        obj = [None] * world
        dist.all_gather_object(obj, (tb, r["final"], r["counts"]))
        if rank == 0:
            q.put(obj)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_sharded_ranks_reproduce_one_run(oracle_mod, mode):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts.sort(key=lambda t: t[0])
    total = sum(len(f) for _, f, _ in parts)
    text = synth.tiny12(1).to_text()
    ref = oracle_mod.simulate(text, 9, 0, total, 400, meta_ids=[0, 1, 2])
    assert np.array_equal(np.concatenate([f for _, f, _ in parts]), ref["final"])
    assert np.array_equal(np.concatenate([c for _, _, c in parts]), ref["counts"])
    pooled = shard.pool([c.sum(axis=0) for _, _, c in parts])
    assert pooled == [int(x) for x in ref["counts"].sum(axis=0)]


def test_ranges_partition_the_ids():
    for world in (1, 2, 3, 8):
        got = [shard.strong_range(r, world, 1001) for r in range(world)]
        assert got[0][0] == 0 and sum(n for _, n in got) == 1001
        for (a, n), (b, _) in zip(got, got[1:]):
            assert a + n == b
        w = [shard.weak_range(r, world, 50) for r in range(world)]
        assert [b for b, _ in w] == [50 * r for r in range(world)]


def _publisher(rank, port, total, world, fail):
    import datetime
    from torch.distributed import TCPStore
    store = TCPStore("127.0.0.1", port, world, False, timeout=datetime.timedelta(seconds=30))
    if fail:
        raise SystemExit(3)  # the injected failure: this rank exits before publishing
    from oracle import oracle
    tb, nt = shard.strong_range(rank, world, total)
    r = oracle.simulate(synth.tiny12(1).to_text(), 9, tb, nt, 300, meta_ids=[0, 1, 2])
    shard.publish(store, rank, tb, nt, {"final": r["final"], "counts": r["counts"]})


def test_failed_rank_range_is_recomputed(oracle_mod):
    """Three ranks share 45 trajectories; rank 2 fails before publishing.  The
    collector times out on it, finds its id range missing and recomputes it; the
    union equals one single-process run bit for bit."""
    import datetime
    from torch.distributed import TCPStore
    world, total = 3, 45
    port = _free_port()
    store = TCPStore("127.0.0.1", port, world, True, timeout=datetime.timedelta(seconds=30),
                     wait_for_workers=False)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_publisher, args=(r, port, total, world, r == 2)) for r in (1, 2)]
    for p in procs:
        p.start()
    text = synth.tiny12(1).to_text()
    tb0, nt0 = shard.strong_range(0, world, total)
    r0 = oracle_mod.simulate(text, 9, tb0, nt0, 300, meta_ids=[0, 1, 2])
    parts = {0: (tb0, nt0, {"final": r0["final"], "counts": r0["counts"]})}
    parts.update(shard.collect(store, [1, 2], timeout_s=20))
    for p in procs:
        p.join(timeout=120)
    assert procs[0].exitcode == 0 and procs[1].exitcode == 3
    assert sorted(parts) == [0, 1]
    miss = shard.missing_ranges([(b, n) for b, n, _ in parts.values()], total)
    assert miss == [shard.strong_range(2, world, total)]
    for b, n in miss:
        r = oracle_mod.simulate(text, 9, b, n, 300, meta_ids=[0, 1, 2])
        parts["re" + str(b)] = (b, n, {"final": r["final"], "counts": r["counts"]})
    ordered = sorted(parts.values(), key=lambda t: t[0])
    ref = oracle_mod.simulate(text, 9, 0, total, 300, meta_ids=[0, 1, 2])
    assert np.array_equal(np.concatenate([a["final"] for _, _, a in ordered]), ref["final"])
    assert np.array_equal(np.concatenate([a["counts"] for _, _, a in ordered]), ref["counts"])


def test_missing_ranges():
    assert shard.missing_ranges([(0, 10), (20, 5)], 30) == [(10, 10), (25, 5)]
    assert shard.missing_ranges([], 7) == [(0, 7)]
    assert shard.missing_ranges([(0, 7)], 7) == []
