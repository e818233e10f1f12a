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
