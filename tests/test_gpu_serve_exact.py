"""Served results against the oracle, exactly (Sec. 4.2's two-state chain estimate).

Ten queries are served together by the continuous-batching server; one of them is
cancelled after two rounds.  The server's settings make the two-state rule restart
counting windows (a burn-in of 2 steps before the first decision, so m* exceeds it)
and grow slow queries (new trajectory blocks with the next ids and their own
counting windows).  For every completed query each trajectory block is replayed by
the oracle -- the plain Eq. 1 simulator of the unreduced network, with the block's
trajectory ids, step count and counting window -- and:

* every trajectory's final state (retained nodes) and its five counts equal the
  oracle's bit for bit;
* the query's pooled counts equal the sum of the oracle's counts over its blocks;
* the query's estimate (pbn_estimate: alpha, beta, pi, m*, N*) equals the oracle's
  two-state formulas on those counts, to 1e-12 for the real numbers and exactly for
  the integers.
"""
import math
import os

import numpy as np
import pytest

from paper_1605_00854_gb300 import api, serve, synth

pytestmark = pytest.mark.gpu

U64_MAX = 2**64 - 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _queries():
    rng = np.random.default_rng(2016)
    qs = []
    for i in range(8):
        n = int(rng.integers(20, 121))
        text = synth.paper100(seed=4100 + i, n=n, p=float(10 ** rng.uniform(-3, -2))).to_text()
        k = int(rng.integers(1, 4))
        meta = sorted(int(x) for x in rng.choice(3, size=k, replace=False))
        vals = [int(v) for v in rng.integers(0, 2, size=k)] if i % 3 == 2 else None
        qs.append(serve.Query(qid=i, text=text, meta_ids=meta, meta_vals=vals,
                              seed=int(rng.integers(1, 2**62)), r=float(rng.choice([0.03, 0.05]))))
    # a slowly mixing small network at a tighter precision: grows its trajectories
    tiny = synth.tiny12(1).to_text()
    qs.append(serve.Query(qid=8, text=tiny, meta_ids=[0, 1, 2], seed=99, r=0.003))
    # the same network at r = 0.001 (N* of millions of states): far from done when cancelled
    qs.append(serve.Query(qid=9, text=tiny, meta_ids=[0, 1, 2], seed=7, r=0.001))
    return qs


def _serve(qs, cancel_qid, kernel):
    srv = serve.Server(n_traj=64, chunk_steps=64, burn_in0=2, min_pairs=1024, max_traj=256, grow_rounds=1,
                       max_steps=1 << 13, record_blocks=True, kernel=kernel, compiled_min_traj=64)
    try:
        for q in qs:
            srv.submit(q)
        steps = 0
        while srv.pending and steps < 10**6 and not any(a.q.qid == cancel_qid and a.rounds >= 2 for a in srv.active):
            srv.step()  # idle until queries are prepared, then rounds
            steps += 1
        srv.cancel(cancel_qid)  # after two of its rounds, with its neighbours in flight
        srv.drain(timeout=600)
    finally:
        srv.close()
    return srv


def _close(a, b):
    if b is None or (isinstance(b, float) and math.isnan(b)):
        return a is None or math.isnan(a)
    return abs(a - b) <= 1e-12 * max(1.0, abs(b))


@pytest.mark.parametrize("kernel", ["batch", "auto"])
def test_served_queries_equal_the_oracle(oracle_mod, kernel):
    qs = _queries()
    cancel = 9
    srv = _serve(qs, cancel, kernel)
    assert cancel in srv.cancelled and srv.in_use == 0 and not srv.failed
    done = {r.qid: r for r in srv.done}
    assert sorted(done) == [q.qid for q in qs if q.qid != cancel]
    # the rule restarted counting windows and grew queries
    assert any(r.restarts > 0 for r in done.values())
    assert any(len(r.blocks) > 1 for r in done.values())
    threads = os.cpu_count() or 1
    for q in qs:
        if q.qid == cancel:
            continue
        r = done[q.qid]
        red, ids = api.Net.load(q.text).reduce(q.meta_ids)
        plan = api.Plan(red)
        total = np.zeros(5, dtype=np.uint64)
        n_eff = 0
        for b in r.blocks:
            orc = oracle_mod.simulate(q.text, q.seed, b["traj_begin"], b["n_traj"], b["steps"],
                                      meta_ids=q.meta_ids, meta_vals=q.meta_vals, count_from=b["count_from"],
                                      nthreads=threads)
            assert np.array_equal(b["counts"].T, orc["counts"]), (q.qid, b["traj_begin"])
            final = plan.unpack(b["state"])
            assert np.array_equal(final[:, ids], orc["final"][:, ids]), (q.qid, b["traj_begin"])
            total += orc["counts"].sum(axis=0, dtype=np.uint64)
            n_eff += b["n_traj"] if b["steps"] >= b["count_from"] else 0
        assert [int(x) for x in total] == r.counts, q.qid
        assert n_eff == r.n_eff
        want = oracle_mod.estimate(total, n_eff, q.r, q.s, q.eps)
        assert r.L == want["L"]
        assert _close(r.alpha, want["alpha"]) and _close(r.beta, want["beta"]) and _close(r.pi, want["pi"])
        assert r.n_star == (U64_MAX if want["n_star"] is None else want["n_star"])
        assert r.m_star == (U64_MAX if want["m_star"] is None else want["m_star"])
        # a query stopped by the rule has enough counted states after a long enough burn-in
        if want["n_star"] is not None and want["m_star"] is not None and r.steps < (1 << 13):
            assert r.L >= want["n_star"]
            assert min(b["count_from"] for b in r.blocks) >= want["m_star"]
