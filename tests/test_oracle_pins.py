"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to a value worked by hand from the paper,
a closed form, a library routine, a brute-force recount or an invariant the paper
states, so that a dropped term, a wrong sign/index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden

MASK32 = 0xFFFFFFFF


# ------------------------------------------------------------------ Philox ----
_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
cases = json.loads(sys.stdin.read())
@triton.jit
def k(out_ptr, c_ptr, seed, N: tl.constexpr):
    o = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c_ptr + o * 4 + 0), tl.load(c_ptr + o * 4 + 1),
                           tl.load(c_ptr + o * 4 + 2), tl.load(c_ptr + o * 4 + 3), 10)
    tl.store(out_ptr + o * 4 + 0, a); tl.store(out_ptr + o * 4 + 1, b)
    tl.store(out_ptr + o * 4 + 2, c); tl.store(out_ptr + o * 4 + 3, d)
res = []
for seed, ctr in cases:
    c = torch.tensor(np.array(ctr, dtype=np.uint32).view(np.int32).reshape(1, 4).repeat(2, 0).reshape(-1))
    out = torch.zeros(8, dtype=torch.int32)
    k[(1,)](out, c, seed, N=2)
    res.append([int(v) & 0xFFFFFFFF for v in out.tolist()[:4]])
print(json.dumps(res))
"""


def test_philox_matches_library_philox(oracle_mod):
    """The oracle's Philox4x32-10 equals Triton's library Philox (run by its CPU
    interpreter) on edge and random counters/keys."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    cases = [(0, [0, 0, 0, 0]), ((1 << 64) - 1, [MASK32] * 4),
             (0x0123456789ABCDEF, [1, 2, 3, 4])]
    for _ in range(12):
        seed = int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))
        cases.append((seed, [int(x) for x in rng.integers(0, 1 << 32, size=4)]))
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                          capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctr), want in zip(cases, ref):
        got = oracle_mod.philox(ctr, [seed & MASK32, seed >> 32])
        assert [int(v) for v in got] == want, (seed, ctr)


def _level(oracle_mod, seed, traj, step, word, level):
    """Level `level` (64 lanes) of the PERT stream, from the Philox block alone."""
    c2 = ((step >> 32) & 0xFFFF) | (((traj >> 32) & 0xFFFF) << 16)
    x = oracle_mod.philox([traj & MASK32, step & MASK32, c2, (1 << 28) | (word << 4) | (level // 2)],
                          [seed & MASK32, seed >> 32])
    x = [int(v) for v in x]
    return (x[1] << 32 | x[0]) if level % 2 == 0 else (x[3] << 32 | x[2])


def _net_const(n, p):
    """n nodes, each with the single function 'copy myself'."""
    lines = [f"pbn {n} {float(p).hex()}"] + [f"f {i} 0x1p+0 1 {i} 2" for i in range(n)]
    return "\n".join(lines) + "\n"


# ------------------------------------------------------------ perturbation ----
@pytest.mark.parametrize("p,fn", [
    (0.5, lambda L0, L1: ~L0),           # u < 2^31      <=> bit 31 of u is 0
    (0.25, lambda L0, L1: ~L0 & ~L1),    # u < 2^30      <=> bits 31, 30 are 0
    (0.75, lambda L0, L1: ~(L0 & L1)),   # u < 3 * 2^30  <=> not both set
])
def test_perturbation_closed_forms(oracle_mod, p, fn):
    """For dyadic p the Bernoulli comparison u < P reduces to Boolean functions of
    the top levels; the last word's lanes beyond n are absent (Theorem 1's masking)."""
    n = 70
    text = _net_const(n, p)
    for seed, traj, step in [(7, 0, 0), (2**40 + 5, 2**33 + 9, 2**35 + 11), (99, 12345, 678)]:
        g, _, _, _ = oracle_mod.draws(text, seed, traj, step)
        for w in range(2):
            L0 = _level(oracle_mod, seed, traj, step, w, 0)
            L1 = _level(oracle_mod, seed, traj, step, w, 1)
            want = fn(L0, L1) & ((1 << 64) - 1)
            for b in range(64):
                i = 64 * w + b
                if i < n:
                    assert g[i] == (want >> b) & 1, (seed, traj, step, i)


def test_perturbation_p_zero_never(oracle_mod):
    text = _net_const(10, 0.0)
    for t in range(50):
        g, _, _, any_ = oracle_mod.draws(text, 1, t, t)
        assert not any_ and g.sum() == 0


def test_perturbation_rate_binomial(oracle_mod):
    """Per-lane rate P / 2^32 on full and partial words (Theorem 1 analogue),
    and pairwise independence of two lanes, within 5 sigma."""
    n, p = 70, 0.05
    text = _net_const(n, p)
    P = math.floor(p * 2**32)
    pe = P / 2**32
    hits = np.zeros(n)
    pair = 0
    T = 3000
    for t in range(T):
        g, _, _, _ = oracle_mod.draws(text, 5, t, 3 * t + 1)
        hits += g
        pair += int(g[3]) * int(g[66])
    sd = math.sqrt(pe * (1 - pe) / T)
    for i in range(n):
        assert abs(hits[i] / T - pe) < 5 * sd + 1e-12, i
    sd2 = math.sqrt(pe * pe * (1 - pe * pe) / T)
    assert abs(pair / T - pe * pe) < 5 * sd2 + 1e-12


# ------------------------------------------------------ geometric sampler ----
def test_geo_thresholds_closed_forms(oracle_mod):
    """G[k] = floor(2^64 (1 - (1 - p')^(k+1))): for p = 1/2 the powers are dyadic,
    G[k] = 2^64 - 2^(63 - k); G[0] = P 2^32 for any p; p = 0 gives 0; increasing."""
    G = oracle_mod.geo_thresholds(0.5)
    assert G == [2**64 - 2**(63 - k) for k in range(64)]
    for p in (1e-4, 0.01, 0.3, 0.75):
        G = oracle_mod.geo_thresholds(p)
        P = math.floor(p * 2**32)
        assert G[0] == P * 2**32
        assert all(G[k] < G[k + 1] or G[k] == 2**64 - 1 for k in range(63))
        assert G[63] < 2**64
    assert oracle_mod.geo_thresholds(0.0) == [0] * 64


def _geo_uniform(oracle_mod, seed, traj, step, word, j):
    """The j-th 64-bit uniform of word `word` in the GEO stream, from the Philox
    block alone: x1:x0 for even words, x3:x2 for odd words of block (word/2) << 8 | j."""
    c2 = ((step >> 32) & 0xFFFF) | (((traj >> 32) & 0xFFFF) << 16)
    x = oracle_mod.philox([traj & MASK32, step & MASK32, c2, (4 << 28) | ((word // 2) << 8) | j],
                          [seed & MASK32, seed >> 32])
    x = [int(v) for v in x]
    return (x[1] << 32 | x[0]) if word % 2 == 0 else (x[3] << 32 | x[2])


def test_geo_sampler_closed_form_at_one_half(oracle_mod):
    """At p = 1/2, G[k] = 2^64 - 2^(63-k), so U < G[k] iff the top k+1 bits of U are
    not all ones: the gap to the next perturbed lane is the number of leading ones
    of the uniform, and a word ends when that count reaches the lanes left.  The
    perturbation vector follows from the Philox blocks alone (70 nodes: a full and a
    partial word)."""
    n = 70
    text = _net_const(n, 0.5)
    for seed, traj, step in [(7, 0, 0), (2**40 + 5, 2**33 + 9, 2**35 + 11), (99, 12345, 678), (3, 1, 2)]:
        g, _ = oracle_mod.gamma(text, seed, traj, step, sampler=1)
        want = np.zeros(n, dtype=np.uint8)
        for w in range(2):
            L = min(64, n - 64 * w)
            pos, j = 0, 0
            while pos < L:
                U = _geo_uniform(oracle_mod, seed, traj, step, w, j)
                j += 1
                ones = 64 - (((~U) & (2**64 - 1)).bit_length())  # leading one bits
                if ones >= L - pos:
                    break
                want[64 * w + pos + ones] = 1
                pos += ones + 1
        assert np.array_equal(g, want), (seed, traj, step)


def test_geo_sampler_rate_and_independence(oracle_mod):
    """The geometric sampler draws i.i.d. Bernoulli(P / 2^32) lanes: per-lane rate
    on full and partial words and pairwise independence within 5 sigma."""
    n, p = 70, 0.05
    text = _net_const(n, p)
    pe = math.floor(p * 2**32) / 2**32
    hits = np.zeros(n)
    pair = pair2 = 0
    T = 3000
    for t in range(T):
        g, _ = oracle_mod.gamma(text, 5, t, 3 * t + 1, sampler=1)
        hits += g
        pair += int(g[3]) * int(g[66])
        pair2 += int(g[10]) * int(g[11])
    sd = math.sqrt(pe * (1 - pe) / T)
    for i in range(n):
        assert abs(hits[i] / T - pe) < 5 * sd + 1e-12, i
    sd2 = math.sqrt(pe * pe * (1 - pe * pe) / T)
    assert abs(pair / T - pe * pe) < 5 * sd2 + 1e-12
    assert abs(pair2 / T - pe * pe) < 5 * sd2 + 1e-12


def test_geo_sampler_word_law(oracle_mod):
    """A 3-node network at p = 0.3: the frequency of each of the 8 perturbation
    patterns follows the product of independent Bernoulli(p') lanes (5 sigma)."""
    p = 0.3
    text = _net_const(3, p)
    pe = math.floor(p * 2**32) / 2**32
    T = 20000
    cnt = np.zeros(8)
    for t in range(T):
        g, _ = oracle_mod.gamma(text, 11, t, 7, sampler=1)
        cnt[int(g[0]) + 2 * int(g[1]) + 4 * int(g[2])] += 1
    for pat in range(8):
        k = bin(pat).count("1")
        q = pe**k * (1 - pe) ** (3 - k)
        assert abs(cnt[pat] / T - q) < 5 * math.sqrt(q * (1 - q) / T), pat


def test_geo_sampler_reaches_exact_pi(oracle_mod):
    """With the geometric sampler the n = 12 network's meta-state frequency still
    agrees with pi(meta) of the exact matrix (same law to 2^-64)."""
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    pi, _ = oracle_mod.stationary(oracle_mod.transition_matrix(text))
    target = oracle_mod.meta_probability(pi, 12, meta)
    r = oracle_mod.simulate(text, 1, 0, 64, 10000, meta_ids=meta, count_from=100, nthreads=8, sampler=1)
    c = r["counts"].astype(np.float64)
    per = c[:, 0] / (c[:, 1:].sum(axis=1) + 1)
    se = per.std(ddof=1) / math.sqrt(len(per))
    assert abs(per.mean() - target) < 5 * se + 1e-3
    # and it is a different stream of draws than the bit-sliced sampler
    r0 = oracle_mod.simulate(text, 1, 0, 64, 10000, meta_ids=meta, count_from=100, nthreads=8)
    assert not np.array_equal(r0["counts"], r["counts"])


# ---------------------------------------------------------------- selection ----
def test_selection_thresholds_dyadic(oracle_mod):
    text = golden("tiny2.pbn")
    P, T = oracle_mod.thresholds(text, 0)
    assert P == 2**28 and T == [2**30]
    P, T = oracle_mod.thresholds(text, 1)
    assert T == []


def test_selection_rank_and_lane(oracle_mod):
    """Only nodes 1 and 3 have >= 2 functions, so they take ranks 0 and 1 and read
    words x0 and x1 of the first SEL block.  Node 3 has three functions with
    c = (1/2, 1/4, 1/4): T_1 = 2^31, T_2 = 3 * 2^30."""
    text = ("pbn 4 0x1p-5\n"
            "f 0 0x1p+0 1 0 2\n"
            "f 1 0x1p-1 1 0 2\nf 1 0x1p-1 1 0 1\n"
            "f 2 0x1p+0 1 1 2\n"
            "f 3 0x1p-1 1 2 2\nf 3 0x1p-2 1 2 1\nf 3 0x1p-2 0 1\n")
    for seed, traj, step in [(3, 0, 0), (11, 77, 5), (2**50, 2**34, 2**33 + 1)]:
        _, ch, _, _ = oracle_mod.draws(text, seed, traj, step)
        c2 = ((step >> 32) & 0xFFFF) | (((traj >> 32) & 0xFFFF) << 16)
        x = [int(v) for v in oracle_mod.philox([traj & MASK32, step & MASK32, c2, 2 << 28],
                                               [seed & MASK32, seed >> 32])]
        assert ch[0] == 0 and ch[2] == 0
        assert ch[1] == (1 if x[0] >= 2**31 else 0)
        assert ch[3] == (x[1] >= 2**31) + (x[1] >= 3 * 2**30)


def test_selection_frequencies(oracle_mod):
    text = ("pbn 2 0x1p-5\n"
            "f 0 0x1.3333333333333p-2 1 0 2\nf 0 0x1p-1 1 0 1\n"
            "f 0 0x1.999999999999ap-3 0 1\n"
            "f 1 0x1p+0 1 0 2\n")
    c = [float.fromhex("0x1.3333333333333p-2"), float.fromhex("0x1p-1"),
         float.fromhex("0x1.999999999999ap-3")]
    T = 4000
    cnt = np.zeros(3)
    for t in range(T):
        _, ch, _, _ = oracle_mod.draws(text, 17, t, 2 * t)
        cnt[ch[0]] += 1
    for j in range(3):
        sd = math.sqrt(c[j] * (1 - c[j]) / T)
        assert abs(cnt[j] / T - c[j]) < 5 * sd


def test_initial_state_words(oracle_mod):
    """s(0): word w is x1:x0 (even w) or x3:x2 (odd w) of INIT block w / 2."""
    n = 130
    text = _net_const(n, 0.01)
    seed, traj = 42, 2**33 + 3
    _, _, s0, _ = oracle_mod.draws(text, seed, traj, 999)
    for w in range(3):
        x = [int(v) for v in oracle_mod.philox([traj & MASK32, 0, ((traj >> 32) & 0xFFFF) << 16,
                                                (3 << 28) | (w >> 1)], [seed & MASK32, seed >> 32])]
        word = (x[1] << 32 | x[0]) if w % 2 == 0 else (x[3] << 32 | x[2])
        for b in range(64):
            if 64 * w + b < n:
                assert s0[64 * w + b] == (word >> b) & 1


def test_truth_table_input_order(oracle_mod):
    """Text format: bit x of a truth table (hex, least significant digit last) is the
    output for inputs a_0..a_{k-1} with a_b the b-th bit of x.  At p = 0 one step is
    deterministic: node 3 = f(s0, s1) with table 0x2 is 1 exactly when s0 = 1 and
    s1 = 0; node 4 with parents (1, 0) and the same table exactly when s1 = 1 and
    s0 = 0; node 5 with parents (0, 1, 2) and the two-digit table 0x10 (bit 4) exactly
    when s0 = s1 = 0 and s2 = 1."""
    text = ("pbn 6 0x0p+0\n"
            "f 0 0x1p+0 1 0 2\n"
            "f 1 0x1p+0 1 1 2\n"
            "f 2 0x1p+0 1 2 2\n"
            "f 3 0x1p+0 2 0 1 2\n"
            "f 4 0x1p+0 2 1 0 2\n"
            "f 5 0x1p+0 3 0 1 2 10\n")
    init = np.array([[a, b, c, 0, 0, 0] for a in (0, 1) for b in (0, 1) for c in (0, 1)], dtype=np.uint8)
    r = oracle_mod.simulate(text, 1, 0, len(init), 1, meta_ids=[0], init_states=init)
    for (a, b, c, _, _, _), fin in zip(init, r["final"]):
        assert list(fin[:3]) == [a, b, c]
        assert fin[3] == (1 if (a, b) == (1, 0) else 0), (a, b)
        assert fin[4] == (1 if (a, b) == (0, 1) else 0), (a, b)
        assert fin[5] == (1 if (a, b, c) == (0, 0, 1) else 0), (a, b, c)


# ------------------------------------------------------ Eq. 1 transition law ----
def _golden_matrix():
    rows = [l.split() for l in golden("tiny2_matrix.txt").splitlines()
            if l.strip() and not l.startswith("#")]
    return [[Fraction(int(v), 1024) for v in r] for r in rows]


def test_transition_matrix_hand_worked(oracle_mod):
    M = oracle_mod.transition_matrix(golden("tiny2.pbn"))
    want = _golden_matrix()
    for s in range(4):
        for t in range(4):
            assert M[s, t] == float(want[s][t]), (s, t)


def _exact_stationary(Q):
    """Solve pi Q = pi, sum pi = 1 with exact rationals (Gauss-Jordan)."""
    S = len(Q)
    A = [[Q[j][i] - (1 if i == j else 0) for j in range(S)] for i in range(S)]
    A[-1] = [Fraction(1)] * S
    b = [Fraction(0)] * (S - 1) + [Fraction(1)]
    for c in range(S):
        piv = next(r for r in range(c, S) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        b[c], b[piv] = b[piv], b[c]
        for r in range(S):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
                b[r] -= f * b[c]
    return [b[i] / A[i][i] for i in range(S)]


def test_stationary_matches_exact_solution(oracle_mod):
    """Power iteration on the oracle's matrix equals the exact rational solution of
    pi Q = pi built from the hand-worked matrix (the limiting distribution that
    ergodicity guarantees, Sec. 2.1)."""
    pi_exact = _exact_stationary(_golden_matrix())
    pi, it = oracle_mod.stationary(oracle_mod.transition_matrix(golden("tiny2.pbn")))
    for s in range(4):
        assert abs(pi[s] - float(pi_exact[s])) < 1e-14


@pytest.mark.parametrize("p", [0.01, 0.3])
def test_stationary_single_node_closed_forms(oracle_mod, p):
    """One node with f = constant 1: pi(1) = 1 / (1 + p').  One node with f = x:
    pi = (1/2, 1/2)."""
    pe = math.floor(p * 2**32) / 2**32
    M = oracle_mod.transition_matrix(f"pbn 1 {p.hex()}\nf 0 0x1p+0 0 1\n")
    pi, _ = oracle_mod.stationary(M)
    assert abs(pi[1] - 1 / (1 + pe)) < 1e-13
    M = oracle_mod.transition_matrix(f"pbn 1 {p.hex()}\nf 0 0x1p+0 1 0 2\n")
    pi, _ = oracle_mod.stationary(M)
    assert abs(pi[0] - 0.5) < 1e-13


def test_one_step_empirical_law(oracle_mod):
    """Many independent keyed trajectories, one step from each fixed state: the
    next-state frequencies follow the hand-worked row within 5 sigma."""
    text = golden("tiny2.pbn")
    Q = _golden_matrix()
    T = 20000
    for s in range(4):
        init = np.array([[s & 1, (s >> 1) & 1]] * T, dtype=np.uint8)
        out = oracle_mod.simulate(text, 1234 + s, 0, T, 1, init_states=init)["final"]
        idx = out[:, 0].astype(int) + 2 * out[:, 1].astype(int)
        for t in range(4):
            q = float(Q[s][t])
            sd = math.sqrt(q * (1 - q) / T)
            assert abs((idx == t).mean() - q) <= 5 * sd + 1e-12, (s, t)


# ------------------------------------------------ node-wise semantics variant ----
def _golden_matrix_pernode():
    rows = [l.split() for l in golden("tiny2_matrix_pernode.txt").splitlines()
            if l.strip() and not l.startswith("#")]
    return [[Fraction(int(v), 1024) for v in r] for r in rows]


def test_pernode_matrix_hand_worked(oracle_mod):
    """Node-wise reading of Sec. 2.1: the exact matrix equals the hand-worked one."""
    M = oracle_mod.transition_matrix(golden("tiny2.pbn"), semantics=1)
    want = _golden_matrix_pernode()
    for s in range(4):
        for t in range(4):
            assert M[s, t] == float(want[s][t]), (s, t)


def test_pernode_one_step_empirical_law(oracle_mod):
    """The node-wise simulator's one-step frequencies follow the hand-worked rows."""
    text = golden("tiny2.pbn")
    Q = _golden_matrix_pernode()
    T = 20000
    for s in range(4):
        init = np.array([[s & 1, (s >> 1) & 1]] * T, dtype=np.uint8)
        out = oracle_mod.simulate(text, 4321 + s, 0, T, 1, init_states=init, semantics=1)["final"]
        idx = out[:, 0].astype(int) + 2 * out[:, 1].astype(int)
        for t in range(4):
            q = float(Q[s][t])
            sd = math.sqrt(q * (1 - q) / T)
            assert abs((idx == t).mean() - q) <= 5 * sd + 1e-12, (s, t)


def test_pernode_equals_global_when_no_flip_and_single_node(oracle_mod):
    """Two special cases fix the node-wise variant against Eq. 1: with p = 0 both
    readings are the same chain, and for a single node they coincide for every p
    (a flip of the only node is the whole perturbation vector)."""
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(2).to_text().replace("pbn 12 " + (0.01).hex(), "pbn 12 0x0p+0")
    assert "pbn 12 0x0p+0" in text
    a = oracle_mod.simulate(text, 5, 0, 8, 300, trace=True)
    b = oracle_mod.simulate(text, 5, 0, 8, 300, trace=True, semantics=1)
    assert np.array_equal(a["trace"], b["trace"])
    one = "pbn 1 0x1p-3\nf 0 0x1p-1 1 0 2\nf 0 0x1p-1 1 0 1\n"
    assert np.array_equal(oracle_mod.transition_matrix(one), oracle_mod.transition_matrix(one, semantics=1))
    a = oracle_mod.simulate(one, 6, 0, 4, 500, trace=True)
    b = oracle_mod.simulate(one, 6, 0, 4, 500, trace=True, semantics=1)
    assert np.array_equal(a["trace"], b["trace"])


def test_pernode_rows_are_distributions(oracle_mod):
    from paper_1605_00854_gb300 import synth
    M = oracle_mod.transition_matrix(synth.tiny12(1).to_text(), semantics=1)
    assert np.allclose(M.sum(axis=1), 1.0, atol=1e-12) and (M >= 0).all()


# ---------------------------------------------------------------- counting ----
def _recount(trace_states, s_start, meta, start_index, count_from, vals=None):
    """Brute-force counts from a list of states s(start_index), s(start_index+1)...
    (meta-state: node meta[m] holds vals[m], default 1)."""
    vals = [1] * len(meta) if vals is None else list(vals)
    z = [int(all(st[m] == v for m, v in zip(meta, vals))) for st in [s_start] + list(trace_states)]
    V = sum(zi for k, zi in enumerate(z) if start_index + k >= count_from)
    n = [0, 0, 0, 0]
    for k in range(1, len(z)):
        if start_index + k - 1 >= count_from:
            n[2 * z[k - 1] + z[k]] += 1
    return [V] + n


@pytest.mark.parametrize("count_from,vals", [(0, None), (1, None), (37, None), (0, [0, 1, 0]), (5, [1, 0, 0])])
def test_counts_match_bruteforce_recount(oracle_mod, count_from, vals):
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    r = oracle_mod.simulate(text, 9, 0, 6, 300, meta_ids=meta, meta_vals=vals, count_from=count_from, trace=True)
    init = np.zeros((6, 12), dtype=np.uint8)
    for t in range(6):
        init[t] = oracle_mod.draws(text, 9, t, 0)[2]
    assert 0 < int(r["counts"][:, 0].sum()) < 6 * 301  # the meta-state is visited, and left
    for t in range(6):
        want = _recount(r["trace"][t], init[t], meta, 0, count_from, vals)
        assert list(map(int, r["counts"][t])) == want
        c = r["counts"][t]
        L = 300 + 1 - count_from
        assert int(c[1] + c[2] + c[3] + c[4]) == L - 1


@pytest.mark.parametrize("count_from", [0, 1, 50, 199, 200, 201, 400, 500])
def test_resume_equals_one_run(oracle_mod, count_from):
    """S steps, then S more from the saved state, equals 2S steps in one run
    (states at every step and the summed counts), wherever the counting window
    starts: before the cut, just before, at, just after it, at the end, beyond it."""
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(1).to_text()
    meta = [11]  # a meta-state that is ON at the cut in some trajectories (8 of 16)
    full = oracle_mod.simulate(text, 4, 100, 16, 400, meta_ids=meta, trace=True, count_from=count_from)
    a = oracle_mod.simulate(text, 4, 100, 16, 200, meta_ids=meta, trace=True, count_from=count_from)
    b = oracle_mod.simulate(text, 4, 100, 16, 200, meta_ids=meta, trace=True, count_from=count_from,
                            step_begin=200, init_states=a["final"])
    assert 0 < int(a["final"][:, meta[0]].sum()) < 16
    assert np.array_equal(full["trace"], np.concatenate([a["trace"], b["trace"]], axis=1))
    assert np.array_equal(full["counts"], a["counts"] + b["counts"])
    # and the window is what it says: max(0, 400 + 1 - count_from) states per trajectory
    L = max(0, 401 - count_from)
    assert np.all(full["counts"][:, 1:].sum(axis=1) + (1 if L else 0) == L)


# ------------------------------------------------------------------ leaves ----
def test_leaves_hand_worked(oracle_mod):
    leaf = oracle_mod.leaves(golden("leaves7.pbn"), [1])
    assert sorted(np.flatnonzero(leaf).tolist()) == [2, 3, 6]


def test_reach_variant_hand_example(oracle_mod):
    removed = oracle_mod.reach_removed(golden("leaves7.pbn"), [1])
    assert sorted(np.flatnonzero(removed).tolist()) == [2, 3, 4, 5, 6]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_reach_variant_equals_graph_ancestors(oracle_mod, seed):
    """The reachability variant keeps exactly the nodes of interest and their
    ancestors in the parent -> child graph (networkx's ancestors on the same edges),
    and keeps no more than Definition 1 does."""
    nx = pytest.importorskip("networkx")
    from paper_1605_00854_gb300 import synth
    net = synth.random_pbn(seed, 50, 0.01, k_choices=(1, 2), sinks=0.3, protect=(0, 1))
    G = nx.DiGraph()
    G.add_nodes_from(range(net.n))
    for u, fl in enumerate(net.funcs):
        for f in fl:
            for a in f.parents:
                if a != u:
                    G.add_edge(a, u)
    keep = {0, 1} | nx.ancestors(G, 0) | nx.ancestors(G, 1)
    removed = oracle_mod.reach_removed(net.to_text(), [0, 1])
    assert set(np.flatnonzero(~removed).tolist()) == keep
    leaf = oracle_mod.leaves(net.to_text(), [0, 1])
    assert not np.any(~removed & leaf)      # kept by reachability => kept by Definition 1


def test_reach_removed_tables_do_not_affect_kept_nodes(oracle_mod):
    """Nodes that reach no node of interest cannot influence the kept nodes:
    rewriting their truth tables keeps the kept nodes' trajectories identical."""
    from paper_1605_00854_gb300 import synth
    net = synth.random_pbn(4, 60, 0.01, k_choices=(1, 2, 3), sinks=0.2, protect=(0, 1, 2))
    text = net.to_text()
    meta = [0, 1, 2]
    removed = oracle_mod.reach_removed(text, meta)
    assert removed.sum() >= 5
    base = oracle_mod.simulate(text, 3, 0, 4, 500, meta_ids=meta, trace=True)
    rng = np.random.default_rng(1)
    for i in np.flatnonzero(removed):
        for f in net.funcs[i]:
            f.tt = int(rng.integers(0, 1 << (1 << len(f.parents))))
    alt = oracle_mod.simulate(net.to_text(), 3, 0, 4, 500, meta_ids=meta, trace=True)
    keep = ~removed
    assert np.array_equal(base["trace"][:, :, keep], alt["trace"][:, :, keep])
    assert np.array_equal(base["counts"], alt["counts"])


def test_leaf_tables_do_not_affect_retained_nodes(oracle_mod):
    """Sec. 3.1: removing leaves leaves every other node's simulation unchanged.
    Rewriting the truth tables of the oracle's leaves keeps the retained nodes'
    trajectories bit-identical; rewriting one retained node's table changes them."""
    from paper_1605_00854_gb300 import synth
    net = synth.paper100(seed=5, n=60, p=0.01)
    text = net.to_text()
    meta = [0, 1, 2]
    leaf = oracle_mod.leaves(text, meta)
    assert leaf.sum() >= 10 and not leaf[meta].any()
    base = oracle_mod.simulate(text, 3, 0, 4, 500, meta_ids=meta, trace=True)
    rng = np.random.default_rng(0)
    for i in np.flatnonzero(leaf):
        for f in net.funcs[i]:
            f.tt = int(rng.integers(0, 1 << (1 << len(f.parents))))
    alt = oracle_mod.simulate(net.to_text(), 3, 0, 4, 500, meta_ids=meta, trace=True)
    keep = ~leaf
    assert np.array_equal(base["trace"][:, :, keep], alt["trace"][:, :, keep])
    assert np.array_equal(base["counts"], alt["counts"])
    j = int(np.flatnonzero(keep & (np.arange(60) > 2))[0])
    net.funcs[j][0].tt ^= (1 << (1 << len(net.funcs[j][0].parents))) - 1
    bad = oracle_mod.simulate(net.to_text(), 3, 0, 4, 500, meta_ids=meta, trace=True)
    assert not np.array_equal(base["trace"][:, :, keep], bad["trace"][:, :, keep])


# ----------------------------------------------------- stationary vs simulation ----
def test_simulation_meets_exact_stationary_probability(oracle_mod):
    """Tiny n = 12 network: the meta-state frequency of 64 keyed trajectories of
    10^4 steps agrees with pi(meta) from power iteration on the 4096 x 4096
    matrix within 5 standard errors of the per-trajectory means."""
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(1).to_text()
    meta = [0, 1, 2]
    M = oracle_mod.transition_matrix(text)
    assert np.allclose(M.sum(axis=1), 1.0, atol=1e-12)
    pi, _ = oracle_mod.stationary(M)
    target = oracle_mod.meta_probability(pi, 12, meta)
    r = oracle_mod.simulate(text, 1, 0, 64, 10000, meta_ids=meta, count_from=100, nthreads=8)
    c = r["counts"].astype(np.float64)
    per = c[:, 0] / (c[:, 1:].sum(axis=1) + 1)
    se = per.std(ddof=1) / math.sqrt(len(per))
    assert abs(per.mean() - target) < 5 * se + 1e-3


# --------------------------------------------------------------- estimator ----
@pytest.mark.parametrize("a,b", [(0.1, 0.1), (0.02, 0.3), (0.4, 0.7), (0.05, 0.01)])
def test_estimator_burn_in_against_matrix_powers(oracle_mod, a, b):
    """m* of the two-state chain: after m* steps every row of Q^m is within eps of
    the limit, and m* - 1 steps are not enough (checked with numpy matrix powers)."""
    N = 10**6
    n01, n00 = round(a * N), N - round(a * N)
    n10, n11 = round(b * N), N - round(b * N)
    eps = 1e-3
    est = oracle_mod.estimate([0, n00, n01, n10, n11], 1, 0.01, 0.95, eps)
    aa, bb = n01 / N, n10 / N
    Q = np.array([[1 - aa, aa], [bb, 1 - bb]])
    lim = np.array([bb, aa]) / (aa + bb)
    m = est["m_star"]
    dev = lambda k: np.abs(np.linalg.matrix_power(Q, k) - lim[None, :]).max()
    assert dev(m) <= eps * (1 + 1e-9)
    if m > 1:
        assert dev(m - 1) > eps


@pytest.mark.parametrize("a,b", [(0.1, 0.1), (0.02, 0.3), (0.4, 0.7)])
def test_estimator_sample_size_against_exact_variance(oracle_mod, a, b):
    """N* of the two-state chain: the exact variance of the mean of N stationary
    steps, summed from the autocovariances lambda^|i-j|, times N tends to the
    asymptotic variance the estimator uses; N* is the smallest N with
    z * sqrt(var / N) <= r."""
    r, s = 0.01, 0.95
    M = 10**6
    counts = [0, M - round(a * M), round(a * M), round(b * M), M - round(b * M)]
    est = oracle_mod.estimate(counts, 1, r, s, 1e-3)
    aa, bb = counts[2] / M, counts[3] / M
    lam = 1 - aa - bb
    pi = aa / (aa + bb)
    N = est["n_star"]
    k = np.arange(1, N)
    exact = pi * (1 - pi) * (N + 2 * np.sum((N - k) * lam ** k)) / N**2
    z = est["z"]
    assert z * math.sqrt(exact) <= r * (1 + 5.0 / N * (1 + abs(lam)) / (1 - abs(lam)) ** 2)
    asym = est["n_star_real"]
    assert asym <= N < asym + 1


def test_estimate_counts_every_counted_state(oracle_mod):
    """L is the number of counted states, the first counted state of each trajectory
    included: T trajectories of S steps counted from step 0 give L = T (S + 1), and
    pi = V / L."""
    from paper_1605_00854_gb300 import synth
    text = synth.tiny12(1).to_text()
    T, S = 16, 300
    r = oracle_mod.simulate(text, 3, 0, T, S, meta_ids=[0, 1, 2], count_from=0)
    c = r["counts"].sum(axis=0)
    est = oracle_mod.estimate(c, T, 0.01, 0.95, 1e-3)
    assert est["L"] == T * (S + 1)
    assert est["pi"] == int(c[0]) / (T * (S + 1))


def test_worked_sample_size_number(oracle_mod):
    """alpha = beta = 0.1, r = 0.01, s = 0.95: a b (2-a-b)/(a+b)^3 = 2.25 and
    (1.959964 / 0.01)^2 = 38414.59, so N* = ceil(86432.82) = 86433 (worked by hand)."""
    est = oracle_mod.estimate([0, 900, 100, 100, 900], 1, 0.01, 0.95, 1e-3)
    assert est["n_star"] == 86433


def test_normal_quantile_matches_library(oracle_mod):
    sp = pytest.importorskip("scipy.special")
    for s in [0.5, 0.8, 0.9, 0.95, 0.99, 0.999999]:
        est = oracle_mod.estimate([1, 10, 5, 5, 10], 1, 0.01, s, 1e-3)
        assert abs(est["z"] - sp.ndtri((1 + s) / 2)) < 1e-12
