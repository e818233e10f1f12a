"""Python face of the PBN oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  It wraps the plain C simulator in ``pbn_oracle.c`` and
adds the parts that are easiest to read in numpy / the standard library:

* ``stationary``: the unique limiting distribution of the ergodic DTMC of a
  perturbed PBN (Sec. 2.1), by power iteration on the exact transition matrix.
* ``estimate``: the two-state Markov chain estimator of Raftery and Lewis that
  the paper uses for steady-state probabilities (Sec. 4.2, cited there as
  [RL92]); the paper does not print its formulas, so they are written here from
  the published method.  Parity of this part against the paper is unpinned (the
  paper gives no worked example); the tests pin it against matrix powers and
  exact variance sums of a two-state chain instead.

Nothing here imports the product package, and the product never imports this.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from statistics import NormalDist

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-pthread", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, i32, vp, cp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_char_p
            L.orc_philox.argtypes = [vp, vp, vp]
            L.orc_philox.restype = None
            L.orc_simulate.argtypes = [cp, u64, u64, u64, u64, u64, u64, vp, vp, i32,
                                       vp, vp, vp, vp, i32]
            L.orc_simulate.restype = i32
            L.orc_draws.argtypes = [cp, u64, u64, u64, vp, vp, vp, vp]
            L.orc_draws.restype = i32
            L.orc_thresholds.argtypes = [cp, i32, vp, vp]
            L.orc_thresholds.restype = i32
            L.orc_shape.argtypes = [cp, vp, vp, vp, vp]
            L.orc_shape.restype = i32
            L.orc_transition_matrix.argtypes = [cp, vp]
            L.orc_transition_matrix.restype = i32
            L.orc_simulate_sem.argtypes = L.orc_simulate.argtypes + [i32]
            L.orc_simulate_sem.restype = i32
            L.orc_simulate_ex.argtypes = L.orc_simulate.argtypes + [i32, i32]
            L.orc_simulate_ex.restype = i32
            L.orc_draws_ex.argtypes = [cp, u64, u64, u64, i32, vp, vp]
            L.orc_draws_ex.restype = i32
            L.orc_geo_thresholds.argtypes = [ctypes.c_double, vp]
            L.orc_geo_thresholds.restype = None
            L.orc_transition_matrix_sem.argtypes = [cp, i32, vp]
            L.orc_transition_matrix_sem.restype = i32
            L.orc_leaves.argtypes = [cp, vp, i32, vp]
            L.orc_leaves.restype = i32
            L.orc_reach.argtypes = [cp, vp, i32, vp]
            L.orc_reach.restype = i32
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4x32 counter under a 2x32 key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def shape(text: str):
    """(n, number of functions, total parents, p) of a network text."""
    n, nf, sp, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_long(), ctypes.c_double()
    rc = lib().orc_shape(text.encode(), ctypes.byref(n), ctypes.byref(nf),
                         ctypes.byref(sp), ctypes.byref(p))
    if rc:
        raise ValueError(f"oracle could not parse the network (rc={rc})")
    return n.value, nf.value, sp.value, p.value


def simulate(text: str, seed: int, traj_begin: int, n_traj: int, n_steps: int, *,
             meta_ids=(), meta_vals=None, step_begin: int = 0, count_from: int = 0,
             init_states=None, trace: bool = False, nthreads: int = 1, semantics: int = 0,
             sampler: int = 0):
    """Run the Eq. 1 simulator of the unreduced network (semantics=1: the node-wise
    variant, a flipped node negates and the others apply their functions; sampler=1:
    the geometric perturbation sampler instead of the bit-sliced levels).

    Returns dict(final=(n_traj, n) uint8, counts=(n_traj, 5) uint64 as
    [V, n00, n01, n10, n11], trace=(n_traj, n_steps, n) uint8 or None)."""
    n = shape(text)[0]
    meta_ids = np.ascontiguousarray(meta_ids, dtype=np.int32)
    if meta_vals is None:
        meta_vals = np.ones(len(meta_ids), dtype=np.uint8)
    meta_vals = np.ascontiguousarray(meta_vals, dtype=np.uint8)
    init = None if init_states is None else np.ascontiguousarray(init_states, dtype=np.uint8)
    if init is not None:
        assert init.shape == (n_traj, n)
    final = np.zeros((n_traj, n), dtype=np.uint8)
    counts = np.zeros((n_traj, 5), dtype=np.uint64)
    tr = np.zeros((n_traj, n_steps, n), dtype=np.uint8) if trace else None
    rc = lib().orc_simulate_ex(text.encode(), seed, traj_begin, n_traj, step_begin, n_steps,
                               count_from, _ptr(meta_ids), _ptr(meta_vals), len(meta_ids),
                               _ptr(init), _ptr(final), _ptr(counts), _ptr(tr), nthreads, semantics, sampler)
    if rc:
        raise ValueError(f"orc_simulate failed (rc={rc})")
    return {"final": final, "counts": counts, "trace": tr}


def draws(text: str, seed: int, traj: int, step: int):
    """The keyed draws of one (trajectory, step): gamma, choices, keyed s(0), any."""
    n = shape(text)[0]
    g = np.zeros(n, dtype=np.uint8)
    c = np.zeros(n, dtype=np.uint8)
    s0 = np.zeros(n, dtype=np.uint8)
    any_ = ctypes.c_int()
    rc = lib().orc_draws(text.encode(), seed, traj, step, _ptr(g), _ptr(c), _ptr(s0),
                         ctypes.byref(any_))
    if rc:
        raise ValueError(f"orc_draws failed (rc={rc})")
    return g, c, s0, bool(any_.value)


def thresholds(text: str, node: int):
    """(P, [T_1..T_{l-1}]) of one node, as integers."""
    P = ctypes.c_uint64()
    T = np.zeros(16, dtype=np.uint64)
    l = lib().orc_thresholds(text.encode(), node, ctypes.byref(P), _ptr(T))
    if l < 0:
        raise ValueError(f"orc_thresholds failed (rc={l})")
    return int(P.value), [int(t) for t in T[: l - 1]]


def gamma(text: str, seed: int, traj: int, step: int, sampler: int = 0):
    """Perturbation vector of one (trajectory, step) under the given sampler; any."""
    n = shape(text)[0]
    g = np.zeros(n, dtype=np.uint8)
    a = ctypes.c_int()
    rc = lib().orc_draws_ex(text.encode(), seed, traj, step, sampler, _ptr(g), ctypes.byref(a))
    if rc:
        raise ValueError(f"orc_draws_ex failed (rc={rc})")
    return g, bool(a.value)


def geo_thresholds(p: float) -> list:
    """The geometric sampler's thresholds G[0..63] (integers below 2^64)."""
    G = np.zeros(64, dtype=np.uint64)
    lib().orc_geo_thresholds(p, _ptr(G))
    return [int(x) for x in G]


def transition_matrix(text: str, semantics: int = 0) -> np.ndarray:
    """Exact 2^n x 2^n transition matrix (row = current state) for n <= 14
    (semantics=1: the node-wise variant)."""
    n = shape(text)[0]
    if n > 14:
        raise ValueError("transition matrix only for n <= 14")
    M = np.zeros((1 << n, 1 << n), dtype=np.float64)
    rc = lib().orc_transition_matrix_sem(text.encode(), semantics, _ptr(M))
    if rc:
        raise ValueError(f"orc_transition_matrix failed (rc={rc})")
    return M


def leaves(text: str, interest) -> np.ndarray:
    """Leaf flags of Definition 1 for the given nodes of interest."""
    n = shape(text)[0]
    it = np.ascontiguousarray(interest, dtype=np.int32)
    out = np.zeros(n, dtype=np.uint8)
    rc = lib().orc_leaves(text.encode(), _ptr(it), len(it), _ptr(out))
    if rc:
        raise ValueError(f"orc_leaves failed (rc={rc})")
    return out.astype(bool)


def reach_removed(text: str, interest) -> np.ndarray:
    """Nodes from which no node of interest can be reached (the reachability
    variant of the reduction): True = removed."""
    n = shape(text)[0]
    it = np.ascontiguousarray(interest, dtype=np.int32)
    out = np.zeros(n, dtype=np.uint8)
    rc = lib().orc_reach(text.encode(), _ptr(it), len(it), _ptr(out))
    if rc:
        raise ValueError(f"orc_reach failed (rc={rc})")
    return out.astype(bool)


def stationary(M: np.ndarray, tol: float = 1e-15, max_iter: int = 200000):
    """Limiting distribution pi of an ergodic chain: iterate pi <- pi M from the
    uniform distribution until the L1 change is below tol.  Returns (pi, iters)."""
    S = M.shape[0]
    pi = np.full(S, 1.0 / S)
    for it in range(1, max_iter + 1):
        nxt = pi @ M
        nxt /= nxt.sum()
        if np.abs(nxt - pi).sum() < tol:
            return nxt, it
        pi = nxt
    return pi, max_iter


def meta_probability(pi: np.ndarray, n: int, meta_ids, meta_vals=None) -> float:
    """Stationary probability that every listed node holds its value."""
    meta_ids = list(meta_ids)
    if meta_vals is None:
        meta_vals = [1] * len(meta_ids)
    idx = np.arange(1 << n, dtype=np.int64)
    hit = np.ones(1 << n, dtype=bool)
    for i, v in zip(meta_ids, meta_vals):
        hit &= ((idx >> i) & 1) == v
    return float(pi[hit].sum())


def estimate(counts5, n_traj: int, r: float, s: float, eps: float):
    """Two-state Markov chain estimate from pooled counts [V, n00, n01, n10, n11]
    of n_traj trajectories (each contributing its own run of states).

    alpha = n01/(n00+n01), beta = n10/(n10+n11), pi = V / L with L the number of
    counted states; burn-in m* = ceil(log(eps (a+b) / max(a,b)) / log|1-a-b|);
    sample size N* = ceil(a b (2-a-b) / (a+b)^3 * (z/r)^2), z = Phi^-1((1+s)/2).
    Degenerate cases: a zero denominator gives nan for that rate; when a+b == 0
    or either rate is nan, m* and N* are None; when |1-a-b| == 0 the chain mixes
    in one step (m* = 1); when |1-a-b| == 1 (a = b = 1) it never mixes (None)."""
    V, n00, n01, n10, n11 = (int(x) for x in counts5)
    L = n00 + n01 + n10 + n11 + int(n_traj)
    a = n01 / (n00 + n01) if (n00 + n01) else math.nan
    b = n10 / (n10 + n11) if (n10 + n11) else math.nan
    pi = V / L if L else math.nan
    z = NormalDist().inv_cdf((1.0 + s) / 2.0)
    out = {"alpha": a, "beta": b, "pi": pi, "L": L, "z": z,
           "m_star": None, "n_star": None, "n_star_real": math.nan, "var": math.nan}
    if math.isnan(a) or math.isnan(b) or a + b == 0.0:
        return out
    lam = abs(1.0 - a - b)
    if lam == 0.0:
        out["m_star"] = 1
    elif lam < 1.0:
        out["m_star"] = max(1, math.ceil(math.log(eps * (a + b) / max(a, b)) / math.log(lam)))
    nreal = a * b * (2.0 - a - b) / (a + b) ** 3 * (z / r) ** 2
    out["n_star_real"] = nreal
    out["n_star"] = math.ceil(nreal)
    out["var"] = a * b * (2.0 - a - b) / ((a + b) ** 3 * L)
    return out
