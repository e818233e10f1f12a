"""Seeded synthetic PBN generators and the network text format.

This module only produces inputs: it draws random network structures, truth
tables and selection probabilities and writes them as text.  It performs none of
the simulation method's arithmetic and loads no native code, so both the CUDA
library and the independent CPU oracle can read what it writes.

Text format (one record per line, '#' starts a comment):

    pbn <n> <p>
    f <node> <c> <k> <a_0> ... <a_{k-1}> <truth table hex>

The j-th ``f`` line of a node is its predictor function f_j with selection
probability c (Sec. 2.1).  The truth table is an integer written in hex whose bit
x is the output for the input pattern x = sum_b s[a_b] 2^b.  Probabilities are
written as C99 hex floats so that text round-trips exactly.

The workload shapes follow the paper's random PBNs (Sec. 4.1: sizes 20..1000,
0..90% leaves, density 1..8.1) and the five benchmark configurations: a tiny
n = 12 network, a paper-scale n = 100 network with ~25% sinks, a scale-free
n = 2000 network, a batch of networks of uneven size, and a stream of queries.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Function:
    c: float
    parents: list
    tt: int  # bit x = output for input pattern x


@dataclass
class Network:
    n: int
    p: float
    funcs: list = field(default_factory=list)  # funcs[i] = list[Function]

    def to_text(self) -> str:
        lines = [f"pbn {self.n} {float(self.p).hex()}"]
        for i, fl in enumerate(self.funcs):
            for f in fl:
                k = len(f.parents)
                digits = max(1, ((1 << k) + 3) // 4)
                lines.append(f"f {i} {float(f.c).hex()} {k} "
                             + "".join(f"{a} " for a in f.parents)
                             + f"{f.tt:0{digits}x}")
        return "\n".join(lines) + "\n"

    @property
    def n_functions(self) -> int:
        return sum(len(fl) for fl in self.funcs)

    def density(self) -> float:
        """D(G) = (1/n) * sum over functions of their parent counts (Sec. 2.1)."""
        return sum(len(f.parents) for fl in self.funcs for f in fl) / self.n

    def children(self):
        ch = [set() for _ in range(self.n)]
        for u, fl in enumerate(self.funcs):
            for f in fl:
                for a in f.parents:
                    if a != u:
                        ch[a].add(u)
        return ch


def from_text(text: str) -> Network:
    """Parse the text format back into a Network (input handling only)."""
    net = None
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].split()
        if not line:
            continue
        if line[0] == "pbn":
            n = int(line[1])
            net = Network(n=n, p=_num(line[2]), funcs=[[] for _ in range(n)])
        elif line[0] == "f":
            i, c, k = int(line[1]), _num(line[2]), int(line[3])
            parents = [int(a) for a in line[4:4 + k]]
            net.funcs[i].append(Function(c=c, parents=parents, tt=int(line[4 + k], 16)))
        else:
            raise ValueError(f"bad record {line[0]!r}")
    return net


def _num(tok: str) -> float:
    return float.fromhex(tok) if "x" in tok.lower() else float(tok)


def _dirichlet(rng, l):
    if l == 1:
        return [1.0]
    c = rng.dirichlet(np.ones(l))
    return [float(v) for v in c]


def _tt(rng, k):
    bits = rng.integers(0, 2, size=1 << k)
    return int(sum(int(b) << x for x, b in enumerate(bits)))


def random_pbn(seed: int, n: int, p: float, *, ell_choices=(1, 2, 3), ell_probs=None,
               k_choices=(1, 2, 3), k_probs=None, sinks=0.0, protect=(),
               parent_weights=None) -> Network:
    """Random PBN: per node l ~ ell_probs over ell_choices, per function
    k ~ k_probs over k_choices distinct parents, truth-table bits Bernoulli(1/2),
    selection probabilities Dirichlet(1).  A fraction ``sinks`` of the nodes
    (never those in ``protect``) are never chosen as parents.  Parents are drawn
    with probability proportional to ``parent_weights`` (uniform if None)."""
    rng = np.random.default_rng(seed)
    ell_choices = np.asarray(ell_choices)
    k_choices = np.asarray(k_choices)
    sink = np.zeros(n, dtype=bool)
    if sinks > 0:
        cand = np.array([i for i in range(n) if i not in set(protect)])
        m = int(round(sinks * n))
        sink[rng.choice(cand, size=m, replace=False)] = True
    pool = np.flatnonzero(~sink)
    w = np.ones(n) if parent_weights is None else np.asarray(parent_weights, dtype=float)
    wp = w[pool] / w[pool].sum()
    net = Network(n=n, p=p, funcs=[])
    for i in range(n):
        l = int(rng.choice(ell_choices, p=ell_probs))
        cs = _dirichlet(rng, l)
        fl = []
        for j in range(l):
            k = int(rng.choice(k_choices, p=k_probs))
            k = min(k, len(pool))
            par = [int(a) for a in rng.choice(pool, size=k, replace=False, p=wp)]
            fl.append(Function(c=cs[j], parents=par, tt=_tt(rng, k)))
        net.funcs.append(fl)
    return net


# -- the benchmark workload shapes -------------------------------------------------

#: per-function in-degree pmf over {1..5} with mean 2.50 (paper-scale network)
INDEG_PMF_1_5 = (0.26, 0.30, 0.22, 0.12, 0.10)


def tiny12(seed: int = 1) -> Network:
    """n = 12; 1-3 functions per node (uniform); 1-3 distinct inputs drawn
    uniformly from all nodes; p = 0.01; meta-state = nodes 0,1,2 all ON."""
    return random_pbn(seed, 12, 0.01, ell_choices=(1, 2, 3), k_choices=(1, 2, 3))


def paper100(seed: int = 2, n: int = 100, p: float = 1e-4) -> Network:
    """Paper-scale network: 70% of nodes with one function, the rest 2-3;
    in-degree 1-5 per function (mean 2.5); 25% sinks (never parents), which
    excludes the meta nodes 0,1,2; p = 1e-4."""
    return random_pbn(seed, n, p, ell_choices=(1, 2, 3), ell_probs=(0.70, 0.15, 0.15),
                      k_choices=(1, 2, 3, 4, 5), k_probs=INDEG_PMF_1_5,
                      sinks=0.25, protect=(0, 1, 2))


def scalefree2000(seed: int = 3, n: int = 2000, p: float = 1e-5, exponent: float = 2.5) -> Network:
    """Large network: out-degree weights of a power law with the given exponent
    (Chung-Lu style: parents drawn proportionally to w_i = (i + 1)^(-1/(exponent-1))
    over a random permutation of ids), in-degree 1-6 per function, 1-3 functions
    per node, Dirichlet(1) selection probabilities, p = 1e-5; meta = 4 nodes."""
    rng = np.random.default_rng(seed + 7919)
    w = (np.arange(n) + 1.0) ** (-1.0 / (exponent - 1.0))
    w = w[rng.permutation(n)]
    return random_pbn(seed, n, p, ell_choices=(1, 2, 3), k_choices=(1, 2, 3, 4, 5, 6),
                      parent_weights=w)


def apoptosis96(seed: int = 5, n: int = 96, n_leaves: int = 36, total_inputs: int = 171,
                p: float = 1e-4) -> Network:
    """Stand-in with the shape of the paper's apoptosis network (Sec. 4.2: 96 nodes,
    37.5% leaves, density 1.78); the real model is not available.  60 core nodes
    lie on one random directed cycle (each core node's first parent in every
    function is its cycle predecessor, so every core node has a core child and is
    never a leaf); the other 36 nodes are never parents, so Definition 1 removes
    exactly them for any meta-state over core nodes.  l = 1 w.p. 0.7 else 2; further
    parents drawn uniformly from the core; in-degrees adjusted to sum to 171 over
    all functions (density 171 / 96 = 1.78); truth tables Bernoulli(1/2), with
    every core function depending on its cycle predecessor; c ~ Dirichlet(1).
    Core nodes are 0..59 (the meta-state nodes are drawn from them)."""
    rng = np.random.default_rng(seed + 104729)
    core = n - n_leaves
    perm = rng.permutation(core)
    pred = np.empty(core, dtype=int)
    pred[perm] = np.roll(perm, 1)
    ells = [1 if rng.random() < 0.7 else 2 for _ in range(n)]
    ks = [[int(rng.choice((1, 2, 3), p=(0.72, 0.19, 0.09))) for _ in range(l)] for l in ells]
    # adjust the in-degrees so that they sum to total_inputs exactly
    flat = [(i, j) for i in range(n) for j in range(ells[i])]
    while sum(map(sum, ks)) != total_inputs:
        i, j = flat[int(rng.integers(len(flat)))]
        if sum(map(sum, ks)) > total_inputs and ks[i][j] > 1:
            ks[i][j] -= 1
        elif sum(map(sum, ks)) < total_inputs and ks[i][j] < 3:
            ks[i][j] += 1
    net = Network(n=n, p=p, funcs=[])
    for i in range(n):
        cs = _dirichlet(rng, ells[i])
        fl = []
        for j in range(ells[i]):
            k = ks[i][j]
            first = [int(pred[i])] if i < core else []
            others = [int(a) for a in rng.permutation(core) if a not in first and a != i][: k - len(first)]
            par = first + others
            while True:
                tt = _tt(rng, k)
                if i >= core:
                    break
                # the output must depend on input 0 (the cycle predecessor)
                if any(((tt >> x) & 1) != ((tt >> (x | 1)) & 1) for x in range(0, 1 << k, 2)):
                    break
            fl.append(Function(c=cs[j], parents=par, tt=tt))
        net.funcs.append(fl)
    return net


def batch_shapes(seed: int = 4, count: int = 256, n_range=(20, 4000), t_range=(1024, 65536),
                 p_range=(1e-5, 1e-2)):
    """Shapes of the batched workload: (n, n_traj, p) log-uniform per network."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        t = int(round(math.exp(rng.uniform(math.log(t_range[0]), math.log(t_range[1])))))
        p = float(math.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1]))))
        out.append((n, t, p))
    return out


def batch_network(seed: int, n: int, p: float) -> Network:
    """One network of the batched workload: the paper-scale generator at size n."""
    return paper100(seed=seed, n=n, p=p)


def query_text(seed: int, n: int, p: float) -> str:
    """Network text of one served query: the paper-scale recipe of `paper100` (70% of
    nodes with one function, the rest 2-3; in-degree 1-5 per function with the same
    pmf; 25% sinks that are never parents, excluding nodes 0-3, the candidates for a
    query's meta-state; Dirichlet(1) selection probabilities; truth-table bits
    Bernoulli(1/2)), drawn with vectorised numpy calls so that a query stream of
    tens of thousands of networks can be produced as fast as it arrives.  Its random
    stream differs from `paper100`'s (same law, other draws)."""
    rng = np.random.default_rng(seed)
    protect = 4 if n > 4 else 0
    m = int(round(0.25 * n))
    sink = np.zeros(n, dtype=bool)
    if m:
        sink[protect + rng.choice(n - protect, size=min(m, n - protect), replace=False)] = True
    pool = np.flatnonzero(~sink)
    ell = rng.choice(np.array([1, 2, 3]), size=n, p=(0.70, 0.15, 0.15))
    node = np.repeat(np.arange(n), ell)
    nf = node.size
    # Dirichlet(1) per node: normalised unit exponentials
    g = rng.exponential(size=nf)
    first = np.concatenate(([0], np.cumsum(ell)[:-1]))
    c = g / np.repeat(np.add.reduceat(g, first), ell)
    c[np.repeat(ell == 1, ell)] = 1.0
    k = np.minimum(rng.choice(np.arange(1, 6), size=nf, p=INDEG_PMF_1_5), pool.size)
    # k distinct parents per function, uniform over the pool: draw five, redraw clashes
    par = pool[rng.integers(0, pool.size, size=(nf, 5))]
    for _ in range(64):
        clash = np.zeros(nf, dtype=bool)
        for a in range(5):
            for b in range(a):
                clash |= (par[:, a] == par[:, b]) & (a < k)
        if not clash.any():
            break
        par[clash] = pool[rng.integers(0, pool.size, size=(int(clash.sum()), 5))]
    tt = rng.integers(0, 1 << 32, size=nf, dtype=np.uint64) & ((np.uint64(1) << (np.uint64(1) << k.astype(np.uint64))) - np.uint64(1))
    digits = np.maximum(1, ((1 << k) + 3) // 4)
    lines = [f"pbn {n} {float(p).hex()}"]
    for f in range(nf):
        kk = int(k[f])
        lines.append(f"f {node[f]} {float(c[f]).hex()} {kk} " + "".join(f"{a} " for a in par[f, :kk])
                     + f"{int(tt[f]):0{int(digits[f])}x}")
    return "\n".join(lines) + "\n"


def query_text_args(args) -> str:
    """query_text(*args), for process pools."""
    return query_text(*args)
