"""CPU tests of the library's host side: the C ABI, parsing, Definition 1 reduction,
grouping (Eq. 2, Algorithms 3-4), merged tables, thresholds and the estimator."""
import math
import os
import re

import numpy as np
import pytest

from conftest import ROOT, golden
import imgdecode
from paper_1605_00854_gb300 import _lib, api, synth


@pytest.fixture(scope="module")
def L():
    return _lib.load()


def test_library_exports_every_declared_symbol(L):
    """libpbn.so loads without a GPU and exports every function include/pbn.h declares."""
    hdr = open(os.path.join(ROOT, "include", "pbn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(pbn_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(L, name), name
        assert name in _lib.SIGNATURES, name
    assert set(_lib.SIGNATURES) == declared


def test_version_and_errors(L):
    assert b"sm_103a" in L.pbn_version()
    with pytest.raises(_lib.PbnError) as e:
        api.Net.load("pbn 2 0.1\nf 0 1.0 1 5 2\nf 1 1.0 0 1\n")
    assert e.value.status == -2 and "parent" in str(e.value)


@pytest.mark.parametrize("text", [
    "",                                          # no header
    "pbn 0 0.1\n",                               # n < 1
    "pbn 2 1.0\nf 0 1 0 1\nf 1 1 0 1\n",         # p = 1
    "pbn 2 0.1\nf 0 1 0 1\n",                    # node 1 has no function
    "pbn 2 0.1\nf 0 0.5 0 1\nf 1 1 0 1\n",       # probabilities sum to 0.5
    "pbn 2 0.1\nf 0 1 1 0 4\nf 1 1 0 1\n",       # truth table wider than 2^k bits
    "pbn 2 0.1\nf 0 1 2 1 1 3\nf 1 1 0 1\n",     # repeated parent
    "pbn 2 0.1\nf 0 1 1 0 z\nf 1 1 0 1\n",       # bad hex digit
    "pbn 2 0.1\nq 0\n",                          # unknown record
])
def test_parse_errors(text):
    with pytest.raises(_lib.PbnError) as e:
        api.Net.load(text)
    assert e.value.status == -2


def test_info_matches_oracle_shape(oracle_mod):
    for seed in range(3):
        net = synth.paper100(seed=seed, n=80)
        text = net.to_text()
        info = api.Net.load(text).info()
        n, nf, sp, p = oracle_mod.shape(text)
        assert (info.n, info.n_functions, info.p) == (n, nf, p)
        assert info.density == pytest.approx(sp / n, rel=1e-15) == net.density()
        assert info.P == math.floor(p * 2**32)


# ---------------------------------------------------------------- reduction ----
def test_reduce_hand_worked():
    net, ids = api.Net.load(golden("leaves7.pbn")).reduce([1])
    assert ids.tolist() == [0, 1, 4, 5]
    assert net.info().n_retained == 4


@pytest.mark.parametrize("seed", range(6))
def test_reduce_matches_oracle_definition(oracle_mod, seed):
    """The library's peeling reduction equals the oracle's literal iteration of
    Definition 1 on random networks with sinks, self-loops and cycles."""
    n = [30, 60, 100, 12, 200, 45][seed]
    net = synth.paper100(seed=100 + seed, n=n, p=0.01) if seed != 3 else synth.tiny12(seed)
    text = net.to_text()
    interest = [0, 1, 2][: 1 + seed % 3]
    leaf = oracle_mod.leaves(text, interest)
    _, ids = api.Net.load(text).reduce(interest)
    assert ids.tolist() == np.flatnonzero(~leaf).tolist()


# ----------------------------------------------------------------- grouping ----
def _plan(text, interest=(0, 1, 2), **kw):
    net = api.Net.load(text)
    red, ids = net.reduce(list(interest))
    return api.Plan(red, **kw), ids


@pytest.mark.parametrize("mode,max_inputs", [(0, 8), (0, 4), (0, 12), (1, 8)])
def test_layout_is_a_valid_grouping(mode, max_inputs):
    net = synth.paper100(seed=2)
    plan, ids = _plan(net.to_text(), mode=mode, max_inputs=max_inputs)
    pos = plan.layout()
    grp = plan.groups()
    retained = set(ids.tolist())
    for i in range(net.n):
        assert (pos[i] != 0xFFFFFFFF) == (i in retained)
    kept = pos[pos != 0xFFFFFFFF]
    assert len(set(kept.tolist())) == len(kept)
    assert kept.max() < 32 * 2 * plan.info.state_words
    # a group occupies consecutive bits of one 32-bit word
    for g in set(grp[grp != 0xFFFFFFFF].tolist()):
        members = sorted(pos[grp == g].tolist())
        assert members[-1] - members[0] == len(members) - 1
        assert members[0] // 32 == members[-1] // 32
        assert len(members) <= 32
        if mode == 1:
            assert len(members) == 1
    # the merge caps hold for every merged group; a lone multi-function node whose
    # inputs exceed the cap is split (one table per function)
    D = imgdecode.decode(plan.image())
    for g, G in enumerate(D["groups"]):
        width = int((grp == g).sum())
        if width > 1:
            assert G["q"] <= max_inputs and G["l2w"] != imgdecode.SPLIT
        if G["l2w"] == imgdecode.SPLIT:
            (v,) = np.flatnonzero(grp == g).tolist()
            fs = net.funcs[v]
            assert G["q"] == len(fs) >= 2 and G["n_mul"] == 1
            assert len(set(a for f in fs for a in f.parents)) > max_inputs
        elif width == 1 and G["q"] > max_inputs:
            assert len(net.funcs[int(np.flatnonzero(grp == g)[0])]) == 1
    assert plan.info.n_split == sum(G["l2w"] == imgdecode.SPLIT for G in D["groups"])


def test_plain_mode_unreduced_is_identity_layout():
    net = synth.tiny12(1)
    plan = api.Plan(api.Net.load(net.to_text()), mode=1)
    assert plan.layout().tolist() == list(range(12))
    assert plan.info.n_groups == 12


def _eq2(omegas, theta):
    L = sum(math.log(w) for w in omegas)
    m = 1
    while m <= max(len(omegas), math.ceil(L) + 2):
        if math.log(m) + L / m <= math.log(theta) + 1e-12:
            return m
        m += 1
    return 0


@pytest.mark.parametrize("seed,theta", [(1, 64.0), (2, 200.0), (3, 1000.0), (4, 30.0)])
def test_theorem2_lower_bound_by_brute_force(seed, theta):
    """Eq. 2 / Theorem 2: no partition into fewer than m^_min groups keeps
    sum_i prod omega <= theta (checked by enumerating all set partitions of a small S),
    and the library's m is at least m^_min whenever its weight sum is within theta."""
    rng = np.random.default_rng(seed)
    om = [int(x) for x in rng.integers(2, 4, size=7)]
    mhat = _eq2(om, theta)

    def partitions(items):
        if not items:
            yield []
            return
        first, rest = items[0], items[1:]
        for p in partitions(rest):
            for i in range(len(p)):
                yield p[:i] + [[first] + p[i]] + p[i + 1:]
            yield [[first]] + p

    best = None
    for part in partitions(list(range(len(om)))):
        s = sum(math.prod(om[i] for i in blk) for blk in part)
        if s <= theta and (best is None or len(part) < best):
            best = len(part)
    if best is not None:
        assert mhat >= 1 and best >= mhat
    # the library on a network whose multi-function nodes have exactly these omegas
    lines = [f"pbn {len(om) + 1} {0.01.hex()}"]
    for i, w in enumerate(om):
        for j in range(w):
            lines.append(f"f {i} {(1.0 / w).hex()} 1 {len(om)} {1 + (j % 2)}")
    lines.append(f"f {len(om)} 0x1p+0 0 1")
    net = api.Net.load("\n".join(lines) + "\n")
    plan = api.Plan(net, theta=theta, max_inputs=24)
    assert plan.info.m_lower_bound == mhat
    if plan.info.sum_weights <= theta:
        assert plan.info.m_found >= mhat


def test_greedy_partition_hand_worked():
    """Algorithm 3 on omega = (3, 3, 2, 2, 2) with m = 2: sorted descending, each to
    the lightest group (empty groups weigh 0): 3 -> A, 3 -> B, 2 -> A (3 <= 3, lowest
    index), 2 -> B (6 > 3), 2 -> A (6 <= 6): weights 12 and 6, sum 18.  With
    theta = 18, Eq. 2 gives m^ = 2 (2 * sqrt(72) = 16.97 <= 18) and the partition
    is accepted at m = 2."""
    om = [3, 3, 2, 2, 2]
    lines = [f"pbn 6 {0.01.hex()}"]
    for i, w in enumerate(om):
        for j in range(w):
            lines.append(f"f {i} {(1.0 / w).hex()} 1 5 {1 + (j % 2)}")
    lines.append("f 5 0x1p+0 0 1")
    plan = api.Plan(api.Net.load("\n".join(lines) + "\n"), theta=18.0, max_inputs=24)
    assert plan.info.m_lower_bound == 2 and plan.info.m_found == 2
    assert plan.info.sum_weights == 18
    g = plan.groups()
    assert g[0] == g[2] == g[4] and g[1] == g[3] and g[0] != g[1]


def _eval_fun(f, state_bits):
    x = 0
    for b, a in enumerate(f.parents):
        x |= int(state_bits[a]) << b
    return (f.tt >> x) & 1


@pytest.mark.parametrize("mode,seed,max_inputs", [(0, 2, 8), (0, 7, 8), (1, 2, 8), (0, 2, 3), (1, 7, 2)])
def test_merged_tables_equal_member_functions(mode, seed, max_inputs):
    """Sec. 3.3: entry (c, x) of a group's merged table holds, in bit i, the output of
    member i's function selected by the mixed-radix choice c on the inputs packed in
    x, for every c and x.  A split node's function j has its own inputs and table."""
    net = synth.paper100(seed=seed, n=60)
    plan, ids = _plan(net.to_text(), mode=mode, max_inputs=max_inputs)
    D = imgdecode.decode(plan.image())
    pos = plan.layout()
    grp = plan.groups()
    inv = {int(pos[v]): v for v in range(net.n) if pos[v] != 0xFFFFFFFF}
    n_split = 0
    for g, G in enumerate(D["groups"]):
        members = sorted(np.flatnonzero(grp == g).tolist(), key=lambda v: pos[v])
        assert (pos[members[0]] & 31) == G["shift"]
        if G["l2w"] == imgdecode.SPLIT:
            n_split += 1
            (v,) = members
            assert D["multi"][imgdecode.multi_index(G, 0)]["radix"] == 1
            for j, (in_chunk, k, tab_off) in enumerate(imgdecode.subs(D, g)):
                f = net.funcs[v][j]
                assert [inv[32 * row + bit] for row, bit in imgdecode.sub_inputs(D, in_chunk, k)] == list(f.parents)
                for x in range(1 << k):
                    assert imgdecode.sub_entry(D, tab_off, x) == (f.tt >> x) & 1
            continue
        # recover input node ids from the records
        ins = [inv[32 * row + bit] for row, bit in imgdecode.inputs(D, g)]
        multi = [v for v in members if len(net.funcs[v]) >= 2]
        assert len(multi) == G["n_mul"]
        radix = [D["multi"][imgdecode.multi_index(G, m)]["radix"] for m in range(G["n_mul"])]
        ells = [len(net.funcs[v]) for v in multi]
        prod = math.prod(ells)
        assert radix == [math.prod(ells[:m]) for m in range(len(ells))]
        rng = np.random.default_rng(g)
        cs = range(prod) if prod * (1 << G["q"]) <= 4096 else rng.integers(0, prod, 8)
        xs = range(1 << G["q"]) if prod * (1 << G["q"]) <= 4096 else rng.integers(0, 1 << G["q"], 64)
        for c in cs:
            js = {v: (int(c) // radix[m]) % ells[m] for m, v in enumerate(multi)}
            for x in xs:
                bits = np.zeros(net.n, dtype=np.uint8)
                for b, a in enumerate(ins):
                    bits[a] = (int(x) >> b) & 1
                want = 0
                for i, v in enumerate(members):
                    f = net.funcs[v][js.get(v, 0)]
                    want |= _eval_fun(f, bits) << i
                assert imgdecode.entry(D, g, (int(c) << G["q"]) | int(x)) == want
    if max_inputs <= 3:
        assert n_split > 0


def test_thresholds_and_sel_slots_match_oracle(oracle_mod):
    net = synth.paper100(seed=3)
    text = net.to_text()
    plan, ids = _plan(text)
    D = imgdecode.decode(plan.image())
    grp = plan.groups()
    pos = plan.layout()
    rank = {}
    for v in range(net.n):
        if len(net.funcs[v]) >= 2:
            rank[v] = len(rank)
    for g, G in enumerate(D["groups"]):
        members = sorted(np.flatnonzero(grp == g).tolist(), key=lambda v: pos[v])
        multi = [v for v in members if len(net.funcs[v]) >= 2]
        for m, v in enumerate(multi):
            rec = D["multi"][imgdecode.multi_index(G, m)]
            P, T = oracle_mod.thresholds(text, v)
            assert imgdecode.thresholds(D, imgdecode.multi_index(G, m)) == [t for t in T if t < 2**32]
            blk = int(D["sel"][rec["u_slot"] // 4])
            assert blk == rank[v] // 4 and rec["u_slot"] % 4 == rank[v] % 4
    assert D["H"]["P"] == math.floor(net.p * 2**32)


def test_plan_specs_over_budget_are_rejected():
    """Group specs must fit the shared-memory staging budget (tables may stay in
    global memory, specs may not)."""
    net = synth.paper100(seed=2)
    red, _ = api.Net.load(net.to_text()).reduce([0, 1, 2])
    with pytest.raises(_lib.PbnError) as e:
        api.Plan(red, smem_budget=1024)
    assert e.value.status == -5
    specs = imgdecode.decode(api.Plan(red).image())["H"]["off_tables"]
    plan = api.Plan(red, smem_budget=specs)
    assert plan.info.tables_in_smem == 0 and plan.info.stage_bytes <= specs


# ---------------------------------------------------------------- estimator ----
@pytest.mark.parametrize("counts,ntraj", [
    ([100, 900, 100, 100, 900], 1), ([5000, 80000, 1200, 1300, 3500], 64),
    ([37, 1000, 3, 40, 7], 3), ([0, 500, 0, 0, 0], 1), ([10, 0, 0, 5, 5], 1),
    ([123456, 10**7, 12345, 12345, 98765], 1024), ([50, 50, 50, 50, 0], 2),
])
@pytest.mark.parametrize("r,s", [(0.01, 0.95), (1e-5, 0.95), (0.001, 0.99)])
def test_estimate_matches_oracle(oracle_mod, counts, ntraj, r, s):
    got = api.estimate(counts, ntraj, r, s, 1e-3)
    want = oracle_mod.estimate(counts, ntraj, r, s, 1e-3)
    for k in ["alpha", "beta", "pi"]:
        a, b = getattr(got, k), want[k]
        assert (math.isnan(a) and math.isnan(b)) or abs(a - b) <= 1e-12 * max(1.0, abs(b))
    assert abs(got.z - want["z"]) < 1e-12
    assert got.L == want["L"]
    if want["n_star"] is None:
        assert got.n_star == 2**64 - 1
    else:
        assert abs(got.n_star_real - want["n_star_real"]) <= 1e-12 * want["n_star_real"]
        assert got.n_star == want["n_star"]
    if want["m_star"] is None:
        assert got.m_star == 2**64 - 1
    else:
        assert got.m_star == want["m_star"]


def test_estimate_rejects_bad_arguments():
    with pytest.raises(_lib.PbnError):
        api.estimate([1, 2, 3, 4, 5], 0, 0.01, 0.95)
    with pytest.raises(_lib.PbnError):
        api.estimate([1, 2, 3, 4, 5], 1, 0.0, 0.95)
    with pytest.raises(_lib.PbnError):
        api.estimate([1, 2, 3, 4, 5], 1, 0.01, 1.0)


# ------------------------------------------------------------ compiled plans ----
@pytest.mark.parametrize("flags", [0, 1, 2, 4, 10])
@pytest.mark.parametrize("which", ["paper100", "paper100_plain", "tiny12", "p0", "one_node", "p_half",
                                   "split_small", "split_wide", "nodewise", "geometric", "wide"])
def test_generated_plan_kernels_compile(tmp_path, which, flags):
    """The source generated for a plan's own kernel compiles for sm_103a."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if which.startswith("paper100"):
        text, meta = synth.paper100(seed=2).to_text(), [0, 1, 2]
    elif which == "tiny12":
        text, meta = synth.tiny12(1).to_text(), [0, 1, 2]
    elif which == "p0":
        text, meta = synth.paper100(seed=9, n=70, p=0.0).to_text(), [0, 1]
    elif which == "p_half":
        text, meta = synth.paper100(seed=9, n=70, p=0.5).to_text(), [0, 1]
    elif which.startswith("split"):
        # split nodes: function tables as immediates (k <= 6) or looked up (k up to 10)
        kmax = 5 if which == "split_small" else 10
        text, meta = synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, kmax + 1))).to_text(), [0, 1]
    else:
        text, meta = "pbn 1 0x1p-3\nf 0 0x1p-1 1 0 2\nf 0 0x1p-1 1 0 1\n", [0]
    red, _ = api.Net.load(text).reduce(meta)
    kw = dict(max_inputs=3) if which.startswith("split") else {}
    if which == "nodewise":
        text, meta = synth.paper100(seed=2).to_text(), [0, 1, 2]
        red, _ = api.Net.load(text).reduce(meta)
        kw = dict(semantics=_lib.PBN_SEM_NODEWISE)
    if which == "wide":
        # more than 24 SEL blocks: only the wide form compiles it
        text, meta = synth.paper100(seed=21, n=400, p=1e-3).to_text(), [0, 1, 2]
        red, _ = api.Net.load(text).reduce(meta)
        with pytest.raises(_lib.PbnError):
            api.Plan(red).source(flags)
        flags |= _lib.PBN_COMPILE_WIDE
    if which == "geometric":
        text, meta = synth.paper100(seed=2, n=150).to_text(), [0, 1, 2]
        red, _ = api.Net.load(text).reduce(meta)
        kw = dict(sampler=_lib.PBN_PERT_GEOMETRIC)
    plan = api.Plan(red, mode=1 if which.endswith("plain") else 0, **kw)
    if which.startswith("split"):
        assert plan.info.n_split > 0
    (tmp_path / "k.cu").write_text(plan.source(flags))
    shutil.copy(os.path.join(ROOT, "paper_1605_00854_gb300", "csrc", "pbn_device.cuh"), tmp_path)
    proc = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c",
                           str(tmp_path / "k.cu"), "-o", str(tmp_path / "k.o")],
                          capture_output=True, text=True)
    assert proc.returncode == 0, proc.stderr[-3000:]


@pytest.mark.parametrize("which,warps,minctas,selsmem", [
    ("tiny12", 1, 0, False), ("p300", 4, 0, False), ("p300", 2, 3, False), ("split_wide", 0, 0, False),
    ("geometric", 3, 0, False), ("p0", 2, 0, False),
    ("tiny12", 1, 0, True), ("p300", 2, 0, True), ("split_wide", 2, 0, True), ("geometric", 3, 0, True)])
def test_warp_split_kernels_compile(tmp_path, which, warps, minctas, selsmem):
    """The warp-split form's generated source compiles for sm_103a, for small and
    mid-size plans, split nodes, the geometric sampler and p = 0, with the selection
    choices in registers or in shared memory; node-wise semantics are refused."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    kw = {}
    if which == "tiny12":
        text, meta = synth.tiny12(1).to_text(), [0, 1, 2]
    elif which == "p300":
        text, meta = synth.paper100(seed=31, n=300, p=1e-3).to_text(), [0, 1, 2]
    elif which == "split_wide":
        text, meta = synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11))).to_text(), [0, 1]
        kw = dict(max_inputs=3)
    elif which == "geometric":
        text, meta = synth.paper100(seed=2, n=150).to_text(), [0, 1, 2]
        kw = dict(sampler=_lib.PBN_PERT_GEOMETRIC)
    else:
        text, meta = synth.paper100(seed=9, n=70, p=0.0).to_text(), [0, 1]
    red, _ = api.Net.load(text).reduce(meta)
    plan = api.Plan(red, **kw)
    flags = _lib.PBN_COMPILE_WARP_SPLIT | _lib.PBN_COMPILE_WARPS(warps) | _lib.PBN_COMPILE_MINCTAS(minctas)
    if selsmem:
        flags |= _lib.PBN_COMPILE_WS_SELSMEM
    src = plan.source(flags)
    assert ("__constant__ uint4 SELS" in src) == (selsmem and plan.info.n_sel_blocks > 0)
    (tmp_path / "k.cu").write_text(src)
    shutil.copy(os.path.join(ROOT, "paper_1605_00854_gb300", "csrc", "pbn_device.cuh"), tmp_path)
    proc = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-Xptxas", "-O1", "-c",
                           str(tmp_path / "k.cu"), "-o", str(tmp_path / "k.o")],
                          capture_output=True, text=True)
    assert proc.returncode == 0, proc.stderr[-3000:]
    nw = api.Plan(red, semantics=_lib.PBN_SEM_NODEWISE)
    with pytest.raises(_lib.PbnError):
        nw.source(flags)


def test_large_plans_are_not_compiled():
    net = synth.scalefree2000(seed=3)
    red, _ = api.Net.load(net.to_text()).reduce([0, 1, 2, 3])
    plan = api.Plan(red)
    with pytest.raises(_lib.PbnError) as e:
        plan.source()
    assert e.value.status == -1


# ------------------------------------------------------------ array loader ----
def _funcs_of(net):
    return [[(f.c, list(f.parents), f.tt) for f in fl] for fl in net.funcs]


@pytest.mark.parametrize("which", ["tiny12", "paper100", "wide"])
def test_load_arrays_equals_text(which):
    """pbn_load_arrays builds the same network as pbn_load: equal shape and a
    byte-identical plan image (reduced and grouped)."""
    net = {"tiny12": synth.tiny12(1), "paper100": synth.paper100(seed=2),
           "wide": synth.random_pbn(5, 40, 1e-2, k_choices=tuple(range(1, 11)))}[which]
    a = api.Net.from_functions(net.n, net.p, _funcs_of(net))
    t = api.Net.load(net.to_text())
    ia, it = a.info(), t.info()
    assert (ia.n, ia.n_functions, ia.n_multi, ia.P, ia.density) == (it.n, it.n_functions, it.n_multi, it.P, it.density)
    ra, _ = a.reduce([0, 1])
    rt, _ = t.reduce([0, 1])
    assert np.array_equal(api.Plan(ra).image(), api.Plan(rt).image())
    assert np.array_equal(api.Plan(a, mode=1).image(), api.Plan(t, mode=1).image())


def test_load_arrays_rejects_bad_input():
    good = [[(0.5, [1], 0b10), (0.5, [0, 1], 0b0110)], [(1.0, [], 1)]]
    api.Net.from_functions(2, 0.01, good)
    bad = [
        (2, 0.01, [[(0.5, [1], 0b10), (0.4, [0, 1], 0b0110)], [(1.0, [], 1)]]),   # sum != 1
        (2, 0.01, [[(1.0, [1, 1], 0)], [(1.0, [], 1)]]),                           # repeated parent
        (2, 0.01, [[(1.0, [5], 0)], [(1.0, [], 1)]]),                              # parent >= n
        (2, 0.01, [[(1.0, [1], 0b100)], [(1.0, [], 1)]]),                          # table wider than 2^k
        (2, 0.01, [[(1.0, [1], 0)], []]),                                          # node without functions
        (2, 1.0, [[(1.0, [1], 0)], [(1.0, [], 1)]]),                               # p = 1
        (2, 0.01, [[(1.5, [1], 0)], [(1.0, [], 1)]]),                              # c > 1
    ]
    for n, p, funcs in bad:
        with pytest.raises(_lib.PbnError) as e:
            api.Net.from_functions(n, p, funcs)
        assert e.value.status == _lib.PBN_EINVAL
    with pytest.raises(_lib.PbnError):   # node index out of range
        api.Net.from_arrays(2, 0.01, [0, 7], [1.0, 1.0], [0, 0], [], [0, 1])


@pytest.mark.parametrize("seed", [1, 2, 5])
def test_reduce_reach_rule_matches_oracle(oracle_mod, seed):
    """PBN_REDUCE_REACH keeps exactly the oracle's reachability set; the default rule
    keeps Definition 1's."""
    net = synth.random_pbn(seed, 80, 0.01, k_choices=(1, 2, 3), sinks=0.25, protect=(0, 1, 2))
    text = net.to_text()
    meta = [0, 1, 2]
    _, ids_reach = api.Net.load(text).reduce(meta, rule=_lib.PBN_REDUCE_REACH)
    _, ids_leaf = api.Net.load(text).reduce(meta)
    assert ids_reach.tolist() == np.flatnonzero(~oracle_mod.reach_removed(text, meta)).tolist()
    assert ids_leaf.tolist() == np.flatnonzero(~oracle_mod.leaves(text, meta)).tolist()
    assert set(ids_reach.tolist()) <= set(ids_leaf.tolist())
    with pytest.raises(_lib.PbnError):
        api.Net.load(text).reduce(meta, rule=7)


# ------------------------------------------------------------ workload shapes ----
def test_apoptosis_stand_in_has_the_papers_shape(oracle_mod):
    """Sec. 4.2's apoptosis network: 96 nodes, 37.5% leaves, density 1.78.  The
    stand-in's leaves (Definition 1, by the oracle) for every meta-state of the
    workload are exactly its 36 non-core nodes."""
    import bench
    net, X, par, metas = bench.apoptosis_queries()
    assert net.n == 96 and abs(net.density() - 1.78) < 0.005
    for m in metas:
        leaf = oracle_mod.leaves(net.to_text(), m)
        assert leaf.sum() == 36 and not leaf[:60].any()
    assert len(metas) == 7 and all(a in {x for f in net.funcs[X] for x in f.parents} for a in par)



@pytest.mark.parametrize("p", [0.0, 1e-4, 0.01, 0.3, 0.75, 0.5])
def test_geometric_thresholds_match_oracle(oracle_mod, p):
    """The library's thresholds of the geometric sampler (in the plan image) equal
    the oracle's, computed by separate exact integer code."""
    text = synth.paper100(seed=2, n=70, p=p).to_text()
    plan = api.Plan(api.Net.load(text), sampler=_lib.PBN_PERT_GEOMETRIC)
    D = imgdecode.decode(plan.image())
    o = D["H"]["off_geo"] // 8
    G = [int(x) for x in np.frombuffer(plan.image().tobytes(), dtype=np.uint64)[o: o + 64]]
    assert G == oracle_mod.geo_thresholds(p)
    assert plan.info.sampler == _lib.PBN_PERT_GEOMETRIC and D["H"]["sampler"] == 1
    assert plan.info.ops_per_step < api.Plan(api.Net.load(text)).info.ops_per_step or p == 0.0


@pytest.mark.parametrize("sampler", [0, 1])
def test_bench_ops_model_equals_library(sampler):
    """The roofline's per-unit figure: bench.py's written-out model and the library's
    pbn_plan_info.ops_per_step agree for both perturbation samplers."""
    import bench
    for text, meta in ((synth.paper100(seed=2).to_text(), [0, 1, 2]), (synth.tiny12(1).to_text(), [0, 1, 2]),
                       (synth.paper100(seed=3, n=300, p=0.01).to_text(), [0, 1])):
        net = api.Net.load(text)
        red, _ = net.reduce(meta)
        plan = api.Plan(red, sampler=sampler)
        assert bench.ops_per_traj_step(plan.info, net.info().n, net.info().P) == pytest.approx(
            plan.info.ops_per_step, rel=1e-12)



def test_magic_gather_fields_are_injective_and_used():
    """Multiply gathers: every field found for a paper-scale plan maps the 2^k input
    patterns of its word to distinct indices (checked here by brute force from the
    generated source's masks and multipliers)."""
    import re
    net = synth.paper100(seed=2)
    red, _ = api.Net.load(net.to_text()).reduce([0, 1, 2])
    plan = api.Plan(red, max_inputs=12)
    src = plan.source(_lib.PBN_COMPILE_INTERLEAVED | _lib.PBN_COMPILE_MAGIC_GATHER)
    terms = re.findall(r"\(\(\(\(s\d+ & 0x([0-9a-f]{8})u\) \* 0x([0-9a-f]{8})u\) >> (\d+)\) & 0x([0-9a-f]{8})u\)", src)
    assert len(terms) >= 10
    for mask, mul, shift, fm in terms:
        mask, mul, shift, fm = int(mask, 16), int(mul, 16), int(shift), int(fm, 16)
        bits = [b for b in range(32) if (mask >> b) & 1]
        k = len(bits)
        assert fm == (1 << k) - 1
        seen = set()
        for x in range(1 << k):
            sw = sum(((x >> i) & 1) << b for i, b in enumerate(bits))
            seen.add((((sw & mask) * mul) % 2**32 >> shift) & fm)
        assert len(seen) == 1 << k


def _rows_max_share(keys):
    """Sum over rows of 32 consecutive entries of the largest number of entries that
    share one key (lanes of a warp queueing on one address)."""
    tot = 0
    for r0 in range(0, len(keys), 32):
        row = keys[r0:r0 + 32]
        tot += max(row.count(k) for k in set(row))
    return tot


def _rows_bank_load(rows_words):
    """Sum over rows of the largest number of distinct 4-byte words in one bank."""
    tot = 0
    for words in rows_words:
        per_bank = {}
        for w in set(words):
            per_bank[w % 32] = per_bank.get(w % 32, 0) + 1
        tot += max(per_bank.values()) if per_bank else 0
    return tot


@pytest.mark.parametrize("which", ["scalefree", "random"])
def test_group_order_alternates_words_and_sel_blocks_spread_banks(which):
    """Evaluation order of the image: shape classes in order; within a class the i-th
    group of every output word before any (i+1)-th; and the SEL blocks ordered so that
    the choice words a row of 32 groups reads spread over the banks at least as well as
    in ascending block order (strictly better on the scale-free network)."""
    if which == "scalefree":
        text, meta, mi = synth.scalefree2000(seed=3).to_text(), [0, 1, 2, 3], 8
    else:
        text, meta, mi = synth.random_pbn(77, 700, 1e-3, k_choices=(1, 2, 3)).to_text(), [0, 1], 6
    red, _ = api.Net.load(text).reduce(meta)
    plan = api.Plan(red, max_inputs=mi)
    D = imgdecode.decode(plan.image())
    H, G = D["H"], D["groups"]
    ng = H["n_groups"]
    gorder = [int(x) for x in D["u32"][H["off_gorder"] // 4: H["off_gorder"] // 4 + ng]]
    assert [g & 0xFFFFF for g in gorder] == list(range(ng))
    word = [g >> 20 for g in gorder]

    def shape(g):
        R = G[g]
        return (0, -R["q"]) if R["l2w"] == imgdecode.SPLIT else (1, -((R["q"] + 3) // 4), -R["n_mul"])

    classes = [shape(g) for g in range(ng)]
    assert classes == sorted(classes)
    seen, occ = {}, []
    for g in range(ng):
        k = (classes[g], word[g])
        occ.append(seen.get(k, 0))
        seen[k] = occ[-1] + 1
    for g in range(1, ng):
        if classes[g] == classes[g - 1]:
            assert (occ[g], word[g]) > (occ[g - 1], word[g - 1])
    # word-by-word order within each class, for comparison
    wb = sorted(range(ng), key=lambda g: (classes[g], word[g], g))
    assert _rows_max_share(word) <= _rows_max_share([word[g] for g in wb])

    sel = [int(x) for x in D["sel"]]
    assert len(set(sel)) == len(sel)
    rank_of = {b: i for i, b in enumerate(sorted(sel))}

    def rows_words(position):
        out = []
        for r0 in range(0, ng, 32):
            ws = []
            for g in range(r0, min(ng, r0 + 32)):
                for m in range(G[g]["n_mul"]):
                    ws.append(position(D["multi"][imgdecode.multi_index(G[g], m)]["u_slot"] // 4))
            out.append(ws)
        return out

    placed = _rows_bank_load(rows_words(lambda i: i))
    ascending = _rows_bank_load(rows_words(lambda i: rank_of[sel[i]]))
    assert placed <= ascending
    if which == "scalefree":
        assert H["n_sel"] > 32 and placed < ascending
        assert _rows_max_share(word) * 3 < _rows_max_share([word[g] for g in wb])


@pytest.mark.parametrize("lane_groups", [True, False])
def test_batch_lane_choice_on_the_host(L, lane_groups):
    """pbn_batch_create only describes the batch (device buffers are not touched until
    a launch).  With lane groups, a 62-word state whose specs leave room for 32
    trajectory slots gets 16 lanes per trajectory (32 x 16 = the CTA's 512 threads);
    by default it runs one team of the CTA's 16 warps on 32 trajectories.  A narrow
    state keeps one lane and many slots per work item either way."""
    import ctypes
    nets = [(synth.scalefree2000(seed=3).to_text(), [0, 1, 2, 3], 8, 64),
            (synth.paper100(seed=2).to_text(), [0, 1, 2], 12, 5000)]
    plans, keep = [], []
    arr = (_lib.BatchNet * len(nets))()
    fake = 1 << 20  # 16-byte aligned stand-ins for device buffers (never dereferenced here)
    for i, (text, meta, mi, T) in enumerate(nets):
        red, _ = api.Net.load(text).reduce(meta)
        plan = api.Plan(red, max_inputs=mi)
        plans.append(plan)
        ids = np.ascontiguousarray(meta, dtype=np.uint32)
        keep.append(ids)
        b = arr[i]
        b.plan, b.d_image, b.seed, b.n_traj = plan._h, fake, 1, T
        b.n_meta, b.meta_ids = len(meta), ids.ctypes.data
        b.d_state, b.d_counts, b.d_pooled = fake, fake, fake
    assert plans[0].info.state_words == 31 and plans[0].info.tables_in_smem == 0
    h = ctypes.c_void_p()
    flags = _lib.PBN_BATCH_LANE_GROUPS if lane_groups else 0
    assert L.pbn_batch_create_ex(arr, len(nets), 512, flags, ctypes.byref(h)) == 0, L.pbn_last_error_detail()
    try:
        info = _lib.BatchInfo()
        assert L.pbn_batch_info_get(h, ctypes.byref(info)) == 0
        assert info.n_nets == 2 and info.threads == 512
        assert (info.max_lanes, info.n_team) == ((16, 0) if lane_groups else (32, 1))
        # 64 trajectories in items of 32 slots, 5,000 in items of at most 512
        assert info.n_items == 2 + math.ceil(5000 / 512)
    finally:
        L.pbn_batch_free(h)
    h = ctypes.c_void_p()
    assert L.pbn_batch_create_ex(arr, len(nets), 512, 0x2, ctypes.byref(h)) != 0

    one = (_lib.BatchNet * 1)()
    one[0] = arr[1]
    h = ctypes.c_void_p()
    assert L.pbn_batch_create(one, 1, ctypes.byref(h)) == 0
    try:
        info = _lib.BatchInfo()
        assert L.pbn_batch_info_get(h, ctypes.byref(info)) == 0
        assert info.max_lanes == 1
    finally:
        L.pbn_batch_free(h)


def test_meta_state_validation_is_shared_by_single_and_batched_launches(L):
    """pbn_simulate and pbn_batch_create turn the meta nodes into state rows with the
    same checks, before any device work (fake, never dereferenced buffers): a node
    listed twice with different values, or a removed node, is refused by both; a node
    listed twice with the same value is accepted by the batch."""
    import ctypes
    text = synth.paper100(seed=2).to_text()
    red, kept = api.Net.load(text).reduce([0, 1, 2])
    plan = api.Plan(red)
    removed = int(next(v for v in range(100) if v not in set(int(x) for x in kept)))
    fake = 1 << 20

    def sim(ids, vals):
        a = _lib.SimArgs()
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        a.n_traj, a.n_steps, a.n_meta = 4, 1, len(ids)
        a.meta_ids, a.meta_vals = ids.ctypes.data, vals.ctypes.data
        a.d_state = fake
        rc = L.pbn_simulate(plan._h, ctypes.c_void_p(fake), ctypes.byref(a), None)
        return rc, L.pbn_last_error_detail().decode()

    def batch(ids, vals):
        arr = (_lib.BatchNet * 1)()
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        b = arr[0]
        b.plan, b.d_image, b.seed, b.n_traj = plan._h, fake, 1, 4
        b.n_meta, b.meta_ids, b.meta_vals = len(ids), ids.ctypes.data, vals.ctypes.data
        b.d_state, b.d_counts, b.d_pooled = fake, fake, fake
        h = ctypes.c_void_p()
        rc = L.pbn_batch_create(arr, 1, ctypes.byref(h))
        detail = L.pbn_last_error_detail().decode()
        if rc == 0:
            L.pbn_batch_free(h)
        return rc, detail

    for call in (sim, batch):
        rc, detail = call([0, 1, 0], [1, 1, 0])
        assert rc == _lib.PBN_EINVAL and "contradictory values for meta node 0" in detail, (call, detail)
        rc, detail = call([0, removed], [1, 1])
        assert rc == _lib.PBN_EINVAL and f"meta node {removed} is not a retained node" in detail, (call, detail)
    assert batch([0, 1, 0], [1, 0, 1])[0] == 0


def test_simulate_argument_checks_before_any_device_work(L):
    """pbn_simulate refuses malformed calls with PBN_EINVAL before it touches the
    device (fake, never dereferenced buffers), and a call with no trajectories is a
    no-op."""
    import ctypes
    text = synth.paper100(seed=2).to_text()
    red, _ = api.Net.load(text).reduce([0, 1, 2])
    plan = api.Plan(red)
    fake = 1 << 20
    ids = np.ascontiguousarray([0, 1, 2], dtype=np.uint32)

    def call(image=fake, plan_h=None, **kw):
        a = _lib.SimArgs()
        a.n_traj, a.n_steps, a.n_meta, a.meta_ids, a.d_state = 4, 1, 3, ids.ctypes.data, fake
        for k, v in kw.items():
            setattr(a, k, v)
        rc = L.pbn_simulate(plan._h if plan_h is None else plan_h, ctypes.c_void_p(image), ctypes.byref(a), None)
        return rc, L.pbn_last_error_detail().decode()

    assert call(n_traj=0)[0] == 0
    bad = [dict(image=fake + 8), dict(d_state=None), dict(n_traj=1 << 31), dict(n_steps=1 << 32),
           dict(traj_begin=(1 << 48) - 2), dict(step_begin=1 << 48, init=_lib.PBN_INIT_STATE),
           dict(init=7), dict(step_begin=5), dict(kernel=9), dict(n_meta=0), dict(meta_ids=None),
           dict(d_trace=fake, n_steps=1 << 31, n_traj=1 << 20)]
    for kw in bad:
        rc, detail = call(**kw)
        assert rc == _lib.PBN_EINVAL and detail.startswith("pbn_simulate"), (kw, rc, detail)
    assert L.pbn_simulate(None, ctypes.c_void_p(fake), None, None) == _lib.PBN_EINVAL


def test_synthetic_workloads_have_their_stated_shape():
    """The seeded stand-ins have the shapes the workload recipe states: the
    paper-scale network (70 % single-function nodes, in-degree 1-5 with mean 2.5,
    25 % sinks that exclude the meta nodes, p = 1e-4), the scale-free network
    (in-degree 1-6, 1-3 functions, a heavy-tailed out-degree, p = 1e-5) and the batch
    shapes (log-uniform n, trajectories and p within their ranges)."""
    from collections import Counter
    net = synth.paper100(seed=2)
    assert net.n == 100 and net.p == 1e-4
    ells = Counter(len(fl) for fl in net.funcs)
    assert set(ells) <= {1, 2, 3} and 0.55 <= ells[1] / 100 <= 0.85
    ks = [len(f.parents) for fl in net.funcs for f in fl]
    assert min(ks) >= 1 and max(ks) <= 5 and 2.1 <= np.mean(ks) <= 2.9
    parents = {a for fl in net.funcs for f in fl for a in f.parents}
    assert len([i for i in range(3, 100) if i not in parents]) >= 25  # the sinks (meta nodes excluded)
    for fl in net.funcs:
        assert abs(sum(f.c for f in fl) - 1.0) < 1e-12

    sf = synth.scalefree2000(seed=3)
    assert sf.n == 2000 and sf.p == 1e-5
    ks = [len(f.parents) for fl in sf.funcs for f in fl]
    assert min(ks) >= 1 and max(ks) <= 6 and set(len(fl) for fl in sf.funcs) == {1, 2, 3}
    out = np.array([len(c) for c in sf.children()])
    assert out.max() > 20 * out.mean()  # hubs of the power law

    shapes = synth.batch_shapes(seed=4)
    assert len(shapes) == 256
    n, t, p = (np.array(x, dtype=float) for x in zip(*shapes))
    assert n.min() >= 20 and n.max() <= 4000 and t.min() >= 1024 and t.max() <= 65536
    assert p.min() >= 1e-5 and p.max() <= 1e-2
    # log-uniform: the median sits near the geometric mean of each range
    assert abs(np.log(np.median(n)) - 0.5 * np.log(20 * 4000)) < 0.6
    assert abs(np.log(np.median(t)) - 0.5 * np.log(1024 * 65536)) < 0.6


def test_device_image_cache_is_per_device():
    """Plan.device_image uploads once per device: the same device gives the cached
    tensor, another device gets its own copy (never the first device's)."""
    torch = pytest.importorskip("torch")
    plan = api.Plan(api.Net.load(synth.tiny12(1).to_text()))
    a = plan.device_image("cpu")
    assert plan.device_image(torch.device("cpu")) is a
    assert np.array_equal(a.numpy(), plan.image())
    m = plan.device_image("meta")
    assert m is not a and m.device.type == "meta" and tuple(m.shape) == tuple(a.shape)
    assert plan.device_image("meta") is m and plan.device_image("cpu") is a


# ------------------------------------------------------------ compiled batches ----
def _fake_batch(sizes, seed=300):
    """A batch over plans of paper-scale networks of the given sizes with aligned
    host addresses standing in for device buffers (pbn_batch_create and
    pbn_batch_compile touch no device memory)."""
    import ctypes
    L = _lib.load()
    buf = np.zeros(1 << 16, dtype=np.uint8)
    base = (buf.ctypes.data + 255) & ~255
    keep = [buf]
    arr = (_lib.BatchNet * len(sizes))()
    for i, n in enumerate(sizes):
        text = synth.paper100(seed=seed + i, n=n, p=1e-3).to_text()
        red, _ = api.Net.load(text).reduce([0, 1, 2])
        plan = api.Plan(red)
        mi = np.array([0, 1, 2], dtype=np.uint32)
        keep += [plan, mi]
        b = arr[i]
        b.plan, b.d_image, b.seed, b.n_traj, b.init = plan._h, base, 11 + i, 700, 0
        b.n_meta, b.meta_ids = 3, mi.ctypes.data
        b.d_state = b.d_counts = b.d_pooled = base
    h = ctypes.c_void_p()
    _lib.check(L.pbn_batch_create(arr, len(sizes), ctypes.byref(h)), "pbn_batch_create")
    return h, keep


def test_batch_module_generates_compiles_and_links():
    """The batch module of a mixed batch (networks that compile and one that stays with
    the interpreter) compiles with NVRTC and links with the interpreter's relocatable
    work-item function; without a GPU only loading it fails."""
    import ctypes
    L = _lib.load()
    h, keep = _fake_batch([30, 90, 1100])
    try:
        rc = L.pbn_batch_compile(h, _lib.PBN_COMPILE_INTERLEAVED, None)
        detail = L.pbn_last_error_detail().decode()
        assert rc == 0 or (rc == _lib.PBN_ECUDA and "loading the batch module failed" in detail), detail
        if rc == 0:
            info = _lib.BatchInfo()
            L.pbn_batch_info_get(h, ctypes.byref(info))
            assert info.n_compiled == 2
    finally:
        L.pbn_batch_free(h)


def test_batch_module_caps_the_compiled_networks():
    """A batch of more compilable networks than a module takes (the linker crashed
    the process on a dispatcher of 136 network functions) compiles and links: the
    surplus networks, those with the least work, stay with the interpreter."""
    L = _lib.load()
    h, keep = _fake_batch([20 + (i % 7) for i in range(110)], seed=900)
    try:
        rc = L.pbn_batch_compile(h, _lib.PBN_COMPILE_INTERLEAVED, None)
        detail = L.pbn_last_error_detail().decode()
        assert rc == 0 or (rc == _lib.PBN_ECUDA and "loading the batch module failed" in detail), detail
    finally:
        L.pbn_batch_free(h)


def test_batch_compile_argument_errors():
    L = _lib.load()
    assert L.pbn_batch_compile(None, 0, None) == _lib.PBN_EINVAL
    h, keep = _fake_batch([30])
    try:
        assert L.pbn_batch_compile(h, _lib.PBN_COMPILE_MAGIC_GATHER, None) == _lib.PBN_EINVAL
        assert L.pbn_batch_compile(h, 0x100, None) == _lib.PBN_EINVAL
    finally:
        L.pbn_batch_free(h)
    h, keep = _fake_batch([1300])  # 21 perturbation words: nothing compiles
    try:
        assert L.pbn_batch_compile(h, _lib.PBN_COMPILE_INTERLEAVED, None) == _lib.PBN_EINVAL
        assert "no network" in L.pbn_last_error_detail().decode()
    finally:
        L.pbn_batch_free(h)


def test_bench_finds_captured_traffic_by_kernel_source():
    """Every `ncu-traffic:` record under profiles/ is found by the bench's lookup for
    its own source hash and trajectory count, and by nothing else."""
    import re
    import sys
    sys.path.insert(0, ROOT)
    import bench
    recs = []
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            recs += re.findall(r"ncu-traffic: source-sha256=([0-9a-f]{64}) n_traj=(\d+) dram-bytes-per-launch=(\d+)",
                               f.read())
    assert recs
    for h, t, b in recs:
        assert bench.captured_traffic(h, int(t))[0] == float(b)
        assert bench.captured_traffic(h, int(t) + 1) == (None, None)
    assert bench.captured_traffic("0" * 64, 65536) == (None, None)


def test_query_networks_have_the_paper_scale_shape():
    """The serving stream's vectorised generator follows the paper-scale recipe:
    function counts 1/2/3 at 70/15/15 %, in-degrees 1-5 with the stated pmf,
    selection probabilities summing to 1 per node, a quarter of the nodes never a
    parent (never nodes 0-3), distinct parents, and the same text on every call."""
    fun_counts, k_counts, sinks = np.zeros(4), np.zeros(6), []
    for seed in range(40):
        text = synth.query_text(100 + seed, 400, 1e-3)
        assert text == synth.query_text(100 + seed, 400, 1e-3)
        net = synth.from_text(text)
        parents = set()
        for i, fl in enumerate(net.funcs):
            fun_counts[len(fl)] += 1
            assert abs(sum(f.c for f in fl) - 1.0) < 1e-12
            for f in fl:
                k_counts[len(f.parents)] += 1
                assert len(set(f.parents)) == len(f.parents) and f.tt < (1 << (1 << len(f.parents)))
                parents |= set(f.parents)
        sinks.append(sum(1 for i in range(4, net.n) if i not in parents) / net.n)
    share = fun_counts[1:] / fun_counts.sum()
    assert abs(share[0] - 0.70) < 0.02 and abs(share[1] - 0.15) < 0.02 and abs(share[2] - 0.15) < 0.02
    pmf = k_counts[1:] / k_counts.sum()
    assert np.all(np.abs(pmf - np.array(synth.INDEG_PMF_1_5)) < 0.015)
    # 25% sinks by construction (a few more nodes are never drawn by chance)
    assert 0.25 <= np.mean(sinks) < 0.30


def test_batch_cta_sizes():
    """pbn_batch_create_cta takes CTAs of 512 or 1,024 threads and nothing else."""
    import ctypes
    L = _lib.load()
    buf = np.zeros(1 << 16, dtype=np.uint8)
    base = (buf.ctypes.data + 255) & ~255
    red, _ = api.Net.load(synth.paper100(seed=3, n=300, p=1e-3).to_text()).reduce([0, 1, 2])
    plan = api.Plan(red)
    mi = np.array([0, 1, 2], dtype=np.uint32)
    arr = (_lib.BatchNet * 1)()
    b = arr[0]
    b.plan, b.d_image, b.seed, b.n_traj, b.init = plan._h, base, 1, 5000, 0
    b.n_meta, b.meta_ids = 3, mi.ctypes.data
    b.d_state = b.d_counts = b.d_pooled = base
    for threads, ok in ((512, True), (1024, True), (256, False), (2048, False)):
        h = ctypes.c_void_p()
        rc = L.pbn_batch_create_cta(arr, 1, threads, ctypes.byref(h))
        assert (rc == 0) == ok, threads
        if ok:
            info = _lib.BatchInfo()
            L.pbn_batch_info_get(h, ctypes.byref(info))
            # at most two trajectories per thread (teams of two trajectories per lane)
            assert info.threads == threads and info.n_items >= 5000 // (2 * threads)
            L.pbn_batch_free(h)


def test_bench_finds_captured_instructions_by_kernel_source():
    """Every `ncu-inst:` record under profiles/ is found for its own source hash."""
    import re
    import sys
    sys.path.insert(0, ROOT)
    import bench
    recs = []
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            recs += re.findall(r"ncu-inst: source-sha256=([0-9a-f]{64}) warp-inst-per-warp-step=(\d+) "
                               r"thread-inst-per-traj-step=(\d+)", f.read())
    assert recs
    for h, w, t in recs:
        assert bench.captured_instructions(h) == (float(w), float(t))
    assert bench.captured_instructions("0" * 64) is None


def _batch_net_desc_type():
    """The per-network batch descriptor (pbn_netdesc in csrc/pbn_batch.cuh) as laid
    out in the device table pbn_batch_image writes."""
    import ctypes as c
    u32, u64, p = c.c_uint32, c.c_uint64, c.c_void_p
    mid = ("n_traj", "init", "stage_bytes", "image_bytes", "smem_state_off", "hmax", "tables_in_smem", "n_meta_rows",
           "n", "W", "W32", "n_sel", "P", "off_words", "off_groups", "off_multi", "off_selslot", "off_thr",
           "off_inputs", "off_selblk", "off_ret", "off_pos", "off_tables", "specs_in_smem", "nt", "off_gorder",
           "n_groups", "lg", "off_subs", "per_node", "sampler", "off_geo")
    fields = ([("image", p), ("state", p), ("counts", p), ("pooled", p), ("traj_begin", u64), ("step_begin", u64),
               ("count_from", u64), ("seed", u64)] + [(f, u32) for f in mid]
              + [("geo_full", u64), ("geo_last", u64)]
              + [(f, u32) for f in ("off_wgroups", "stage_off", "compiled", "team")]
              + [("meta_row", u32 * 16), ("meta_mask", u32 * 16), ("meta_val", u32 * 16)])
    return type("BatchNetDesc", (c.Structure,), {"_fields_": fields})


@pytest.mark.parametrize("threads", [512, 1024])
def test_batch_team_shapes_on_the_host(L, threads):
    """The batch's choice of interpreter per network, read back from its device table:
    a state of 8 rows or more runs the team interpreter with the records staged, two
    trajectories per lane when such a team fits beside them, the largest power-of-two
    number of teams (at most the CTA's warps) that fits the per-CTA shared memory,
    and the CTA's warps split evenly over the teams; a narrower state keeps lane
    groups, and PBN_BATCH_LANE_GROUPS keeps lane groups everywhere."""
    import ctypes
    cap = 224 * 1024
    nets = [(synth.scalefree2000(seed=3).to_text(), [0, 1, 2, 3], 8, 64),
            (synth.paper100(seed=3, n=300, p=1e-3).to_text(), [0, 1, 2], 8, 5000),
            (synth.paper100(seed=5, n=1000, p=1e-3).to_text(), [0, 1, 2], 8, 3000),
            (synth.paper100(seed=2).to_text(), [0, 1, 2], 12, 700)]
    plans, keep = [], []
    arr = (_lib.BatchNet * len(nets))()
    fake = 1 << 20  # 16-byte aligned stand-ins for device buffers (never dereferenced here)
    for i, (text, meta, mi, T) in enumerate(nets):
        red, _ = api.Net.load(text).reduce(meta)
        plan = api.Plan(red, max_inputs=mi)
        plans.append(plan)
        ids = np.ascontiguousarray(meta, dtype=np.uint32)
        keep.append(ids)
        b = arr[i]
        b.plan, b.d_image, b.seed, b.n_traj = plan._h, fake, 1, T
        b.n_meta, b.meta_ids = len(meta), ids.ctypes.data
        b.d_state, b.d_counts, b.d_pooled = fake, fake, fake
    _BatchNetDesc = _batch_net_desc_type()
    assert ctypes.sizeof(_BatchNetDesc) == 416
    for flags in (0, _lib.PBN_BATCH_LANE_GROUPS):
        h = ctypes.c_void_p()
        assert L.pbn_batch_create_ex(arr, len(nets), threads, flags, ctypes.byref(h)) == 0, L.pbn_last_error_detail()
        try:
            info = _lib.BatchInfo()
            assert L.pbn_batch_info_get(h, ctypes.byref(info)) == 0
            img = np.zeros(info.desc_bytes, dtype=np.uint8)
            assert L.pbn_batch_image(h, img.ctypes.data, img.size) == 0
            descs = [_BatchNetDesc.from_buffer_copy(img[416 * i: 416 * (i + 1)].tobytes()) for i in range(len(nets))]
            items = img[416 * len(nets):].view(np.uint32).reshape(-1, 4)
            assert len(items) == info.n_items
            for i, (D, plan, (_, _, _, T)) in enumerate(zip(descs, plans, nets)):
                assert D.n_traj == T and D.W32 == 2 * plan.info.state_words
                # the items of network i cover its trajectories in ranges of at most nt
                mine = items[items[:, 0] == i]
                assert mine[:, 2].sum() == T and mine[:, 2].max() <= D.nt
                assert len(mine) == math.ceil(T / D.nt)
                if flags or D.W32 < 8:
                    assert D.team == 0
                    continue
                tpl, teams = D.lg, D.nt // (32 * D.lg)
                assert tpl in (1, 2) and D.specs_in_smem == 1 and D.team * teams == threads // 32
                assert teams & (teams - 1) == 0

                def team_bytes(t):
                    return 128 * t * (2 * (D.W32 + 1) + D.n_sel + 1)
                assert D.smem_state_off == (D.stage_bytes + 127) // 128 * 128
                assert D.smem_state_off + teams * team_bytes(tpl) <= cap
                assert teams == threads // 32 or D.smem_state_off + 2 * teams * team_bytes(tpl) > cap
                if tpl == 1:  # two trajectories per lane would not fit, with or without tables
                    assert (plan.info.stage_bytes + 127) // 128 * 128 + team_bytes(2) > cap
            n_team = sum(1 for D in descs if D.team)
            assert info.n_team == n_team == (0 if flags else 3)
            if not flags:
                assert descs[0].team and descs[0].lg == 1     # scale-free: 62 rows, one trajectory per lane
                assert descs[1].lg == 2 and descs[2].lg == 2  # 300 and 1,000 nodes: two per lane
        finally:
            L.pbn_batch_free(h)
