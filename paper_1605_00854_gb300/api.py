"""Python API over the C ABI: networks, plans, simulation and estimation.

Device memory and streams come from PyTorch; every step of the simulation runs in
the library's CUDA kernels.  Buffers holding 64-bit words are torch.int64 tensors
(bit patterns; view them as uint64 on the host).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import check


def _ptr(t):
    """Raw data pointer of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


class Net:
    """A PBN G(X, F) with perturbation rate p (opaque pbn_net handle)."""

    def __init__(self, handle, text: str | None = None):
        self._h = handle
        self.text = text

    @classmethod
    def load(cls, text: str) -> "Net":
        L = _lib.load()
        h = ctypes.c_void_p()
        b = text.encode()
        check(L.pbn_load(b, len(b), ctypes.byref(h)), "pbn_load")
        return cls(h, text)

    @classmethod
    def from_arrays(cls, n: int, p: float, fun_node, fun_c, fun_k, parents, tt) -> "Net":
        """pbn_load_arrays: functions as flat arrays (node, c, k per function; parent
        lists and 64-bit truth-table words concatenated function by function)."""
        L = _lib.load()
        arrs = dict(fun_node=np.ascontiguousarray(fun_node, dtype=np.uint32),
                    fun_c=np.ascontiguousarray(fun_c, dtype=np.float64),
                    fun_k=np.ascontiguousarray(fun_k, dtype=np.uint32),
                    parents=np.ascontiguousarray(parents, dtype=np.uint32),
                    tt=np.ascontiguousarray(tt, dtype=np.uint64))
        nf = len(arrs["fun_node"])
        if not (len(arrs["fun_c"]) == len(arrs["fun_k"]) == nf):
            raise ValueError("fun_node, fun_c and fun_k differ in length")
        if len(arrs["parents"]) != int(arrs["fun_k"].sum()):
            raise ValueError("parents must hold sum(fun_k) entries")
        if len(arrs["tt"]) != sum((1 << int(k)) + 63 >> 6 for k in arrs["fun_k"]):
            raise ValueError("tt must hold sum(ceil(2^k / 64)) words")
        d = _lib.NetDesc(n=n, n_functions=nf, p=p)
        ctype = {np.uint32: ctypes.c_uint32, np.float64: ctypes.c_double, np.uint64: ctypes.c_uint64}
        for name, a in arrs.items():  # arrs keeps the buffers alive during the call
            setattr(d, name, a.ctypes.data_as(ctypes.POINTER(ctype[a.dtype.type])))
        h = ctypes.c_void_p()
        check(L.pbn_load_arrays(ctypes.byref(d), ctypes.byref(h)), "pbn_load_arrays")
        return cls(h)

    @classmethod
    def from_functions(cls, n: int, p: float, funcs) -> "Net":
        """funcs[i] = [(c, parents, truth table as int), ...] for node i, in order j."""
        fun_node, fun_c, fun_k, parents, tt = [], [], [], [], []
        for i, fl in enumerate(funcs):
            for c, par, table in fl:
                k = len(par)
                fun_node.append(i)
                fun_c.append(c)
                fun_k.append(k)
                parents.extend(par)
                for w in range(((1 << k) + 63) >> 6):
                    tt.append((int(table) >> (64 * w)) & 0xFFFFFFFFFFFFFFFF)
        return cls.from_arrays(n, p, fun_node, fun_c, fun_k, parents, tt)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.load().pbn_net_free(self._h)
            self._h = None

    def info(self) -> _lib.NetInfo:
        out = _lib.NetInfo()
        check(_lib.load().pbn_net_info_get(self._h, ctypes.byref(out)), "pbn_net_info_get")
        return out

    def reduce(self, interest, rule: int = _lib.PBN_REDUCE_LEAVES):
        """Leaf-node reduction (Definition 1) for the given nodes of interest, or with
        rule=PBN_REDUCE_REACH the removal of every node that reaches none of them.
        Returns (reduced Net, retained original ids)."""
        L = _lib.load()
        n = self.info().n
        it = np.ascontiguousarray(interest, dtype=np.uint32)
        ids = np.zeros(n, dtype=np.uint32)
        cnt = ctypes.c_uint32()
        h = ctypes.c_void_p()
        if rule == _lib.PBN_REDUCE_LEAVES:
            check(L.pbn_reduce(self._h, _ptr(it), len(it), ctypes.byref(h), _ptr(ids),
                               ctypes.byref(cnt)), "pbn_reduce")
        else:
            check(L.pbn_reduce_rule(self._h, _ptr(it), len(it), rule, ctypes.byref(h), _ptr(ids),
                                    ctypes.byref(cnt)), "pbn_reduce_rule")
        return Net(h, self.text), ids[: cnt.value].copy()


def group_params(mode: int = _lib.PBN_PLAN_GROUPED, max_inputs: int = 8, max_width: int = 32,
                 theta: float = 65536.0, smem_budget: int = 0,
                 semantics: int = _lib.PBN_SEM_EQ1, sampler: int = _lib.PBN_PERT_BITSLICED) -> _lib.GroupParams:
    p = _lib.GroupParams()
    _lib.load().pbn_group_params_default(ctypes.byref(p))
    p.mode, p.max_inputs, p.max_width, p.theta = mode, max_inputs, max_width, theta
    p.semantics = semantics
    p.sampler = sampler
    if smem_budget:
        p.smem_budget = smem_budget
    return p


class Plan:
    """Simulation plan (Algorithm 5, Preparation) and its device image."""

    def __init__(self, net: Net, params: _lib.GroupParams | None = None, **kw):
        L = _lib.load()
        prm = params if params is not None else group_params(**kw)
        h = ctypes.c_void_p()
        check(L.pbn_group(net._h, ctypes.byref(prm), ctypes.byref(h)), "pbn_group")
        self._h = h
        self.net = net
        self.info = _lib.PlanInfo()
        check(L.pbn_plan_info_get(self._h, ctypes.byref(self.info)), "pbn_plan_info_get")
        self._dev = {}  # device -> uploaded image

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.load().pbn_plan_free(self._h)
            self._h = None

    def image(self) -> np.ndarray:
        buf = np.zeros(self.info.image_bytes, dtype=np.uint8)
        check(_lib.load().pbn_plan_image(self._h, _ptr(buf), buf.size), "pbn_plan_image")
        return buf

    def layout(self) -> np.ndarray:
        pos = np.zeros(self.info.n, dtype=np.uint32)
        check(_lib.load().pbn_plan_layout(self._h, _ptr(pos)), "pbn_plan_layout")
        return pos

    def groups(self) -> np.ndarray:
        g = np.zeros(self.info.n, dtype=np.uint32)
        check(_lib.load().pbn_plan_groups(self._h, _ptr(g)), "pbn_plan_groups")
        return g

    def compile(self, flags: int = 0) -> float:
        """Compile the plan into its own kernel (pbn_plan_compile); returns host ms."""
        ms = ctypes.c_double()
        check(_lib.load().pbn_plan_compile(self._h, flags, ctypes.byref(ms)), "pbn_plan_compile")
        return ms.value

    def compiled_attrs(self) -> dict:
        """Registers, spill bytes and flags of the compiled kernel (pbn_plan_compiled_attrs)."""
        r, l, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(_lib.load().pbn_plan_compiled_attrs(self._h, ctypes.byref(r), ctypes.byref(l), ctypes.byref(f)),
              "pbn_plan_compiled_attrs")
        return {"regs": r.value, "local_bytes": l.value, "flags": f.value}

    def source(self, flags: int = 0) -> str:
        """CUDA source of the plan's own kernel (pbn_plan_source)."""
        L = _lib.load()
        n = ctypes.c_size_t()
        check(L.pbn_plan_source(self._h, flags, None, 0, ctypes.byref(n)), "pbn_plan_source")
        buf = ctypes.create_string_buffer(n.value + 1)
        check(L.pbn_plan_source(self._h, flags, buf, n.value + 1, ctypes.byref(n)), "pbn_plan_source")
        return buf.value.decode()

    def device_image(self, device="cuda"):
        """The image uploaded to `device` (once per device, then cached)."""
        import torch
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        img = self._dev.get(dev)
        if img is None:
            img = torch.from_numpy(self.image()).to(dev)
            self._dev[dev] = img
        return img

    def unpack(self, words: np.ndarray) -> np.ndarray:
        """Grouped state words [state_words, T] (uint64) -> bits [T, n] in original node
        order, with 0 in the columns of removed nodes."""
        words = np.asarray(words).view(np.uint64)
        pos = self.layout()
        T = words.shape[-1]
        out = np.zeros((T, self.info.n), dtype=np.uint8)
        keep = pos != np.uint32(0xFFFFFFFF)
        rows = (pos[keep] >> 5).astype(np.int64)
        bits = (pos[keep] & 31).astype(np.uint64)
        w64 = words[rows >> 1, :]  # [k, T]
        sh = (bits + np.uint64(32) * (rows & 1).astype(np.uint64))[:, None]
        out[:, keep] = ((w64 >> sh) & np.uint64(1)).astype(np.uint8).T
        return out


@dataclass
class SimBuffers:
    state: "object"       # torch.int64 [state_words, T]
    counts: "object"      # torch.int64 [5, T]
    pooled: "object"      # torch.int64 [5]
    status: "object"      # torch.int32 [1]


def alloc_buffers(plan: Plan, n_traj: int, device="cuda") -> SimBuffers:
    import torch
    return SimBuffers(
        state=torch.zeros((plan.info.state_words, n_traj), dtype=torch.int64, device=device),
        counts=torch.zeros((5, n_traj), dtype=torch.int64, device=device),
        pooled=torch.zeros(5, dtype=torch.int64, device=device),
        status=torch.zeros(1, dtype=torch.int32, device=device))


def simulate(plan: Plan, bufs: SimBuffers, *, seed: int, n_steps: int, meta_ids, meta_vals=None,
             traj_begin: int = 0, step_begin: int = 0, count_from: int = 0, init: int | None = None,
             trace=None, lanes_per_traj: int = 0, trajs_per_block: int = 0, stream=None,
             d_image=None, n_traj: int | None = None, kernel: int = _lib.PBN_KERNEL_AUTO,
             trace_stride: int = 1, team_warps: int = 0, team_trajs_per_lane: int = 0):
    """Enqueue pbn_simulate on `stream` (default: torch's current stream)."""
    import torch
    L = _lib.load()
    T = bufs.state.shape[1] if n_traj is None else n_traj
    a = _lib.SimArgs()
    a.seed, a.traj_begin, a.n_traj = seed, traj_begin, T
    a.step_begin, a.n_steps, a.count_from = step_begin, n_steps, count_from
    if init is None:
        init = _lib.PBN_INIT_KEYED if step_begin == 0 else _lib.PBN_INIT_STATE
    a.init = init
    mi = np.ascontiguousarray(meta_ids, dtype=np.uint32)
    mv = None if meta_vals is None else np.ascontiguousarray(meta_vals, dtype=np.uint8)
    a.n_meta = len(mi)
    a.meta_ids = mi.ctypes.data
    a.meta_vals = None if mv is None else mv.ctypes.data
    a.d_state = bufs.state.data_ptr()
    a.d_counts = None if bufs.counts is None else bufs.counts.data_ptr()
    a.d_pooled = None if bufs.pooled is None else bufs.pooled.data_ptr()
    a.d_status = None if bufs.status is None else bufs.status.data_ptr()
    a.d_trace = None if trace is None else trace.data_ptr()
    a.lanes_per_traj, a.trajs_per_block = lanes_per_traj, trajs_per_block
    a.kernel = kernel
    a.trace_stride = trace_stride
    a.team_warps = team_warps
    a.team_trajs_per_lane = team_trajs_per_lane
    img = plan.device_image(bufs.state.device) if d_image is None else d_image
    st = torch.cuda.current_stream(bufs.state.device) if stream is None else stream
    check(L.pbn_simulate(plan._h, ctypes.c_void_p(img.data_ptr()), ctypes.byref(a),
                         ctypes.c_void_p(st.cuda_stream)), "pbn_simulate")


def estimate(counts5, n_traj: int, r: float, s: float, eps: float = 1e-3,
             burn_in_used: int = 0) -> _lib.EstimateOut:
    """Two-state Markov chain estimate (pbn_estimate) from pooled counts."""
    c = np.ascontiguousarray([int(x) for x in counts5], dtype=np.uint64)
    out = _lib.EstimateOut()
    check(_lib.load().pbn_estimate(_ptr(c), n_traj, burn_in_used, r, s, eps, ctypes.byref(out)),
          "pbn_estimate")
    return out


class Batch:
    """Many networks simulated by one persistent launch per step chunk, fed by a
    device work queue (pbn_batch_create / pbn_batch_run).

    `entries` is a list of dicts with keys plan, bufs (SimBuffers), seed, meta_ids and
    optionally meta_vals, traj_begin, step_begin, count_from, init.  With
    compile_flags (pbn_batch_compile) the networks whose plans compile run their own
    generated code in the same persistent launch, the others the interpreter (wide
    states as teams of warps on 32 trajectories, unless lane_groups)."""

    def __init__(self, entries, device="cuda", compile_flags: int | None = None, threads: int = 512,
                 lane_groups: bool = False):
        import torch
        L = _lib.load()
        self.entries = entries
        self._keep = []
        arr = (_lib.BatchNet * len(entries))()
        for i, e in enumerate(entries):
            plan, bufs = e["plan"], e["bufs"]
            mi = np.ascontiguousarray(e["meta_ids"], dtype=np.uint32)
            mv = None if e.get("meta_vals") is None else np.ascontiguousarray(e["meta_vals"], dtype=np.uint8)
            self._keep += [mi, mv]
            b = arr[i]
            b.plan = plan._h
            b.d_image = plan.device_image(device).data_ptr()
            b.seed = e["seed"]
            b.traj_begin = e.get("traj_begin", 0)
            b.n_traj = bufs.state.shape[1]
            b.step_begin = e.get("step_begin", 0)
            b.count_from = e.get("count_from", 0)
            b.init = e.get("init", _lib.PBN_INIT_KEYED if b.step_begin == 0 else _lib.PBN_INIT_STATE)
            b.n_meta = len(mi)
            b.meta_ids = mi.ctypes.data
            b.meta_vals = None if mv is None else mv.ctypes.data
            b.d_state = bufs.state.data_ptr()
            b.d_counts = None if bufs.counts is None else bufs.counts.data_ptr()
            b.d_pooled = None if bufs.pooled is None else bufs.pooled.data_ptr()
        h = ctypes.c_void_p()
        flags = _lib.PBN_BATCH_LANE_GROUPS if lane_groups else 0
        check(L.pbn_batch_create_ex(arr, len(entries), threads, flags, ctypes.byref(h)), "pbn_batch_create_ex")
        self._h = h
        self.compile_ms = 0.0
        if compile_flags is not None:
            ms = ctypes.c_double()
            check(L.pbn_batch_compile(self._h, compile_flags, ctypes.byref(ms)), "pbn_batch_compile")
            self.compile_ms = ms.value
        self.info = _lib.BatchInfo()
        check(L.pbn_batch_info_get(self._h, ctypes.byref(self.info)), "pbn_batch_info_get")
        host = np.zeros(self.info.desc_bytes, dtype=np.uint8)
        check(L.pbn_batch_image(self._h, _ptr(host), host.size), "pbn_batch_image")
        self.desc = torch.from_numpy(host).to(device)
        self.queue = torch.zeros(2, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.steps_done = 0

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.load().pbn_batch_free(self._h)
            self._h = None

    def run(self, n_steps: int, step_offset: int | None = None, ctas_per_sm: int = 0, stream=None):
        """One persistent launch advancing every network by n_steps steps."""
        import torch
        st = torch.cuda.current_stream(self.desc.device) if stream is None else stream
        off = self.steps_done if step_offset is None else step_offset
        check(_lib.load().pbn_batch_run(self._h, ctypes.c_void_p(self.desc.data_ptr()),
                                        ctypes.c_void_p(self.queue.data_ptr()), off, n_steps,
                                        ctas_per_sm, ctypes.c_void_p(self.status.data_ptr()),
                                        ctypes.c_void_p(st.cuda_stream)), "pbn_batch_run")
        self.steps_done = off + n_steps

    def run_static(self, n_steps: int, slot: int = 0, step_offset: int | None = None,
                   ctas_per_sm: int = 0, stream=None):
        """Like run(), with the work-queue scratch taken from the library's static
        device array (pbn_batch_run_static): allocates nothing."""
        import torch
        st = torch.cuda.current_stream(self.desc.device) if stream is None else stream
        off = self.steps_done if step_offset is None else step_offset
        check(_lib.load().pbn_batch_run_static(self._h, ctypes.c_void_p(self.desc.data_ptr()), slot, off, n_steps,
                                               ctas_per_sm, ctypes.c_void_p(self.status.data_ptr()),
                                               ctypes.c_void_p(st.cuda_stream)), "pbn_batch_run_static")
        self.steps_done = off + n_steps

    def capture(self, chunks, step_offset: int = 0):
        """Capture the launches of `chunks` (list of step counts) starting at
        step_offset in a CUDA graph; returns the torch.cuda.CUDAGraph to replay."""
        import torch
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.desc.device)
        s.wait_stream(torch.cuda.current_stream(self.desc.device))
        with torch.cuda.stream(s):
            # launch configuration queries happen outside the capture
            pass
        off = step_offset
        with torch.cuda.graph(g, stream=s):
            for c in chunks:
                self.run(c, step_offset=off, stream=s)
                off += c
        torch.cuda.current_stream(self.desc.device).wait_stream(s)
        self.steps_done = step_offset
        return g
