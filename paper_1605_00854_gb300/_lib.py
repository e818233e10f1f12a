"""ctypes binding of libpbn.so (declared in include/pbn.h): argument marshalling only.

The library is loaded on first use.  If it is missing it is built in-tree; if that
fails an error is raised: there is no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

u32, u64, i32, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
vp, cp = ctypes.c_void_p, ctypes.c_char_p

PBN_OK = 0
PBN_EINVAL = -1
PBN_EPARSE = -2
PBN_ENOMEM = -3
PBN_ECUDA = -4
PBN_ETOOBIG = -5
PBN_ETIMEOUT = -6
PBN_EDEVICE = -7
PBN_REDUCE_LEAVES = 0
PBN_REDUCE_REACH = 1
PBN_PLAN_GROUPED = 0
PBN_SEM_EQ1 = 0
PBN_SEM_NODEWISE = 1
PBN_PERT_BITSLICED = 0
PBN_PERT_GEOMETRIC = 1
PBN_PLAN_PLAIN = 1
PBN_INIT_KEYED = 0
PBN_INIT_STATE = 1
PBN_COMPILE_PERT_UNROLLED = 0x1
PBN_COMPILE_INTERLEAVED = 0x2
PBN_COMPILE_PIPELINED = 0x4
PBN_COMPILE_MAGIC_GATHER = 0x8
PBN_COMPILE_WIDE = 0x10
PBN_COMPILE_WARP_SPLIT = 0x20


def PBN_COMPILE_WARPS(k: int) -> int:
    return (k & 31) << 8


def PBN_COMPILE_MINCTAS(m: int) -> int:
    return (m & 7) << 13


def PBN_COMPILE_WS_BATCH(b: int) -> int:
    return (b & 3) << 16


PBN_COMPILE_WS_O1 = 0x40000
PBN_COMPILE_WS_SELSMEM = 0x80000
PBN_BATCH_LANE_GROUPS = 0x1
PBN_BATCH_SPLIT = 0x80000000
PBN_STATIC_QUEUE_SLOTS = 16
PBN_KERNEL_AUTO = 0
PBN_KERNEL_INTERP = 1
PBN_KERNEL_COMPILED = 2
PBN_KERNEL_TEAM = 3
PBN_DEV_STAGE_TIMEOUT = 0x1
PBN_DEV_BAD_PLAN = 0x2
PBN_DEV_BAD_MODULE = 0x4


class NetInfo(ctypes.Structure):
    _fields_ = [("n", u32), ("n_retained", u32), ("n_functions", u32), ("n_multi", u32),
                ("p", f64), ("P", u64), ("density", f64)]


class NetDesc(ctypes.Structure):
    _fields_ = [("n", u32), ("n_functions", u32), ("p", f64),
                ("fun_node", ctypes.POINTER(u32)), ("fun_c", ctypes.POINTER(f64)),
                ("fun_k", ctypes.POINTER(u32)), ("parents", ctypes.POINTER(u32)),
                ("tt", ctypes.POINTER(u64))]


class GroupParams(ctypes.Structure):
    _fields_ = [("mode", u32), ("max_inputs", u32), ("max_width", u32), ("semantics", u32),
                ("theta", f64), ("smem_budget", u64), ("sampler", u32), ("reserved", u32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", u32), ("n_retained", u32), ("n_groups", u32), ("n_groups_multi", u32),
                ("state_words", u32), ("n_sel_blocks", u32), ("m_lower_bound", u32),
                ("m_found", u32), ("sum_weights", u64), ("table_bytes", u64),
                ("image_bytes", u64), ("stage_bytes", u64), ("tables_in_smem", u32),
                ("total_inputs", u32), ("n_multi", u32), ("total_thresholds", u32),
                ("n_split", u32), ("semantics", u32), ("sampler", u32), ("reserved", u32),
                ("ops_per_step", f64)]


class BatchNet(ctypes.Structure):
    _fields_ = [("plan", vp), ("d_image", vp), ("seed", u64), ("traj_begin", u64), ("n_traj", u64),
                ("step_begin", u64), ("count_from", u64), ("init", u32), ("n_meta", u32),
                ("meta_ids", vp), ("meta_vals", vp), ("d_state", vp), ("d_counts", vp),
                ("d_pooled", vp)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_nets", u32), ("n_items", u32), ("threads", u32), ("max_lanes", u32),
                ("desc_bytes", u64), ("smem_bytes", u64), ("est_ops_per_step", f64),
                ("n_compiled", u32), ("n_items_compiled", u32), ("n_team", u32), ("reserved", u32)]


class SimArgs(ctypes.Structure):
    _fields_ = [("seed", u64), ("traj_begin", u64), ("n_traj", u64), ("step_begin", u64),
                ("n_steps", u64), ("count_from", u64), ("init", u32), ("n_meta", u32),
                ("meta_ids", vp), ("meta_vals", vp), ("d_state", vp), ("d_counts", vp),
                ("d_pooled", vp), ("d_status", vp), ("d_trace", vp),
                ("lanes_per_traj", u32), ("trajs_per_block", u32), ("kernel", u32), ("trace_stride", u32),
                ("team_warps", u32), ("team_trajs_per_lane", u32)]


class EstimateOut(ctypes.Structure):
    _fields_ = [("alpha", f64), ("beta", f64), ("pi", f64), ("var", f64), ("z", f64),
                ("n_star_real", f64), ("L", u64), ("m_star", u64), ("n_star", u64),
                ("defined", i32), ("done", i32)]


#: every symbol include/pbn.h declares, with (restype, argtypes)
SIGNATURES = {
    "pbn_load": (i32, [cp, ctypes.c_size_t, ctypes.POINTER(vp)]),
    "pbn_load_arrays": (i32, [ctypes.POINTER(NetDesc), ctypes.POINTER(vp)]),
    "pbn_plan_compiled_attrs": (i32, [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]),
    "pbn_net_info_get": (i32, [vp, ctypes.POINTER(NetInfo)]),
    "pbn_reduce": (i32, [vp, vp, u32, ctypes.POINTER(vp), vp, ctypes.POINTER(u32)]),
    "pbn_reduce_rule": (i32, [vp, vp, u32, u32, ctypes.POINTER(vp), vp, ctypes.POINTER(u32)]),
    "pbn_group_params_default": (None, [ctypes.POINTER(GroupParams)]),
    "pbn_group": (i32, [vp, ctypes.POINTER(GroupParams), ctypes.POINTER(vp)]),
    "pbn_plan_info_get": (i32, [vp, ctypes.POINTER(PlanInfo)]),
    "pbn_plan_image": (i32, [vp, vp, ctypes.c_size_t]),
    "pbn_plan_layout": (i32, [vp, vp]),
    "pbn_plan_groups": (i32, [vp, vp]),
    "pbn_simulate": (i32, [vp, vp, ctypes.POINTER(SimArgs), vp]),
    "pbn_plan_compile": (i32, [vp, u32, ctypes.POINTER(f64)]),
    "pbn_batch_create": (i32, [ctypes.POINTER(BatchNet), u32, ctypes.POINTER(vp)]),
    "pbn_batch_info_get": (i32, [vp, ctypes.POINTER(BatchInfo)]),
    "pbn_batch_image": (i32, [vp, vp, ctypes.c_size_t]),
    "pbn_batch_compile": (i32, [vp, u32, ctypes.POINTER(f64)]),
    "pbn_batch_create_cta": (i32, [ctypes.POINTER(BatchNet), u32, u32, ctypes.POINTER(vp)]),
    "pbn_batch_create_ex": (i32, [ctypes.POINTER(BatchNet), u32, u32, u32, ctypes.POINTER(vp)]),
    "pbn_batch_run": (i32, [vp, vp, vp, u64, u64, u32, vp, vp]),
    "pbn_batch_free": (None, [vp]),
    "pbn_batch_run_static": (i32, [vp, vp, u32, u64, u64, u32, vp, vp]),
    "pbn_plan_source": (i32, [vp, u32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "pbn_estimate": (i32, [vp, u64, u64, f64, f64, f64, ctypes.POINTER(EstimateOut)]),
    "pbn_strerror": (cp, [i32]),
    "pbn_last_error_detail": (cp, []),
    "pbn_net_free": (None, [vp]),
    "pbn_plan_free": (None, [vp]),
    "pbn_version": (cp, []),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpbn.so (building it in-tree if absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libpbn.so not built at {path}")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


class PbnError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = load()
        detail = L.pbn_last_error_detail().decode()
        super().__init__(f"{where}: {L.pbn_strerror(status).decode()} ({status}): {detail}")
        self.status = status


def check(status: int, where: str):
    if status != PBN_OK:
        raise PbnError(status, where)
