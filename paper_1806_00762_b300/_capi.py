"""ctypes mirror of include/seraph.h (structures, prototypes, error codes).

Argument marshalling only: every step of the graph method runs inside
libseraph.so.  Loading fails loudly when the library is missing -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libseraph.so")

SERAPH_OK = 0
SERAPH_EINVAL = -1
SERAPH_ENOMEM = -2
SERAPH_EBUDGET = -3
SERAPH_ECUDA = -4
SERAPH_ETIMEOUT = -5
SERAPH_EOVERFLOW = -6
SERAPH_ENOTCONV = -7
ERROR_NAMES = {
    SERAPH_EINVAL: "EINVAL", SERAPH_ENOMEM: "ENOMEM", SERAPH_EBUDGET: "EBUDGET",
    SERAPH_ECUDA: "ECUDA", SERAPH_ETIMEOUT: "ETIMEOUT", SERAPH_EOVERFLOW: "EOVERFLOW",
    SERAPH_ENOTCONV: "ENOTCONV",
}

SSSP, BFS, CC, PAGERANK = 0, 1, 2, 3
ALGOS = {"sssp": SSSP, "bfs": BFS, "cc": CC, "pagerank": PAGERANK, "pr": PAGERANK}
MEM_HOST, MEM_DEVICE = 0, 1
PVU_OFF, PVU_STRONG, PVU_WEAK = 0, 1, 2
PVUS = {"off": PVU_OFF, "strong": PVU_STRONG, "weak": PVU_WEAK}
SCHED_FIXED, SCHED_LEARNED = 0, 1
ORDER_CYCLIC, ORDER_ZIGZAG = 0, 1
ORDERS = {"cyclic": ORDER_CYCLIC, "zigzag": ORDER_ZIGZAG}
SYMMETRIZE = 1
REORDER = 2
COMPRESS = 4
OUT_EDGES = 8
COLUMNS = {"auto": 0, "plain": 1, "packed": 2, "hybrid": 3}
NOALLOC_MAX_VERTICES = 1 << 20
INF = 0xFFFFFFFF

u8, u32, i32, u64, dbl, vp = (ctypes.c_uint8, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64,
                              ctypes.c_double, ctypes.c_void_p)


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", u64), ("m_raw", u64), ("m", u64), ("struct_bytes", u64),
                ("weight_bytes", u64), ("max_page_struct_bytes", u64),
                ("max_page_weight_bytes", u64), ("num_pages", u32), ("weighted", u32),
                ("symmetrized", u32), ("max_in_degree", u32), ("weight_width", u32),
                ("reordered", u32), ("packed", u32), ("reserved", u32), ("packed_bytes", u64),
                ("packed_data_bytes", u64), ("max_page_packed_bytes", u64),
                ("out_edge_bytes", u64)]


class Params(ctypes.Structure):
    _fields_ = [("algo", i32), ("source", u32), ("budget_bytes", u64), ("window", u32),
                ("passes", u32), ("pvu", i32), ("verify", u32), ("fsm_next", u8 * 12),
                ("fsm_skip_mask", u8), ("kahan", u8), ("pr_normalize", u8), ("pad0", u8), ("max_sweeps", u32),
                ("damping", dbl), ("tol", dbl), ("pr_fail_eps", dbl),
                ("pr_pvu_off_below", dbl), ("thread_max_deg", u32), ("warp_max_deg", u32),
                ("sched", i32), ("timeout_ms", u32), ("profile", u32), ("order", u32),
                ("max_passes", u32), ("slots", u32), ("group4_max_deg", u32),
                ("group8_max_deg", u32),
                ("sched_model", vp), ("stream", vp), ("trace", vp), ("columns", u32),
                ("pad1", u32), ("l2_hot_bytes", u64), ("pr_omega", dbl), ("push", u32),
                ("pad2", u32), ("push_below", u64), ("count_clean", u32), ("stream_packed", u32)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", u32), ("steps", u32), ("passes_run", u32), ("passes_skipped", u32),
                ("chunks", u32), ("resident", u32), ("converged", u32), ("verify_sweeps", u32),
                ("bytes_streamed", u64), ("edges_relaxed", u64), ("vertices_attempted", u64),
                ("vertices_skipped", u64), ("changes", u64), ("time_ms", dbl),
                ("copy_ms", dbl), ("compute_ms", dbl), ("wall_ms", dbl), ("residual", dbl),
                ("relax_ms", dbl), ("relax_launches", u64), ("kernel_launches", u64),
                ("packed_edges", u64), ("code_bytes", u64), ("push_edges", u64),
                ("push_rounds", u32), ("push_sweep", u32), ("clean_pages", u64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Trace(ctypes.Structure):
    _fields_ = [("capacity", u64), ("count", u64), ("features", vp), ("gains", vp),
                ("vertices", vp)]


SCHED_FEATURES, SCHED_OUTPUTS, SCHED_PARAMS = 16, 17, 6353
MAP_AUTO, MAP_THREAD, MAP_WARP, MAP_CTA = 0, 1, 2, 3
MAPPINGS = {"auto": MAP_AUTO, "thread": MAP_THREAD, "warp": MAP_WARP, "cta": MAP_CTA}


class Query(ctypes.Structure):
    _fields_ = [("graph", u32), ("algo", i32), ("source", u32), ("reserved", u32), ("out", vp)]


class BatchParams(ctypes.Structure):
    _fields_ = [("mapping", i32), ("tile", u32), ("use_graph", u32), ("replays", u32),
                ("timeout_ms", u32), ("delta", u32), ("stream", vp), ("bfs_pull_div", u32),
                ("group", u32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("time_ms", dbl), ("tune_ms", dbl), ("edges", u64), ("tasks", u64),
                ("rounds_max", u32), ("graph_captured", u32), ("mapping", u32 * 16),
                ("tile", u32 * 16)]

# name -> (restype, argtypes); every symbol include/seraph.h declares
PROTOTYPES = {
    "seraph_graph_from_edges": (ctypes.c_int, [u64, u64, vp, vp, vp, ctypes.c_int, u32, u32, vp,
                                               ctypes.POINTER(vp)]),
    "seraph_graph_from_csr": (ctypes.c_int, [u64, vp, vp, vp, ctypes.c_int, u32, u32, vp,
                                             ctypes.POINTER(vp)]),
    "seraph_graph_get_info": (ctypes.c_int, [vp, ctypes.POINTER(GraphInfo)]),
    "seraph_graph_page_bounds": (ctypes.c_int, [vp, vp]),
    "seraph_graph_export_csc": (ctypes.c_int, [vp, vp, vp, vp, vp]),
    "seraph_graph_export_perm": (ctypes.c_int, [vp, vp]),
    "seraph_graph_export_packed": (ctypes.c_int, [vp, vp, vp]),
    "seraph_graph_export_out_edges": (ctypes.c_int, [vp, vp, vp, vp]),
    "seraph_graph_release_buffers": (ctypes.c_int, [vp]),
    "seraph_graph_free": (None, [vp]),
    "seraph_params_default": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int]),
    "seraph_run": (ctypes.c_int, [vp, ctypes.POINTER(Params), vp, ctypes.c_int,
                                  ctypes.POINTER(Stats)]),
    "seraph_pull_fixpoint_noalloc": (ctypes.c_int, [ctypes.c_int, u64, vp, vp, vp, u32, vp, vp,
                                                    vp]),
    "seraph_gather_probe": (ctypes.c_int, [u64, u64, u64, dbl, u32, vp,
                                           ctypes.POINTER(dbl)]),
    "seraph_sched_create": (ctypes.c_int, [u64, ctypes.c_int, ctypes.POINTER(vp)]),
    "seraph_sched_get_params": (ctypes.c_int, [vp, vp]),
    "seraph_sched_set_params": (ctypes.c_int, [vp, vp]),
    "seraph_sched_loss_grad": (ctypes.c_int, [vp, vp, vp, vp, u64, ctypes.c_int, vp, vp]),
    "seraph_sched_train": (ctypes.c_int, [vp, vp, vp, vp, u64, ctypes.c_int, u32, u32,
                                          ctypes.c_float, u64, vp]),
    "seraph_sched_infer": (ctypes.c_int, [vp, vp, u64, ctypes.c_int, vp, vp]),
    "seraph_sched_targets": (ctypes.c_int, [ctypes.POINTER(Trace), ctypes.c_float, vp, vp]),
    "seraph_sched_free": (None, [vp]),
    "seraph_bgraph_from_edges": (ctypes.c_int, [u64, u64, vp, vp, vp, ctypes.c_int, vp,
                                                ctypes.POINTER(vp)]),
    "seraph_bgraph_free": (None, [vp]),
    "seraph_batch_params_default": (ctypes.c_int, [ctypes.POINTER(BatchParams)]),
    "seraph_batch_run": (ctypes.c_int, [vp, u32, vp, u32, ctypes.c_int,
                                        ctypes.POINTER(BatchParams), ctypes.POINTER(BatchStats)]),
    "seraph_batch_plan_create": (ctypes.c_int, [vp, u32, vp, u32, ctypes.POINTER(BatchParams),
                                                ctypes.POINTER(vp)]),
    "seraph_batch_plan_run": (ctypes.c_int, [vp, vp, ctypes.POINTER(BatchStats)]),
    "seraph_batch_plan_free": (None, [vp]),
    "seraph_debug_fail_pinned_alloc": (ctypes.c_int, [u32]),
    "seraph_debug_pinned_bytes": (u64, []),
    "seraph_debug_l2_setaside": (ctypes.c_int, [ctypes.POINTER(u64)]),
    "seraph_last_error": (ctypes.c_char_p, []),
    "seraph_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libseraph.so (building it first if it is absent or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build
        _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libseraph.so missing at {LIB_PATH}; the CUDA path is required")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SeraphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != SERAPH_OK:
        raise SeraphError(rc, lib().seraph_last_error().decode())
