"""Seraph on B300: streamed-graph pipelined subgraph iteration with predictive
vertex updating (arXiv 1806.00762), as a C-ABI library with a thin Python
binding.

    g = Graph.from_edges(n, src, dst, w, num_pages=64)     # GPU partitioner
    values, stats = run(g, "sssp", source=0, budget_bytes=2 << 30, window=4)

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); torch is
used only for device memory and streams.  All graph work runs in
libseraph.so (see include/seraph.h).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C
from ._capi import SeraphError, INF

__all__ = ["Graph", "run", "default_params", "SeraphError", "INF", "version", "SchedModel",
           "TraceBuffer", "BGraph", "batch_run"]


def version() -> str:
    return C.lib().seraph_version().decode()


def _ptr_mem(a):
    """(pointer, mem kind, keep-alive) for a numpy array or torch tensor."""
    if a is None:
        return None, C.MEM_HOST, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, C.MEM_HOST, a
    import torch
    if isinstance(a, torch.Tensor):
        a = a.contiguous()
        return a.data_ptr(), (C.MEM_DEVICE if a.is_cuda else C.MEM_HOST), a
    raise TypeError(f"unsupported array type {type(a)}")


def _is_u32(a) -> bool:
    if isinstance(a, np.ndarray):
        return a.dtype == np.uint32
    return a.element_size() == 4 and not a.is_floating_point()


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _flags(symmetrize: bool, reorder: bool, compress: bool = False, out_edges: bool = False) -> int:
    return ((C.SYMMETRIZE if symmetrize else 0) | (C.REORDER if reorder else 0) |
            (C.COMPRESS if compress else 0) | (C.OUT_EDGES if out_edges else 0))


class Graph:
    """Paged CSC graph in library-owned pinned host memory (Sec. 3.1)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def from_edges(cls, n, src, dst, w=None, symmetrize=False, num_pages=1, stream=None,
                   reorder=False, compress=False, out_edges=False):
        ps, ms, ks = _ptr_mem(src)
        pd, md, kd = _ptr_mem(dst)
        pw, mw, kw = _ptr_mem(w)
        if ms != md or (w is not None and mw != ms):
            raise ValueError("src, dst and w must live in the same memory")
        m = int(len(src))
        if len(dst) != m or (w is not None and len(w) != m):
            raise ValueError("src, dst and w must have equal lengths")
        for arr in (ks, kd, kw):
            if arr is not None and not _is_u32(arr):
                raise TypeError("edge arrays must hold 32-bit unsigned integers")
        out = ctypes.c_void_p()
        C.check(C.lib().seraph_graph_from_edges(n, m, ps, pd, pw, ms,
                                                _flags(symmetrize, reorder, compress, out_edges),
                                                num_pages, _stream_ptr(stream), ctypes.byref(out)))
        return cls(out.value)

    @classmethod
    def from_csr(cls, n, row_off, col, w=None, symmetrize=False, num_pages=1, stream=None,
                 reorder=False, compress=False, out_edges=False):
        pr, mr, kr = _ptr_mem(row_off)
        pc, mc, kc = _ptr_mem(col)
        pw, mw, kw = _ptr_mem(w)
        out = ctypes.c_void_p()
        C.check(C.lib().seraph_graph_from_csr(n, pr, pc, pw, mr,
                                              _flags(symmetrize, reorder, compress, out_edges),
                                              num_pages, _stream_ptr(stream), ctypes.byref(out)))
        return cls(out.value)

    def info(self) -> dict:
        gi = C.GraphInfo()
        C.check(C.lib().seraph_graph_get_info(self._h, ctypes.byref(gi)))
        return {k: getattr(gi, k) for k, _ in gi._fields_}

    def page_bounds(self) -> np.ndarray:
        vb = np.empty(self.info()["num_pages"] + 1, dtype=np.uint64)
        C.check(C.lib().seraph_graph_page_bounds(self._h, vb.ctypes.data))
        return vb

    def export_csc(self):
        """(col_off, row, w or None, out_degree) copied out of the pinned pages."""
        i = self.info()
        col_off = np.empty(i["n"] + 1, dtype=np.uint64)
        row = np.empty(max(i["m"], 1), dtype=np.uint32)
        w = np.empty(max(i["m"], 1), dtype=np.uint32) if i["weighted"] else None
        od = np.empty(i["n"], dtype=np.uint32)
        C.check(C.lib().seraph_graph_export_csc(self._h, col_off.ctypes.data, row.ctypes.data,
                                                None if w is None else w.ctypes.data,
                                                od.ctypes.data))
        return col_off, row[:i["m"]], (None if w is None else w[:i["m"]]), od

    def export_packed(self):
        """(boff[n+1], data) of the packed gap streams (compress=True graphs)."""
        i = self.info()
        boff = np.empty(i["n"] + 1, dtype=np.uint64)
        data = np.empty(max(i["packed_data_bytes"], 1), dtype=np.uint8)
        C.check(C.lib().seraph_graph_export_packed(self._h, boff.ctypes.data, data.ctypes.data))
        return boff, data[:i["packed_data_bytes"]]

    def export_out_edges(self):
        """(out_off[n+1], out_col, out_w or None) of an out_edges=True graph,
        in internal ids."""
        i = self.info()
        off = np.empty(i["n"] + 1, dtype=np.uint64)
        col = np.empty(max(i["m"], 1), dtype=np.uint32)
        w = np.empty(max(i["m"], 1), dtype=np.uint32) if i["weighted"] else None
        C.check(C.lib().seraph_graph_export_out_edges(self._h, off.ctypes.data, col.ctypes.data,
                                                      None if w is None else w.ctypes.data))
        return off, col[:i["m"]], (None if w is None else w[:i["m"]])

    def release_buffers(self) -> None:
        """Give back the device buffers that runs keep with the graph."""
        C.check(C.lib().seraph_graph_release_buffers(self._h))

    def perm(self) -> np.ndarray:
        """Internal vertex order: perm[i] = the caller's id of internal vertex i."""
        p = np.empty(self.info()["n"], dtype=np.uint32)
        C.check(C.lib().seraph_graph_export_perm(self._h, p.ctypes.data))
        return p

    def free(self):
        if self._h and self._h.value:
            C.lib().seraph_graph_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class TraceBuffer:
    """Host buffers for a trace of pipeline steps (features + per-pass gains)."""

    def __init__(self, capacity: int):
        self.features = np.zeros((capacity, C.SCHED_FEATURES), dtype=np.float32)
        self.gains = np.zeros((capacity, 16), dtype=np.uint32)
        self.vertices = np.zeros(capacity, dtype=np.uint32)
        self.struct = C.Trace(capacity, 0, self.features.ctypes.data, self.gains.ctypes.data,
                              self.vertices.ctypes.data)

    @property
    def count(self) -> int:
        return int(self.struct.count)

    def rows(self):
        n = self.count
        return self.features[:n], self.gains[:n], self.vertices[:n]

    def targets(self, share: float = 0.95):
        n = self.count
        k = np.empty(n, dtype=np.int32)
        prio = np.empty(n, dtype=np.float32)
        C.check(C.lib().seraph_sched_targets(ctypes.byref(self.struct), share, k.ctypes.data,
                                             prio.ctypes.data))
        return k, prio


class SchedModel:
    """The learned scheduler's network (see include/seraph.h)."""

    def __init__(self, seed: int = 0, fp32: bool = False):
        h = ctypes.c_void_p()
        C.check(C.lib().seraph_sched_create(seed, 1 if fp32 else 0, ctypes.byref(h)))
        self._h = h

    def get_params(self) -> np.ndarray:
        out = np.empty(C.SCHED_PARAMS, dtype=np.float32)
        C.check(C.lib().seraph_sched_get_params(self._h, out.ctypes.data))
        return out

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        C.check(C.lib().seraph_sched_set_params(self._h, p.ctypes.data))

    def loss_grad(self, x, k, prio):
        x = np.ascontiguousarray(x, dtype=np.float32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        prio = np.ascontiguousarray(prio, dtype=np.float32)
        loss = ctypes.c_float()
        grad = np.empty(C.SCHED_PARAMS, dtype=np.float32)
        C.check(C.lib().seraph_sched_loss_grad(self._h, x.ctypes.data, k.ctypes.data,
                                               prio.ctypes.data, len(k), C.MEM_HOST,
                                               ctypes.byref(loss), grad.ctypes.data))
        return loss.value, grad

    def train(self, x, k, prio, epochs=10, batch=256, lr=1e-3, seed=0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        prio = np.ascontiguousarray(prio, dtype=np.float32)
        losses = np.empty(epochs, dtype=np.float32)
        C.check(C.lib().seraph_sched_train(self._h, x.ctypes.data, k.ctypes.data, prio.ctypes.data,
                                           len(k), C.MEM_HOST, epochs, batch, lr, seed,
                                           losses.ctypes.data))
        return losses

    def infer(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = x.shape[0]
        k = np.empty(n, dtype=np.int32)
        prio = np.empty(n, dtype=np.float32)
        C.check(C.lib().seraph_sched_infer(self._h, x.ctypes.data, n, C.MEM_HOST, k.ctypes.data,
                                           prio.ctypes.data))
        return k, prio

    @property
    def handle(self):
        return self._h.value

    def free(self):
        if self._h and self._h.value:
            C.lib().seraph_sched_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def default_params(algo) -> C.Params:
    p = C.Params()
    C.check(C.lib().seraph_params_default(ctypes.byref(p), C.ALGOS[algo] if isinstance(algo, str) else algo))
    return p


def run(graph: Graph, algo, out=None, stream=None, **kw):
    """Run `algo` ("sssp", "bfs", "cc", "pagerank") to its fixpoint.

    Keyword arguments override fields of seraph_params (e.g. source, window,
    passes, budget_bytes, pvu="weak").  `out` may be a preallocated numpy
    array or torch tensor (host or CUDA) of n uint32/float32 values; by
    default a numpy array is returned.  Returns (values, stats dict)."""
    p = default_params(algo)
    trace = kw.pop("trace", None)
    model = kw.pop("sched_model", None)
    if model is not None:
        p.sched_model = model.handle
        p.sched = C.SCHED_LEARNED
    if trace is not None:
        p.trace = ctypes.cast(ctypes.pointer(trace.struct), ctypes.c_void_p)
    for k, v in kw.items():
        if k == "pvu" and isinstance(v, str):
            v = C.PVUS[v]
        if k == "order" and isinstance(v, str):
            v = C.ORDERS[v]
        if k == "columns" and isinstance(v, str):
            v = C.COLUMNS[v]
        if k == "fsm_next":
            for i, x in enumerate(v):
                p.fsm_next[i] = int(x)
            continue
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    p.stream = _stream_ptr(stream)
    n = graph.info()["n"]
    if out is None:
        out = np.empty(n, dtype=np.float32 if p.algo == C.PAGERANK else np.uint32)
    po, mo, ko = _ptr_mem(out)
    st = C.Stats()
    C.check(C.lib().seraph_run(graph._h, ctypes.byref(p), po, mo, ctypes.byref(st)))
    return out, st.as_dict()


def debug_fail_pinned_alloc(k: int) -> None:
    """Make the k-th pinned host allocation from now fail (0 = off); a test
    hook for the ENOMEM path (seraph_debug_fail_pinned_alloc)."""
    C.check(C.lib().seraph_debug_fail_pinned_alloc(int(k)))


def debug_pinned_bytes() -> int:
    """Pinned host bytes the library holds (seraph_debug_pinned_bytes)."""
    return int(C.lib().seraph_debug_pinned_bytes())


def debug_l2_setaside() -> int:
    """The context's persisting-L2 set-aside limit in bytes
    (seraph_debug_l2_setaside)."""
    v = C.u64(0)
    C.check(C.lib().seraph_debug_l2_setaside(ctypes.byref(v)))
    return int(v.value)


def gather_probe(n_values, n_gathers, hot_values, hot_frac=1.0, reps=5, stream=None) -> float:
    """Fastest of `reps` timed launches (seconds) of the random-gather probe:
    n_gathers 4-byte reads of n_values device values, a fraction hot_frac of
    them uniform over the first hot_values (L2 evict-last), the rest uniform
    over the others (seraph_gather_probe in include/seraph.h)."""
    sec = ctypes.c_double(0.0)
    C.check(C.lib().seraph_gather_probe(int(n_values), int(n_gathers), int(hot_values),
                                        float(hot_frac), int(reps), _stream_ptr(stream),
                                        ctypes.byref(sec)))
    return sec.value


class BGraph:
    """Device-resident out-edge CSR for batched queries."""

    def __init__(self, n, src, dst, w=None, stream=None):
        ps, ms, ks = _ptr_mem(src)
        pd, md, kd = _ptr_mem(dst)
        pw, mw, kw = _ptr_mem(w)
        for arr in (ks, kd, kw):
            if arr is not None and not _is_u32(arr):
                raise TypeError("edge arrays must hold 32-bit unsigned integers")
        h = ctypes.c_void_p()
        C.check(C.lib().seraph_bgraph_from_edges(n, int(len(src)), ps, pd, pw, ms,
                                                 _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.n = int(n)

    def free(self):
        if self._h and self._h.value:
            C.lib().seraph_bgraph_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def batch_run(graphs, queries, outs=None, stream=None, **kw):
    """Run queries [(graph index, "bfs"|"sssp", source), ...] in one batched
    launch.  `outs` may give one preallocated array per query (numpy or torch,
    all on the host or all on the device); by default numpy arrays are
    returned.  Keyword arguments override seraph_batch_params (mapping may be
    "auto", "thread", "warp" or "cta")."""
    p = C.BatchParams()
    C.check(C.lib().seraph_batch_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "mapping" and isinstance(v, str):
            v = C.MAPPINGS[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    p.stream = _stream_ptr(stream)
    if outs is None:
        # the library validates indices; an out-of-range one still needs a buffer
        outs = [np.empty(graphs[g].n if 0 <= g < len(graphs) else 1, dtype=np.uint32)
                for g, _, _ in queries]
    arr = (C.Query * len(queries))()
    keep = []
    mem = None
    for i, ((g, algo, src), o) in enumerate(zip(queries, outs)):
        po, mo, ko = _ptr_mem(o)
        keep.append(ko)
        if mem is None:
            mem = mo
        elif mem != mo:
            raise ValueError("all outputs must live in the same memory")
        arr[i] = C.Query(g, C.ALGOS.get(algo, -1) if isinstance(algo, str) else algo, src, 0, po)
    hs = (ctypes.c_void_p * len(graphs))(*[g._h.value for g in graphs])
    st = C.BatchStats()
    C.check(C.lib().seraph_batch_run(hs, len(graphs), arr, len(queries), mem, ctypes.byref(p),
                                     ctypes.byref(st)))
    stats = {k: getattr(st, k) for k, _ in st._fields_ if k not in ("mapping", "tile")}
    stats["mapping"] = list(st.mapping)[:len(graphs)]
    stats["tile"] = list(st.tile)[:len(graphs)]
    return outs, stats


def _batch_params(kw, stream):
    p = C.BatchParams()
    C.check(C.lib().seraph_batch_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "mapping" and isinstance(v, str):
            v = C.MAPPINGS[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    p.stream = _stream_ptr(stream)
    return p


def _batch_stats(st, ng):
    stats = {k: getattr(st, k) for k, _ in st._fields_ if k not in ("mapping", "tile")}
    stats["mapping"] = list(st.mapping)[:ng]
    stats["tile"] = list(st.tile)[:ng]
    return stats


class BatchPlan:
    """A prepared batch (seraph_batch_plan_*): queries [(graph index,
    "bfs"|"sssp", source), ...] with one caller-owned CUDA uint32/int32 tensor
    per query, planned once (autotuning, grouping, device tables, captured
    launch) and run any number of times; each run writes the outputs."""

    def __init__(self, graphs, queries, outs, stream=None, **kw):
        p = _batch_params(kw, stream)
        arr = (C.Query * len(queries))()
        for i, ((g, algo, src), o) in enumerate(zip(queries, outs)):
            po, mo, _ = _ptr_mem(o)
            if mo != C.MEM_DEVICE:
                raise ValueError("plan outputs must be device arrays")
            arr[i] = C.Query(g, C.ALGOS.get(algo, -1) if isinstance(algo, str) else algo, src, 0, po)
        hs = (ctypes.c_void_p * len(graphs))(*[g._h.value for g in graphs])
        h = ctypes.c_void_p()
        C.check(C.lib().seraph_batch_plan_create(hs, len(graphs), arr, len(queries), ctypes.byref(p),
                                                 ctypes.byref(h)))
        self._h = h
        self._keep = (graphs, outs)
        self.nq = len(queries)
        self.ng = len(graphs)

    def run(self, sources=None) -> dict:
        """One launch; `sources` (nq values) replaces the queries' sources."""
        src = None
        if sources is not None:
            src = np.ascontiguousarray(sources, dtype=np.uint32)
            if src.shape != (self.nq,):
                raise ValueError("one source per query")
        st = C.BatchStats()
        C.check(C.lib().seraph_batch_plan_run(self._h, None if src is None else src.ctypes.data,
                                              ctypes.byref(st)))
        return _batch_stats(st, self.ng)

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            C.lib().seraph_batch_plan_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

