"""CPU oracle for the Seraph streamed-graph hot path (arXiv 1806.00762).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_1806_00762_b300``) never imports,
links or executes anything here, and this package never touches the product.

The C part (``oracle.c``) writes out the plain definitions: Dijkstra, FIFO
BFS, union-find weakly-connected components and FP64 PageRank power iteration
(evaluation section "Graph Algorithms"; Sec. 4.3 for PageRank), the CSR/CSC
build and the destination-range page cut (Sec. 3.1 "Subgraph Organization"),
the FP64 PageRank step certificate over a replayed raw edge stream
(``pagerank_step_edges``: one map application for graphs too large for one
CSR build, whose residual bounds the L1 distance to the fixpoint),
the out-degree vertex order (``degree_order``; a layout outside the paper
that renames vertices only) and the packed page columns (``pack_gaps``;
LEB128 gaps, a lossless encoding outside the paper).
``mlp.py`` holds the FP64 reference of the learned scheduler's network.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(brute force, Floyd-Warshall, dense linear solves, closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
INF = 0xFFFFFFFF

_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(verbose: bool = False) -> None:
    """Compile liboracle.so with gcc (OpenMP only inside PageRank's vertex loop
    and the certificate edge loop)."""
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
    if os.path.exists(_SO) and all(os.path.getmtime(s) <= os.path.getmtime(_SO) for s in srcs):
        return
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", srcs[0], "-o", _SO, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True, cwd=_HERE)


_lib = None


def _L():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    c_u64, c_u32, c_int, c_dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_build_csr.restype = c_u64
    lib.oracle_build_csr.argtypes = [c_u64, c_u64, _u32p, _u32p, vp, _u64p, _u32p, vp]
    lib.oracle_csc.restype = None
    lib.oracle_csc.argtypes = [c_u64, _u64p, _u32p, vp, _u64p, _u32p, vp]
    lib.oracle_page_cut.restype = None
    lib.oracle_page_cut.argtypes = [c_u64, _u64p, c_u32, _u64p]
    lib.oracle_sssp.restype = c_int
    lib.oracle_sssp.argtypes = [c_u64, _u64p, _u32p, vp, c_u32, _u32p]
    lib.oracle_bfs.restype = None
    lib.oracle_bfs.argtypes = [c_u64, _u64p, _u32p, c_u32, _u32p]
    lib.oracle_cc.restype = None
    lib.oracle_cc.argtypes = [c_u64, _u64p, _u32p, _u32p]
    lib.oracle_cc_edges.restype = None
    lib.oracle_cc_edges.argtypes = [c_u64, c_u64, _u32p, _u32p, _u32p]
    lib.oracle_pagerank.restype = c_int
    lib.oracle_pagerank.argtypes = [c_u64, _u64p, _u32p, c_dbl, c_dbl, c_int, _f64p,
                                    ctypes.POINTER(c_dbl)]
    lib.oracle_pagerank_apply.restype = None
    lib.oracle_pagerank_apply.argtypes = [c_u64, _u64p, _u32p, c_dbl, _f64p, _f64p]
    lib.oracle_pr_bucket_keys.restype = c_u64
    lib.oracle_pr_bucket_keys.argtypes = [c_u64, _u32p, _u32p, c_u32, c_u32, _u64p, c_u64, c_u64]
    lib.oracle_pr_bucket_apply.restype = c_u64
    lib.oracle_pr_bucket_apply.argtypes = [c_u64, _u64p, _u64p, c_u32, c_int, _u32p, c_u64, c_u32,
                                           vp, vp]
    lib.oracle_sp_check_edges.restype = c_u64
    lib.oracle_sp_check_edges.argtypes = [c_u64, _u32p, _u32p, vp, _u32p, _u8p]
    lib.oracle_sp_check_tight.restype = c_u64
    lib.oracle_sp_check_tight.argtypes = [c_u64, c_u32, _u32p, _u8p]
    _lib = lib
    return lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a):
    return None if a is None else a.ctypes.data


class CSR:
    """Simple directed graph: rows = sources, columns ascending in each row."""

    def __init__(self, n, row_off, col, w=None):
        self.n, self.row_off, self.col, self.w = int(n), row_off, col, w

    @property
    def m(self) -> int:
        return int(self.row_off[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_off)


def build_csr(n: int, src, dst, w=None) -> CSR:
    """Drop self-loops, collapse duplicate (u,v) keeping the smallest weight."""
    src, dst = _u32(src), _u32(dst)
    m = src.shape[0]
    wa = None if w is None else _u32(w)
    row_off = np.zeros(n + 1, dtype=np.uint64)
    col = np.empty(max(m, 1), dtype=np.uint32)
    wout = None if w is None else np.empty(max(m, 1), dtype=np.uint32)
    E = _L().oracle_build_csr(n, m, src, dst, _ptr(wa), row_off, col, _ptr(wout))
    return CSR(n, row_off, col[:E].copy(), None if w is None else wout[:E].copy())


def symmetrize(src, dst, w=None):
    """Raw edge list plus its reverse (for the undirected view used by CC)."""
    s = np.concatenate([_u32(src), _u32(dst)])
    d = np.concatenate([_u32(dst), _u32(src)])
    return s, d, (None if w is None else np.concatenate([_u32(w), _u32(w)]))


def csc(g: CSR):
    """(col_off, row, w_csc): in-edges per destination, sources ascending."""
    col_off = np.zeros(g.n + 1, dtype=np.uint64)
    row = np.empty(max(g.m, 1), dtype=np.uint32)
    wc = None if g.w is None else np.empty(max(g.m, 1), dtype=np.uint32)
    _L().oracle_csc(g.n, g.row_off, g.col, _ptr(g.w), col_off, row, _ptr(wc))
    return col_off, row[:g.m].copy(), (None if wc is None else wc[:g.m].copy())


def degree_order(g: CSR) -> np.ndarray:
    """perm[i] = the vertex listed i-th when vertices are ordered by
    non-increasing out-degree (kept edges), ties by ascending id.

    Not in the paper: the product may renumber vertices this way before the
    page cut (a memory-layout choice that leaves every result unchanged).  The
    plain definition is a stable two-key sort."""
    deg = g.out_degree().astype(np.int64)
    return np.lexsort((np.arange(g.n, dtype=np.int64), -deg)).astype(np.uint32)


def relabel(g: CSR, perm) -> CSR:
    """The same graph with vertex perm[i] renamed i (weights kept)."""
    perm = _u32(perm)
    inv = np.empty(g.n, dtype=np.uint32)
    inv[perm] = np.arange(g.n, dtype=np.uint32)
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.row_off).astype(np.int64))
    return build_csr(g.n, inv[src], inv[g.col], g.w)


def leb128(value: int) -> bytes:
    """Unsigned LEB128: 7 bits per byte, least significant group first, the
    high bit set on every byte but the last."""
    out = bytearray()
    while True:
        b = value & 0x7F
        value >>= 7
        if value:
            out.append(b | 0x80)
        else:
            out.append(b)
            return bytes(out)


def pack_gaps(col_off, row):
    """Packed page columns of a CSC (not in the paper; a lossless form of its
    compact pages): for each destination, its first source id and then each
    gap to the next source minus one, every value as unsigned LEB128, the
    destinations' bytes back to back.  Returns (boff[n+1] byte offsets, data)."""
    col_off = np.asarray(col_off, dtype=np.int64)
    row = np.asarray(row, dtype=np.int64)
    n = col_off.shape[0] - 1
    first = np.zeros(row.shape[0], dtype=bool)
    first[col_off[:-1][np.diff(col_off) > 0]] = True
    vals = row.copy()
    gaps = np.zeros_like(row)
    gaps[1:] = row[1:] - row[:-1] - 1
    vals[~first] = gaps[~first]
    nbytes = 1 + sum((vals >= (1 << (7 * k))).astype(np.int64) for k in range(1, 5))
    pos = np.zeros(row.shape[0] + 1, dtype=np.int64)
    np.cumsum(nbytes, out=pos[1:])
    data = np.zeros(int(pos[-1]), dtype=np.uint8)
    for k in range(5):
        sel = nbytes > k
        byte = (vals[sel] >> (7 * k)) & 0x7F
        more = nbytes[sel] > k + 1
        data[pos[:-1][sel] + k] = (byte | np.where(more, 0x80, 0)).astype(np.uint8)
    boff = pos[col_off].astype(np.uint64)
    return boff, data


def unpack_gaps(boff, data, n: int):
    """Inverse of pack_gaps (pure Python; small inputs): per destination the
    list of source ids."""
    out = []
    for v in range(n):
        ids, prev, val, shift = [], -1, 0, 0
        for b in data[int(boff[v]):int(boff[v + 1])]:
            val |= (int(b) & 0x7F) << shift
            shift += 7
            if not b & 0x80:
                prev = val if not ids else prev + val + 1
                ids.append(prev)
                val, shift = 0, 0
        out.append(ids)
    return out


def page_cut(n: int, col_off: np.ndarray, P: int) -> np.ndarray:
    """Vertex boundaries vb[0..P] of P destination-range pages balanced on
    (vertices + in-edges)."""
    vb = np.zeros(P + 1, dtype=np.uint64)
    _L().oracle_page_cut(n, np.ascontiguousarray(col_off, dtype=np.uint64), P, vb)
    return vb


class OverflowError_(RuntimeError):
    pass


def sssp(g: CSR, source: int) -> np.ndarray:
    dist = np.empty(g.n, dtype=np.uint32)
    rc = _L().oracle_sssp(g.n, g.row_off, g.col, _ptr(g.w), source, dist)
    if rc == -6:
        raise OverflowError_("a shortest distance does not fit below 0xFFFFFFFF")
    return dist


def bfs(g: CSR, source: int) -> np.ndarray:
    level = np.empty(g.n, dtype=np.uint32)
    _L().oracle_bfs(g.n, g.row_off, g.col, source, level)
    return level


def cc(g: CSR) -> np.ndarray:
    label = np.empty(g.n, dtype=np.uint32)
    _L().oracle_cc(g.n, g.row_off, g.col, label)
    return label


def cc_edges(n: int, src, dst) -> np.ndarray:
    """Weakly connected components (min-id labels) straight from a raw edge
    list: the union-find of ``cc`` without the CSR build (large graphs)."""
    src, dst = _u32(src), _u32(dst)
    label = np.empty(n, dtype=np.uint32)
    _L().oracle_cc_edges(n, src.shape[0], src, dst, label)
    return label


def pagerank(g: CSR, d: float = 0.85, tol: float = 1e-15, maxit: int = 2000):
    """Returns (x, iterations, last L1 change)."""
    x = np.empty(g.n, dtype=np.float64)
    r = ctypes.c_double(0.0)
    it = _L().oracle_pagerank(g.n, g.row_off, g.col, d, tol, maxit, x, ctypes.byref(r))
    return x, it, r.value


def pagerank_apply(g: CSR, x: np.ndarray, d: float = 0.85) -> np.ndarray:
    y = np.empty(g.n, dtype=np.float64)
    _L().oracle_pagerank_apply(g.n, g.row_off, g.col, d,
                               np.ascontiguousarray(x, dtype=np.float64), y)
    return y


def pagerank_step_edges(n: int, edge_chunks, x, d: float = 0.85, nbuckets: int = 4,
                        nsub: int = 256, cap: int | None = None, m_hint: int | None = None):
    """One FP64 PageRank map application T(x) (same definition as
    ``pagerank_apply``) over a raw edge stream, for graphs too large to build
    as one CSR; ``x`` may also hold several vectors as the rows of an (nx, n)
    array, each mapped in the same rounds.  ``edge_chunks()`` must return a fresh iterator of (src, dst)
    uint32 chunks of the raw edges (self-loops and duplicates as drawn); it is
    replayed 2 * nbuckets times: one round over the destination classes for
    the kept out-degrees, one for the pull sums.  Returns (T(x), distinct
    edge count).  ``cap`` bounds the keys held at once (default 1.25 m /
    nbuckets + 2^20 with ``m_hint`` raw edges).

    ||x - x*||_1 <= ||T(x) - x||_1 / (1 - d) for every x (T is a
    d-contraction in L1), which makes this a certificate of a claimed
    fixpoint without computing the fixpoint."""
    L = _L()
    x = np.ascontiguousarray(x, dtype=np.float64)
    single = x.ndim == 1
    x = x.reshape(-1, n)
    nx = x.shape[0]
    if cap is None:
        if m_hint is None:
            raise ValueError("give cap or m_hint")
        cap = int(1.25 * m_hint / nbuckets) + (1 << 20)
    keys = np.empty(cap, dtype=np.uint64)
    tmp = np.empty(cap, dtype=np.uint64)
    outdeg = np.zeros(n, dtype=np.uint32)
    s = np.zeros((nx, n), dtype=np.float64)
    distinct = 0
    for mode in (0, 1):
        for b in range(nbuckets):
            k = 0
            for src, dst in edge_chunks():
                src, dst = _u32(src), _u32(dst)
                k = int(L.oracle_pr_bucket_keys(src.shape[0], src, dst, b, nbuckets, keys, k, cap))
                if k == (1 << 64) - 1:
                    raise MemoryError("destination class larger than cap")
            cnt = int(L.oracle_pr_bucket_apply(k, keys, tmp, nsub, mode, outdeg, n, nx,
                                               x.ctypes.data if mode else None,
                                               s.ctypes.data if mode else None))
            if mode == 0:
                distinct += cnt
    del keys, tmp
    dangling = x[:, outdeg == 0].sum(axis=1)
    y = (1.0 - d) / n + d * (s + dangling[:, None] / n)
    return (y[0] if single else y), distinct


def sp_check_edges(src, dst, w, dist, tight) -> int:
    """Triangle-inequality violations over a raw edge stream; marks tight[v]."""
    src, dst = _u32(src), _u32(dst)
    wa = None if w is None else _u32(w)
    return int(_L().oracle_sp_check_edges(src.shape[0], src, dst, _ptr(wa), _u32(dist), tight))


def sp_check_tight(source: int, dist, tight) -> int:
    dist = _u32(dist)
    return int(_L().oracle_sp_check_tight(dist.shape[0], source, dist, tight))
