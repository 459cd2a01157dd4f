"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Generates raw R-MAT edge lists (with self-loops and duplicates as drawn),
edge weights in [1, 255] and query sources.  The generator definitions are in
``synth.h``; this file builds the two small shared libraries (host: gcc +
OpenMP, device: nvcc for sm_103a) and wraps them with ctypes.

Nothing here builds graph structures or runs any part of the graph method:
the oracle and the product library each do that from the raw edges.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libsynth_host.so")
_DEV_SO = os.path.join(_HERE, "libsynth_dev.so")

# Paper's RMAT-k shape: 2^k vertices, edge factor 16 (evaluation section,
# Table 2); quadrant probabilities a,b,c,d = .57,.19,.19,.05.
RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)
SEED_GRAPH, SEED_WEIGHT, SEED_SOURCE = 1, 2, 3


class _Rmat(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("tA", ctypes.c_uint32), ("tAB", ctypes.c_uint32),
                ("tABC", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


def _threshold(p: Fraction) -> int:
    return min(int(p * (1 << 32)), (1 << 32) - 1)


def rmat_config(scale: int, edge_factor: int = 16, abcd=RMAT_ABCD,
                seed: int = SEED_GRAPH) -> _Rmat:
    """Generator parameters for RMAT-scale with m = edge_factor * 2^scale."""
    if not 1 <= scale <= 32:
        raise ValueError("scale must be in [1, 32]")
    a, b, c = (Fraction(str(x)) for x in abcd[:3])
    return _Rmat(scale, edge_factor << scale, _threshold(a), _threshold(a + b),
                 _threshold(a + b + c), seed)


def build(verbose: bool = False) -> None:
    """Compile libsynth_host.so (gcc) and libsynth_dev.so (nvcc, sm_103a)."""
    host_src = os.path.join(_HERE, "synth_host.c")
    dev_src = os.path.join(_HERE, "synth_dev.cu")
    cmds = []
    if _stale(_HOST_SO, [host_src, os.path.join(_HERE, "synth.h")]):
        cmds.append(["gcc", "-O3", "-march=x86-64-v3", "-fopenmp", "-shared", "-fPIC",
                     host_src, "-o", _HOST_SO])
    if _stale(_DEV_SO, [dev_src, os.path.join(_HERE, "synth.h")]):
        cmds.append(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                     "-lineinfo", "-Xcompiler", "-fPIC", "-shared", dev_src,
                     "-o", _DEV_SO])
    for c in cmds:
        if verbose:
            print(" ".join(c))
        subprocess.run(c, check=True, cwd=_HERE)


def _stale(out, srcs) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        build()
        lib = ctypes.CDLL(_HOST_SO)
        lib.synth_draw.restype = ctypes.c_uint64
        lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_rmat_host.restype = None
        lib.synth_rmat_host.argtypes = [ctypes.POINTER(_Rmat), ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_weights_host.restype = None
        lib.synth_weights_host.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
        _host = lib
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        build()
        lib = ctypes.CDLL(_DEV_SO)
        lib.synth_rmat_device.restype = ctypes.c_int
        lib.synth_rmat_device.argtypes = [ctypes.POINTER(_Rmat), ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        _dev = lib
    return _dev


def draw(seed: int, i: int) -> int:
    """i-th output of the splitmix64 stream seeded with `seed`."""
    return int(_host_lib().synth_draw(seed, i))


def rmat_edges(scale: int, edge_factor: int = 16, abcd=RMAT_ABCD, seed: int = SEED_GRAPH,
               e0: int = 0, count: int | None = None):
    """Raw R-MAT edges [e0, e0+count) on the host: (src, dst) uint32 arrays."""
    cfg = rmat_config(scale, edge_factor, abcd, seed)
    if count is None:
        count = cfg.m - e0
    src = np.empty(count, dtype=np.uint32)
    dst = np.empty(count, dtype=np.uint32)
    _host_lib().synth_rmat_host(ctypes.byref(cfg), e0, count,
                                src.ctypes.data, dst.ctypes.data)
    return src, dst


def weights(src: np.ndarray, dst: np.ndarray, seed_w: int = SEED_WEIGHT) -> np.ndarray:
    """Edge weights w(u,v) in [1,255] for the given endpoint arrays (host)."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    w = np.empty(src.shape[0], dtype=np.uint32)
    _host_lib().synth_weights_host(seed_w, src.shape[0], src.ctypes.data, dst.ctypes.data,
                                   w.ctypes.data)
    return w


def rmat_edges_device(scale: int, src_ptr: int, dst_ptr: int, w_ptr: int | None = None,
                      edge_factor: int = 16, abcd=RMAT_ABCD, seed: int = SEED_GRAPH,
                      seed_w: int = SEED_WEIGHT, stream: int = 0, e0: int = 0,
                      count: int | None = None) -> None:
    """Raw R-MAT edges (and optionally weights) written into device buffers."""
    cfg = rmat_config(scale, edge_factor, abcd, seed)
    if count is None:
        count = cfg.m - e0
    rc = _dev_lib().synth_rmat_device(ctypes.byref(cfg), e0, count, src_ptr, dst_ptr,
                                      w_ptr or None, seed_w, stream or None)
    if rc != 0:
        raise RuntimeError(f"synth_rmat_device failed with CUDA error {rc}")


def pick_sources(n: int, has_out: np.ndarray, count: int, seed: int = SEED_SOURCE) -> list[int]:
    """`count` sources drawn uniformly (with rejection) among vertices that have
    at least one out-edge other than a self-loop.  Draw i is synth draw(seed, i)
    mod n; rejected draws are skipped.  Duplicates are allowed."""
    if not has_out.any():
        raise ValueError("graph has no vertex with an out-edge")
    out, i = [], 0
    while len(out) < count:
        v = draw(seed, i) % n
        i += 1
        if has_out[v]:
            out.append(int(v))
    return out


def has_out_edge(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Mask of vertices with an out-edge that is not a self-loop."""
    mask = np.zeros(n, dtype=bool)
    keep = src != dst
    mask[src[keep]] = True
    return mask


# Batched-query workload: 16 R-MAT graphs of uneven size (scales 14..22,
# edge factors 8..32, four quadrant skews), 256 queries split evenly between
# BFS and SSSP, sources uniform over vertices that have an out-edge.
BATCH_SKEWS = ((0.57, 0.19, 0.19, 0.05), (0.45, 0.15, 0.15, 0.25),
               (0.25, 0.25, 0.25, 0.25), (0.70, 0.10, 0.10, 0.10))


def batch_workload(n_graphs: int = 16, n_queries: int = 256, min_scale: int = 14,
                   max_scale: int = 22, seed: int = 7):
    """Graph specs (scale, edge_factor, abcd, seed) and query specs
    (graph, algo, source-draw seed).  Scales are spread evenly from min to max."""
    graphs = []
    for i in range(n_graphs):
        scale = min_scale + round(i * (max_scale - min_scale) / max(1, n_graphs - 1))
        graphs.append(dict(scale=scale, edge_factor=(8, 16, 32)[i % 3],
                           abcd=BATCH_SKEWS[i % 4], seed=seed * 1000 + i))
    queries = [dict(graph=q % n_graphs, algo="bfs" if (q // n_graphs) % 2 == 0 else "sssp")
               for q in range(n_queries)]
    return graphs, queries
