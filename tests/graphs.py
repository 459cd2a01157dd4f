"""Seeded small test graphs (raw edge lists) for pins and parity cases.

Shapes follow the adversarial list used for the streamed path: paths,
stars, a hub larger than a page, isolated vertices, a single vertex, no
edges, maximum weights.  Random graphs use numpy's seeded PCG64.
"""
import numpy as np


def random_graph(n, m, seed, wmax=255, self_loops=True, dups=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    if not self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    if dups and len(src) > 2:
        src = np.concatenate([src, src[: len(src) // 4]])
        dst = np.concatenate([dst, dst[: len(dst) // 4]])
    w = rng.integers(1, wmax + 1, len(src), dtype=np.uint32)
    return src.astype(np.uint32), dst.astype(np.uint32), w


def path_graph(n, w=1, directed=True):
    src = np.arange(n - 1, dtype=np.uint32)
    dst = src + 1
    if not directed:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    return src, dst, np.full(len(src), w, dtype=np.uint32)


def reverse_path_graph(n, w=1):
    """Edges i+1 -> i: the worst order for a forward sweep from vertex n-1."""
    dst = np.arange(n - 1, dtype=np.uint32)
    src = dst + 1
    return src, dst, np.full(len(src), w, dtype=np.uint32)


def star_graph(n, center=0, undirected=True):
    leaves = np.array([v for v in range(n) if v != center], dtype=np.uint32)
    c = np.full(len(leaves), center, dtype=np.uint32)
    if undirected:
        src, dst = np.concatenate([c, leaves]), np.concatenate([leaves, c])
    else:
        src, dst = c, leaves
    return src, dst, np.ones(len(src), dtype=np.uint32)


def cycle_graph(n):
    src = np.arange(n, dtype=np.uint32)
    dst = ((src + 1) % n).astype(np.uint32)
    return src, dst, np.ones(n, dtype=np.uint32)


def complete_graph(n):
    src, dst = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32))
    src, dst = src.ravel(), dst.ravel()
    keep = src != dst
    return src[keep], dst[keep], np.ones(int(keep.sum()), dtype=np.uint32)
