"""Pins for the CPU oracle: each oracle function is checked against something
other than itself -- brute force, Floyd-Warshall, dense linear solves, closed
forms, published generator vectors and invariants -- chosen so that a dropped
term, a wrong sign or index or a transposed operand fails at least one case.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import graphs

INF = oracle.INF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ input module

def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, i, out = (int(t) for t in line.split())
        assert synth.draw(seed, i) == out


def _rmat_edge_python(cfg, e):
    """The R-MAT definition of synth.h, restated with Python integers."""
    M = (1 << 64) - 1
    g = 0x9E3779B97F4A7C15

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    s = d = 0
    k = cfg.scale
    for level in range(k):
        r64 = mix((cfg.seed + (e * 16 + (level >> 1) + 1) * g) & M)
        r = (r64 >> 32) if level & 1 else (r64 & 0xFFFFFFFF)
        sb, db = (0, 0) if r < cfg.tA else (0, 1) if r < cfg.tAB else (1, 0) if r < cfg.tABC else (1, 1)
        s |= sb << (k - 1 - level)
        d |= db << (k - 1 - level)
    return s, d


def test_rmat_matches_definition():
    cfg = synth.rmat_config(14)
    src, dst = synth.rmat_edges(14, e0=1000, count=64)
    for t in range(64):
        assert (int(src[t]), int(dst[t])) == _rmat_edge_python(cfg, 1000 + t)


def test_rmat_thresholds_and_quadrant_frequencies():
    cfg = synth.rmat_config(16)
    assert (cfg.tA, cfg.tAB, cfg.tABC) == (2448131358, 3264175144, 4080218931)
    src, dst = synth.rmat_edges(16)
    assert len(src) == 16 << 16
    # each level sets a source bit with probability c+d = .24 and a
    # destination bit with probability b+d = .24
    for bit in (0, 7, 15):
        fs = ((src >> bit) & 1).mean()
        fd = ((dst >> bit) & 1).mean()
        assert abs(fs - 0.24) < 0.003 and abs(fd - 0.24) < 0.003


def test_weights_range_and_symmetry_of_definition():
    src, dst = synth.rmat_edges(12)
    w = synth.weights(src, dst)
    assert w.min() >= 1 and w.max() <= 255
    # the weight depends only on (u, v): duplicates agree
    w2 = synth.weights(src[::-1].copy(), dst[::-1].copy())[::-1]
    assert np.array_equal(w, w2)
    assert abs(w.mean() - 128) < 2


# ------------------------------------------------------------ graph build

def test_build_csr_against_numpy_unique():
    src, dst, w = graphs.random_graph(300, 5000, seed=1, wmax=9)
    g = oracle.build_csr(300, src, dst, w)
    keep = src != dst
    key = (src[keep].astype(np.uint64) << np.uint64(32)) | dst[keep]
    order = np.lexsort((w[keep], key))
    k_sorted, w_sorted = key[order], w[keep][order]
    first = np.ones(len(k_sorted), dtype=bool)
    first[1:] = k_sorted[1:] != k_sorted[:-1]
    assert g.m == first.sum()
    assert np.array_equal(g.col, (k_sorted[first] & np.uint64(0xFFFFFFFF)).astype(np.uint32))
    assert np.array_equal(g.w, w_sorted[first])  # smallest weight per duplicate group
    assert np.array_equal(np.diff(g.row_off), np.bincount((k_sorted[first] >> np.uint64(32)).astype(np.int64), minlength=300))


def test_csc_is_transpose():
    import scipy.sparse as sp
    src, dst, w = graphs.random_graph(200, 3000, seed=2)
    g = oracle.build_csr(200, src, dst, w)
    col_off, row, wc = oracle.csc(g)
    A = sp.csr_matrix((g.w.astype(np.int64), g.col, g.row_off.astype(np.int64)), shape=(200, 200))
    T = A.T.tocsr()
    T.sort_indices()
    assert np.array_equal(col_off.astype(np.int64), T.indptr)
    assert np.array_equal(row, T.indices.astype(np.uint32))
    assert np.array_equal(wc, T.data.astype(np.uint32))


@pytest.mark.parametrize("P", [1, 2, 3, 7, 64])
def test_page_cut_definition(P):
    src, dst, _ = graphs.random_graph(500, 4000, seed=P)
    g = oracle.build_csr(500, src, dst)
    col_off, _, _ = oracle.csc(g)
    vb = oracle.page_cut(500, col_off, P).astype(np.int64)
    n, E = 500, int(col_off[-1])
    cost = np.arange(n + 1) + col_off.astype(np.int64)
    assert vb[0] == 0 and vb[P] == n and np.all(np.diff(vb) >= 0)
    for j in range(1, P):
        # smallest v with cost(v) * P >= j * (n + E), by brute force
        want = next(v for v in range(n + 1) if cost[v] * P >= j * (n + E))
        assert vb[j] == want


def test_degree_order_worked_example():
    """Out-degrees (kept edges) 0:1 1:3 2:0 3:3 4:1 5:2 -- the self-loop 2->2
    and the duplicate 1->2 do not count -- so the order is 1, 3 (degree 3, by
    id), 5, 0, 4 (degree 1, by id), 2."""
    src = np.array([0, 1, 1, 1, 1, 2, 3, 3, 3, 4, 5, 5], np.uint32)
    dst = np.array([1, 0, 2, 2, 3, 2, 0, 1, 5, 0, 0, 4], np.uint32)
    g = oracle.build_csr(6, src, dst)
    assert list(oracle.degree_order(g)) == [1, 3, 5, 0, 4, 2]


def test_degree_order_by_brute_force_and_relabel_is_an_isomorphism():
    for seed in range(6):
        n = 40
        src, dst, w = graphs.random_graph(n, 160, seed=seed)
        g = oracle.build_csr(n, src, dst, w)
        perm = oracle.degree_order(g)
        deg = [sum(1 for u, v in set(zip(src.tolist(), dst.tolist())) if u == x and u != v)
               for x in range(n)]
        # brute force: position of x = vertices that must precede it
        for x in range(n):
            before = sum(1 for y in range(n) if deg[y] > deg[x] or (deg[y] == deg[x] and y < x))
            assert perm[before] == x
        h = oracle.relabel(g, perm)
        inv = np.empty(n, np.int64)
        inv[perm] = np.arange(n)
        assert h.m == g.m
        edges_g = {(int(inv[u]), int(v_), int(c)) for u in range(n)
                   for v_, c in zip(inv[g.col[g.row_off[u]:g.row_off[u + 1]]],
                                    g.w[g.row_off[u]:g.row_off[u + 1]])}
        edges_h = {(u, int(v_), int(c)) for u in range(n)
                   for v_, c in zip(h.col[h.row_off[u]:h.row_off[u + 1]],
                                    h.w[h.row_off[u]:h.row_off[u + 1]])}
        assert edges_g == edges_h
        assert np.all(np.diff(h.out_degree().astype(np.int64)) <= 0)


def test_leb128_published_example_and_boundaries():
    """The unsigned-LEB128 example of the DWARF specification (624485 ->
    E5 8E 26) and the code-length boundaries of the definition."""
    assert oracle.leb128(624485) == bytes([0xE5, 0x8E, 0x26])
    assert oracle.leb128(0) == b"\x00" and oracle.leb128(127) == b"\x7f"
    assert oracle.leb128(128) == b"\x80\x01" and oracle.leb128(16383) == b"\xff\x7f"
    assert oracle.leb128(16384) == b"\x80\x80\x01"
    assert oracle.leb128(2**32 - 1) == b"\xff\xff\xff\xff\x0f"


def test_pack_gaps_against_scalar_codes_and_decoder():
    rng = np.random.default_rng(3)
    for seed in range(5):
        n = 60
        src, dst, _ = graphs.random_graph(n, 400, seed=seed)
        g = oracle.build_csr(n, src, dst)
        col_off, row, _ = oracle.csc(g)
        # scale ids up so that 1- to 5-byte codes all occur
        big = (row.astype(np.int64) * rng.integers(1, 70_000_000, size=1)[0]) % (2**32 - 1)
        lists = [sorted(set(big[col_off[v]:col_off[v + 1]].tolist())) for v in range(n)]
        co = np.zeros(n + 1, dtype=np.int64)
        co[1:] = np.cumsum([len(x) for x in lists])
        rw = np.array([u for x in lists for u in x], dtype=np.int64)
        boff, data = oracle.pack_gaps(co, rw)
        want = b"".join(oracle.leb128(x[0]) + b"".join(oracle.leb128(b - a - 1) for a, b in zip(x, x[1:]))
                        if x else b"" for x in lists)
        assert data.tobytes() == want
        assert oracle.unpack_gaps(boff, data, n) == lists
        assert boff[0] == 0 and boff[-1] == len(want)


# ------------------------------------------------------------------ SSSP

def floyd_warshall(n, src, dst, w):
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    for u, v, c in zip(src, dst, w):
        if u != v:
            D[u, v] = min(D[u, v], c)
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def _as_u32(row):
    return np.where(np.isinf(row), INF, row).astype(np.uint64).astype(np.uint32)


@pytest.mark.parametrize("seed", range(12))
def test_sssp_vs_floyd_warshall(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 65))
    m = int(rng.integers(0, 4 * n + 1))
    src, dst, w = graphs.random_graph(n, m, seed=seed)
    g = oracle.build_csr(n, src, dst, w)
    D = floyd_warshall(n, src, dst, w)
    for s in range(0, n, max(1, n // 5)):
        assert np.array_equal(oracle.sssp(g, s), _as_u32(D[s]))


@pytest.mark.parametrize("seed", range(8))
def test_bfs_vs_floyd_warshall_unit(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 65))
    src, dst, _ = graphs.random_graph(n, int(rng.integers(0, 3 * n + 1)), seed=seed)
    g = oracle.build_csr(n, src, dst)
    D = floyd_warshall(n, src, dst, np.ones(len(src)))
    for s in range(0, n, max(1, n // 4)):
        assert np.array_equal(oracle.bfs(g, s), _as_u32(D[s]))


def test_sssp_invariants_rmat():
    src, dst = synth.rmat_edges(12)
    w = synth.weights(src, dst)
    g = oracle.build_csr(1 << 12, src, dst, w)
    dist = oracle.sssp(g, 0)
    u = np.repeat(np.arange(g.n), np.diff(g.row_off).astype(np.int64))
    du = dist[u].astype(np.uint64)
    dv = dist[g.col].astype(np.uint64)
    fin = dist[u] != INF
    assert np.all(dv[fin] <= du[fin] + g.w[fin])                 # triangle inequality
    tight = np.zeros(g.n, bool)
    tight[g.col[fin & (dv == du + g.w)]] = True                   # tightness
    reached = (dist != INF)
    reached[0] = False
    assert np.all(tight[reached]) and dist[0] == 0


def test_sssp_overflow_detected():
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 3], np.uint32)
    w = np.array([0xFFFFFF00, 0xFF, 0x10], np.uint32)
    g = oracle.build_csr(4, src, dst, w)
    with pytest.raises(oracle.OverflowError_):
        oracle.sssp(g, 0)


def test_sp_certificate_accepts_exact_and_rejects_planted_mistakes():
    src, dst = synth.rmat_edges(11)
    w = synth.weights(src, dst)
    g = oracle.build_csr(1 << 11, src, dst, w)
    dist = oracle.sssp(g, 0)
    tight = np.zeros(g.n, np.uint8)
    assert oracle.sp_check_edges(src, dst, w, dist, tight) == 0
    assert oracle.sp_check_tight(0, dist, tight) == 0
    reached = np.nonzero((dist != INF) & (dist > 0))[0]
    for delta in (-1, +1):                     # too small / too large by one
        bad = dist.copy()
        i = reached[len(reached) // 2]
        bad[i] = np.uint32(int(bad[i]) + delta)
        tight = np.zeros(g.n, np.uint8)
        e = oracle.sp_check_edges(src, dst, w, bad, tight)
        t = oracle.sp_check_tight(0, bad, tight)
        assert e + t > 0


# -------------------------------------------------------------------- CC

@pytest.mark.parametrize("seed", range(10))
def test_cc_vs_reachability(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 65))
    src, dst, _ = graphs.random_graph(n, int(rng.integers(0, n + 1)), seed=seed)
    g = oracle.build_csr(n, src, dst)
    R = np.eye(n, dtype=bool)
    for u, v in zip(src, dst):
        R[u, v] = R[v, u] = True
    for _ in range(max(1, int(np.ceil(np.log2(max(n, 2)))) + 1)):  # transitive closure
        R = (R.astype(np.int64) @ R.astype(np.int64)) > 0
    # the CSR form and the raw-edge form (self-loops and duplicates as drawn)
    for lab in (oracle.cc(g), oracle.cc_edges(n, src, dst)):
        for v in range(n):
            comp = np.nonzero(R[v])[0]
            assert lab[v] == comp.min()                         # label = min id
            assert np.all(lab[comp] == lab[v])                  # equal iff connected
            assert np.all(lab[np.nonzero(~R[v])[0]] != lab[v])


def test_cc_vs_scipy_rmat():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    src, dst = synth.rmat_edges(13)
    g = oracle.build_csr(1 << 13, src, dst)
    lab = oracle.cc(g)
    A = csr_matrix((np.ones(g.m), g.col, g.row_off.astype(np.int64)), shape=(g.n, g.n))
    k, sc = connected_components(A, directed=True, connection="weak")
    assert len(np.unique(lab)) == k
    # same partition: map scipy's component ids to min vertex ids
    mins = np.full(k, g.n)
    np.minimum.at(mins, sc, np.arange(g.n))
    assert np.array_equal(lab, mins[sc].astype(np.uint32))
    assert np.array_equal(oracle.cc_edges(g.n, src, dst), lab)  # raw edges, one direction each


# -------------------------------------------------------------- PageRank

D = 0.85


def pr_dense_solve(n, src, dst, d=D):
    """(I - d A) x = (1-d)/n 1 with A = P^T + (1/n) 1 e_dangling^T."""
    adj = np.zeros((n, n))
    for u, v in zip(src, dst):
        if u != v:
            adj[u, v] = 1.0
    out = adj.sum(1)
    A = np.zeros((n, n))
    for u in range(n):
        if out[u] > 0:
            A[:, u] = adj[u] / out[u]
        else:
            A[:, u] = 1.0 / n
    return np.linalg.solve(np.eye(n) - d * A, np.full(n, (1 - d) / n))


@pytest.mark.parametrize("seed", range(10))
def test_pagerank_vs_dense_solve(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(1, 65))
    src, dst, _ = graphs.random_graph(n, int(rng.integers(0, 3 * n + 1)), seed=seed)
    g = oracle.build_csr(n, src, dst)
    x, it, r = oracle.pagerank(g)
    ref = pr_dense_solve(n, src, dst)
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-14)
    assert abs(x.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_pagerank_cycle_and_complete_are_uniform(n):
    for src, dst, _ in (graphs.cycle_graph(n), graphs.complete_graph(n)):
        g = oracle.build_csr(n, src, dst)
        x, _, _ = oracle.pagerank(g)
        assert np.allclose(x, 1.0 / n, rtol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 10, 64])
def test_pagerank_star_closed_form(n):
    src, dst, _ = graphs.star_graph(n, center=0)
    g = oracle.build_csr(n, src, dst)
    x, _, _ = oracle.pagerank(g)
    centre = ((1 - D) / n + D) / (1 + D)
    assert abs(x[0] - centre) < 1e-13
    assert np.allclose(x[1:], (1 - centre) / (n - 1), rtol=1e-12)


def test_pagerank_all_dangling_is_uniform():
    g = oracle.build_csr(7, np.array([], np.uint32), np.array([], np.uint32))
    x, _, _ = oracle.pagerank(g)
    assert np.allclose(x, 1 / 7, rtol=1e-14)


def test_pagerank_apply_fixpoint_and_contraction():
    src, dst = synth.rmat_edges(10)
    g = oracle.build_csr(1 << 10, src, dst)
    x, _, _ = oracle.pagerank(g)
    assert np.abs(oracle.pagerank_apply(g, x) - x).sum() < 1e-14
    y0 = np.random.default_rng(0).random(g.n)
    y0 /= y0.sum()
    y1 = oracle.pagerank_apply(g, y0)
    # L1 contraction by d on probability vectors
    assert np.abs(oracle.pagerank_apply(g, y1) - y1).sum() <= D * np.abs(y1 - y0).sum() + 1e-15


# ------------------------------------------- PageRank step certificate

def pr_dense_map(n, src, dst, x, d=D):
    """T(x) = (1-d)/n + d A x with the same dense A as pr_dense_solve."""
    adj = np.zeros((n, n))
    for u, v in zip(src, dst):
        if u != v:
            adj[u, v] = 1.0
    out = adj.sum(1)
    A = np.where(out[None, :] > 0, adj.T / np.maximum(out, 1)[None, :], 1.0 / n)
    return (1 - d) / n + d * (A @ x)


def _chunks(src, dst, size):
    def it():
        for e0 in range(0, len(src), size):
            yield src[e0:e0 + size], dst[e0:e0 + size]
    return it


@pytest.mark.parametrize("seed", range(6))
def test_pagerank_step_edges_vs_dense_map(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 65))
    src, dst, _ = graphs.random_graph(n, int(rng.integers(0, 3 * n + 1)), seed=seed)
    x = rng.random(n)
    y, E = oracle.pagerank_step_edges(n, _chunks(src, dst, 7), x, nbuckets=int(rng.integers(1, 5)),
                                      nsub=int(rng.integers(1, 9)), m_hint=max(len(src), 1))
    assert np.allclose(y, pr_dense_map(n, src, dst, x), rtol=1e-13, atol=1e-16)
    assert E == len({(int(u), int(v)) for u, v in zip(src, dst) if u != v})


@pytest.mark.parametrize("nb,nsub", [(1, 1), (3, 7), (8, 256)])
def test_pagerank_step_edges_matches_csr_map_on_rmat(nb, nsub):
    n = 1 << 12
    src, dst = synth.rmat_edges(12)
    g = oracle.build_csr(n, src, dst)
    x = np.random.default_rng(nb).random(n)
    y, E = oracle.pagerank_step_edges(n, _chunks(src, dst, 10007), x, nbuckets=nb, nsub=nsub,
                                      m_hint=len(src))
    assert E == g.m
    assert np.allclose(y, oracle.pagerank_apply(g, x), rtol=1e-14, atol=0)


def test_pagerank_step_certificate_bounds_the_error():
    n = 1 << 11
    src, dst = synth.rmat_edges(11)
    g = oracle.build_csr(n, src, dst)
    xs, _, _ = oracle.pagerank(g)
    it = _chunks(src, dst, 1 << 14)
    y, _ = oracle.pagerank_step_edges(n, it, xs, nbuckets=2, m_hint=len(src))
    assert np.abs(y - xs).sum() < 1e-14
    rng = np.random.default_rng(5)
    for scale in (1e-3, 1e-6):
        x = xs + scale * rng.standard_normal(n) / n
        y, _ = oracle.pagerank_step_edges(n, it, x, nbuckets=2, m_hint=len(src))
        r = np.abs(y - x).sum()
        # (1 - d) ||x - x*||_1 <= ||T x - x||_1 <= (1 + d) ||x - x*||_1
        assert np.abs(x - xs).sum() <= r / (1 - D) * (1 + 1e-9)
        assert r <= (1 + D) * np.abs(x - xs).sum() * (1 + 1e-9)
    # one vertex off by delta: (1-d)|delta| <= residual <= (1+d)|delta|
    for v in (0, 17, n - 1):
        x = xs.copy()
        x[v] += 1e-4
        y, _ = oracle.pagerank_step_edges(n, it, x, nbuckets=3, m_hint=len(src))
        r = np.abs(y - x).sum()
        assert (1 - D) * 1e-4 * (1 - 1e-9) <= r <= (1 + D) * 1e-4 * (1 + 1e-9)


def test_pagerank_step_edges_rejects_a_too_small_buffer():
    src, dst = synth.rmat_edges(10)
    with pytest.raises(MemoryError):
        oracle.pagerank_step_edges(1 << 10, _chunks(src, dst, 4096), np.ones(1 << 10), cap=100)


def test_pagerank_step_edges_maps_several_vectors_at_once():
    n = 1 << 10
    src, dst = synth.rmat_edges(10)
    g = oracle.build_csr(n, src, dst)
    X = np.random.default_rng(3).random((3, n))
    Y, _ = oracle.pagerank_step_edges(n, _chunks(src, dst, 5000), X, nbuckets=2, m_hint=len(src))
    for j in range(3):
        assert np.allclose(Y[j], oracle.pagerank_apply(g, X[j]), rtol=1e-14, atol=0)
