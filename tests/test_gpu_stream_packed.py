"""Plain chunks streamed compact and rebuilt on the device
(seraph_params.stream_packed): the host link carries, per page, a header of
two bytes per vertex (in-degree, code bytes; larger counts escaped) with a
checkpoint of both offsets every 256 vertices, and the page's LEB128 gap
stream; a kernel rebuilds each page's plain form in the ring slot (page by
page, each page's plain bytes ending before its staged bytes start), and the
run relaxes plain pages as before.

Checked against the oracle -- bit-exact for SSSP, BFS and CC, within the
PageRank tolerance -- for plain and hybrid page forms, resident and
streamed rings (every sweep decodes again), windows 1 and 4, vertex
orders, weight widths of 1, 2 and 4 bytes, hub vertices whose code bytes
need the warp decode, escaped counts at and around tile boundaries of
ragged pages, and graphs of a few vertices; fewer bytes streamed than
without it; a ring too small for the staging falls back to plain copies; a
graph without the packed form is rejected."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C
from tests import graphs
from tests.test_gpu_parity import PR_L1, PR_REL, oracle_graph, pr_errors, rmat

pytestmark = pytest.mark.gpu


def plain_budget(g, slots, use_w=True, per_slot=1.6):
    i = g.info()
    slot = (i["max_page_struct_bytes"] + 255) // 256 * 256 + (i["max_page_weight_bytes"] if use_w else 0)
    slot += (i["max_page_packed_bytes"] + 255) // 256 * 256  # the staging slack
    return int(slots * slot * per_slot) + 256 * slots


@pytest.fixture(scope="module")
def r14():
    import torch
    torch.cuda.set_device(0)
    n, src, dst, w = rmat(14)
    og = oracle_graph(n, src, dst, w)
    mk = dict(num_pages=40, compress=True)
    g = seraph.Graph.from_edges(n, src, dst, w, **mk)
    gr = seraph.Graph.from_edges(n, src, dst, w, reorder=True, **mk)
    gs = seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, reorder=True, **mk)
    ref = dict(sssp=oracle.sssp(og, 3), bfs=oracle.bfs(og, 3), cc=oracle.cc_edges(n, src, dst),
               pr=oracle.pagerank(og)[0])
    yield dict(n=n, g=g, gr=gr, gs=gs, ref=ref)
    for x in (g, gr, gs):
        x.free()


SCHEDULES = {
    "streamed-w1": dict(order="cyclic", window=1, slots=4),
    "streamed-w4": dict(order="cyclic", window=4, slots=5),
    "zigzag": dict(order="zigzag", window=1, slots=3),
    "resident": dict(order="cyclic", window=1, slots=48),
}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("which", ["g", "gr"])
@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc", "pagerank"])
def test_stream_packed_results(r14, sched, which, algo):
    g = r14["gs"] if algo == "cc" else r14[which]
    kw = dict(SCHEDULES[sched])
    use_w = algo == "sssp"
    budget = plain_budget(g, kw["slots"], use_w)
    pvu = "weak" if algo == "pagerank" else "strong"
    base, sb = seraph.run(g, algo, source=3, columns="plain", pvu=pvu, budget_bytes=budget, **kw)
    got, st = seraph.run(g, algo, source=3, columns="plain", pvu=pvu, budget_bytes=budget,
                         stream_packed=1, **kw)
    assert st["converged"] == 1
    if algo == "pagerank":
        l1, rel = pr_errors(got, r14["ref"]["pr"])
        assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel)
    else:
        assert np.array_equal(got, r14["ref"][algo]) and np.array_equal(base, got)
    # fewer bytes over the link for the same loads (every chunk once per
    # sweep, or once in all)
    if st["sweeps"] == sb["sweeps"] and sched in ("streamed-w4", "resident"):
        assert st["bytes_streamed"] < sb["bytes_streamed"]


def test_stream_packed_with_hybrid_pages(r14):
    g = r14["gr"]
    budget = plain_budget(g, 12, True, per_slot=1.2)
    for algo in ("sssp", "pagerank"):
        got, st = seraph.run(g, algo, source=3, columns="hybrid", window=1, slots=12,
                             budget_bytes=budget, stream_packed=1,
                             pvu="strong" if algo == "sssp" else "weak")
        if algo == "pagerank":
            l1, rel = pr_errors(got, r14["ref"]["pr"])
            assert l1 <= PR_L1 and rel <= PR_REL
        else:
            assert np.array_equal(got, r14["ref"]["sssp"])


@pytest.mark.parametrize("wmax,width", [(1000, 2), (70000, 4)])
def test_stream_packed_weight_widths(wmax, width):
    src, dst, w = graphs.random_graph(3000, 40000, seed=wmax, wmax=wmax)
    g = seraph.Graph.from_edges(3000, src, dst, w, num_pages=9, compress=True)
    assert g.info()["weight_width"] == width
    og = oracle_graph(3000, src, dst, w)
    for window in (1, 2):
        got, st = seraph.run(g, "sssp", source=1, window=window, columns="plain", stream_packed=1,
                             budget_bytes=plain_budget(g, window + 1, True, 1.3))
        assert st["resident"] == 0
        assert np.array_equal(got, oracle.sssp(og, 1))
    g.free()


def test_stream_packed_hubs_and_tiny_graphs():
    # a star: the centre's in-list is long (warp decode), the leaves' short
    for n, (src, dst, w) in ((3000, graphs.star_graph(3000, center=7)),
                             (5, graphs.random_graph(5, 12, seed=1)),
                             (200, graphs.path_graph(200, w=9))):
        g = seraph.Graph.from_edges(n, src, dst, w, num_pages=3, compress=True)
        og = oracle_graph(n, src, dst, w)
        for algo in ("sssp", "bfs"):
            got, _ = seraph.run(g, algo, source=1, window=1, columns="plain", stream_packed=1,
                                budget_bytes=plain_budget(g, 2, algo == "sssp", 1.1))
            ref = oracle.sssp(og, 1) if algo == "sssp" else oracle.bfs(og, 1)
            assert np.array_equal(got, ref), (n, algo)
        g.free()


def test_stream_compact_escapes_at_tile_boundaries():
    """In-degrees and code byte counts on both sides of the one-byte limit
    (254, 255, 256 and beyond; long codes push the byte count over it at
    in-degrees below 255), placed on the vertices around each 256-vertex
    checkpoint of pages whose last tile is partial."""
    rng = np.random.default_rng(7)
    n = 40000  # gaps of ~200 between a vertex's sources: mostly 2-byte codes
    deg = np.zeros(n, np.int64)
    for b in range(0, n, 256):
        for off, d in ((-2, 254), (-1, 255), (0, 256), (1, 600), (2, 0), (3, 1), (5, 200)):
            if 0 <= b + off < n:
                deg[b + off] = d
    rest = deg == 0
    deg[rest] = rng.integers(0, 4, rest.sum())
    dst = np.repeat(np.arange(n, dtype=np.int64), deg)
    src = np.concatenate([rng.choice(n, d, replace=False) for d in deg if d > 0])
    keep = src != dst
    src, dst = src[keep].astype(np.uint32), dst[keep].astype(np.uint32)
    w = (rng.integers(1, 256, len(src))).astype(np.uint32)
    og = oracle_graph(n, src, dst, w)
    # in-degrees 200 and 254 (no escape by in-degree) take more than 254 code bytes
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=3, compress=True)
    for algo in ("sssp", "bfs"):
        for src_v in (0, 1, 30001):
            got, st = seraph.run(g, algo, source=src_v, window=1, slots=2, columns="plain",
                                 stream_packed=1, budget_bytes=plain_budget(g, 2, algo == "sssp", 1.2))
            assert st["resident"] == 0
            ref = oracle.sssp(og, src_v) if algo == "sssp" else oracle.bfs(og, src_v)
            assert np.array_equal(got, ref), (algo, src_v)
    g.free()


def test_stream_packed_falls_back_without_room_and_needs_packed_pages(r14):
    g = r14["g"]
    i = g.info()
    # one page of plain bytes per slot: no room for the packed staging
    tight = 3 * ((i["max_page_struct_bytes"] + 255) // 256 * 256 + i["max_page_weight_bytes"] + 256)
    got, st = seraph.run(g, "sssp", source=3, window=1, slots=3, columns="plain",
                         budget_bytes=tight, stream_packed=1)
    assert np.array_equal(got, r14["ref"]["sssp"])
    n, src, dst, w = rmat(10)
    plain = seraph.Graph.from_edges(n, src, dst, w, num_pages=4)
    with pytest.raises(seraph.SeraphError) as ei:
        seraph.run(plain, "sssp", budget_bytes=1 << 24, stream_packed=1)
    assert ei.value.code == C.SERAPH_EINVAL
    plain.free()
