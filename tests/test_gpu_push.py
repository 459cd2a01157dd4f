"""The dense -> sparse switch with a GPU push stage (Sec. 3.1, heterogeneous
execution model), against the oracle.

- The out-edge CSR that SERAPH_OUT_EDGES keeps in pinned memory is the
  oracle's CSR (bit-exact; in internal ids for reordered graphs).
- SSSP, BFS and CC with the push stage are bit-exact against Dijkstra, FIFO
  BFS and union-find across schedules (sliding window, double buffer, forced
  streaming, resident, zigzag), prediction modes (off, strong; weak switches
  only after its prediction-off sweep), page forms (plain, packed), vertex
  orders and switch thresholds -- including a switch right after the first
  sweep, when the frontier is most of the graph and holds the hubs that the
  whole grid walks.
- An SSSP candidate that overflows during the push stage ends in the same
  SERAPH_EOVERFLOW as without it.
- It runs under the learned schedule too (every chunk still processed after
  the switch point's sweeps), bit-exact.
- Misuse is rejected (PageRank, a graph without out-edges, CC on a directed
  graph)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C
from tests import graphs

pytestmark = pytest.mark.gpu


def slot_bytes(g, use_w=True, packed=False):
    i = g.info()
    s = i["max_page_packed_bytes"] if packed else i["max_page_struct_bytes"]
    return (s + 255) // 256 * 256 + (i["max_page_weight_bytes"] if use_w else 0)


@pytest.fixture(scope="module")
def r15():
    import torch
    torch.cuda.set_device(0)
    n = 1 << 15
    src, dst = synth.rmat_edges(15)
    w = synth.weights(src, dst)
    og = oracle.build_csr(n, src, dst, w)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=24, out_edges=True)
    gr = seraph.Graph.from_edges(n, src, dst, w, num_pages=24, out_edges=True, reorder=True,
                                 compress=True)
    gs = seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, num_pages=24, out_edges=True)
    has_out = synth.has_out_edge(n, src, dst)
    srcs = synth.pick_sources(n, has_out, 3)
    ref = {("sssp", s): oracle.sssp(og, s) for s in [0] + srcs}
    ref.update({("bfs", s): oracle.bfs(og, s) for s in [0] + srcs})
    ref["cc"] = oracle.cc_edges(n, src, dst)
    yield dict(n=n, src=src, dst=dst, w=w, og=og, g=g, gr=gr, gs=gs, srcs=srcs, ref=ref)
    for x in (g, gr, gs):
        x.free()


def test_out_edge_csr_matches_oracle(r15):
    og = r15["og"]
    off, col, w = r15["g"].export_out_edges()
    assert np.array_equal(off, og.row_off) and np.array_equal(col, og.col)
    assert np.array_equal(w, og.w)
    # reordered: the same graph renamed by the library's permutation
    gr = r15["gr"]
    ogr = oracle.relabel(og, gr.perm())
    off, col, w = gr.export_out_edges()
    assert np.array_equal(off, ogr.row_off) and np.array_equal(col, ogr.col)
    assert np.array_equal(w, ogr.w)
    assert gr.info()["out_edge_bytes"] == 8 * (og.n + 1) + 5 * og.m


SCHEDULES = {
    "window4-off": dict(order="cyclic", window=4, slots=5, pvu="off"),
    "window4-strong": dict(order="cyclic", window=4, slots=5, pvu="strong", verify=0),
    "double-buffer-k3": dict(order="cyclic", window=1, slots=2, passes=3, pvu="strong"),
    "zigzag-weak": dict(order="zigzag", window=1, slots=4, pvu="weak"),
    "resident-strong": dict(order="cyclic", window=1, slots=32, pvu="strong", verify=0),
}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("below", [1 << 30, 64, 0])
def test_sssp_bfs_with_push_bit_exact(r15, sched, below):
    g, ref = r15["g"], r15["ref"]
    kw = dict(SCHEDULES[sched])
    resident = kw.pop("slots") == 32
    switched = 0
    for algo in ("sssp", "bfs"):
        use_w = algo == "sssp"
        slots = 32 if resident else SCHEDULES[sched]["slots"]
        budget = slots * slot_bytes(g, use_w) * (1.0 if resident else 1.3) + 256 * slots
        for s in [0] + r15["srcs"][:1]:
            got, st = seraph.run(g, algo, source=s, slots=slots, budget_bytes=int(budget), push=1,
                                 push_below=below, **kw)
            assert st["converged"] == 1
            assert np.array_equal(got, ref[(algo, s)]), (algo, s, sched, below)
            if st["push_sweep"]:
                switched += 1
                assert st["push_rounds"] >= 1  # (its frontier may hold sinks only)
    if below == 1 << 30 and kw["pvu"] != "weak":
        assert switched == 4  # a threshold above n switches after the first valid sweep


def test_push_after_the_first_sweep_walks_hubs_with_the_whole_grid(r15):
    """A switch after sweep 1 starts from most of the graph, hubs included
    (out-degree above the one-warp limit of 2048 on R-MAT-15)."""
    g, ref = r15["g"], r15["ref"]
    og = r15["og"]
    assert int(og.out_degree().max()) > 2048
    got, st = seraph.run(g, "sssp", source=0, window=1, slots=32, pvu="off",
                         budget_bytes=32 * (slot_bytes(g) + 256), push=1, push_below=1 << 30)
    assert st["push_sweep"] == 1 and st["sweeps"] == 1
    assert np.array_equal(got, ref[("sssp", 0)])


def test_push_on_reordered_packed_pages(r15):
    gr, ref = r15["gr"], r15["ref"]
    for algo in ("sssp", "bfs"):
        for below in (1 << 30, 100):
            got, st = seraph.run(gr, algo, source=0, window=1, slots=6, pvu="strong", verify=0,
                                 columns="packed",
                                 budget_bytes=6 * (slot_bytes(gr, algo == "sssp", True) + 256),
                                 push=1, push_below=below)
            assert np.array_equal(got, ref[(algo, 0)]), (algo, below)


@pytest.mark.parametrize("below", [1 << 30, 16])
def test_cc_with_push_bit_exact(r15, below):
    gs = r15["gs"]
    for kw in (dict(window=4, slots=5, pvu="off"), dict(window=1, slots=3, pvu="strong", verify=0)):
        got, st = seraph.run(gs, "cc", budget_bytes=int(kw["slots"] * (slot_bytes(gs, False) * 1.3 + 256)),
                             push=1, push_below=below, **kw)
        assert np.array_equal(got, r15["ref"]["cc"]), (kw, below)


def test_push_small_graphs_and_edge_cases():
    cases = [
        ("path", 200) + graphs.path_graph(200, w=7),
        ("reverse-path", 200) + graphs.reverse_path_graph(200, w=3),
        ("random-dups", 300) + graphs.random_graph(300, 4000, seed=11),
        ("star", 500) + graphs.star_graph(500, center=3),
    ]
    for name, n, src, dst, w in cases:
        og = oracle.build_csr(n, src, dst, w)
        g = seraph.Graph.from_edges(n, src, dst, w, num_pages=5, out_edges=True)
        for s in (0, 3, n - 1):
            got, st = seraph.run(g, "sssp", source=s, window=2, slots=3, pvu="off",
                                 budget_bytes=3 * slot_bytes(g) + 4096, push=1, push_below=1 << 30)
            assert np.array_equal(got, oracle.sssp(og, s)), (name, s)
        g.free()
    # no edges at all: nothing changes, so the switch never happens
    g = seraph.Graph.from_edges(9, np.zeros(0, np.uint32), np.zeros(0, np.uint32), None,
                                num_pages=3, out_edges=True)
    got, st = seraph.run(g, "bfs", source=4, window=1, slots=2, budget_bytes=1 << 16, push=1)
    assert got[4] == 0 and (np.delete(got, 4) == seraph.INF).all() and st["push_sweep"] == 0
    g.free()


def test_push_overflow_is_reported_like_the_pull_path():
    # 0 -> 1 -> 2 with weights 2^31 (distance 2^32 does not fit), plus a
    # branch that keeps the push stage busy for a few rounds
    src = np.array([0, 1, 0, 3, 4], np.uint32)
    dst = np.array([1, 2, 3, 4, 5], np.uint32)
    w = np.array([1 << 31, 1 << 31, 1, 1, 1], np.uint32)
    with pytest.raises(oracle.OverflowError_):
        oracle.sssp(oracle.build_csr(6, src, dst, w), 0)
    g = seraph.Graph.from_edges(6, src, dst, w, num_pages=2, out_edges=True)
    for push in (0, 1):
        with pytest.raises(seraph.SeraphError) as ei:
            seraph.run(g, "sssp", source=0, window=1, slots=2, budget_bytes=1 << 16, push=push,
                       push_below=1 << 30)
        assert ei.value.code == C.SERAPH_EOVERFLOW
    g.free()


def test_push_misuse_is_rejected(r15):
    g, gs = r15["g"], r15["gs"]
    n, src, dst = r15["n"], r15["src"], r15["dst"]
    plain = seraph.Graph.from_edges(n, src, dst, None, num_pages=4)
    bad = [(g, "pagerank", {}), (plain, "bfs", {}), (g, "cc", {})]
    for gg, algo, kw in bad:
        with pytest.raises(seraph.SeraphError) as ei:
            seraph.run(gg, algo, budget_bytes=1 << 24, push=1, **kw)
        assert ei.value.code == C.SERAPH_EINVAL, (algo, kw)
    plain.free()


def test_push_under_the_learned_schedule(r15):
    g, ref = r15["g"], r15["ref"]
    from paper_1806_00762_b300 import train_sched
    model = seraph.SchedModel()
    params = train_sched.load()
    if params is not None:
        model.set_params(params)
    for verify, pvu in ((0, "strong"), (1, "strong"), (1, "off")):
        got, st = seraph.run(g, "sssp", source=0, window=1, slots=6, pvu=pvu, verify=verify,
                             budget_bytes=6 * (slot_bytes(g) + 256), sched_model=model, max_passes=4,
                             push=1, push_below=2000)
        assert np.array_equal(got, ref[("sssp", 0)]), (verify, pvu)
