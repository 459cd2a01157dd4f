"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (partitioner output, SSSP distances, BFS levels, CC labels)
must be bit-exact; PageRank must be within L1 <= 1e-5 and per-vertex relative
error <= 1e-4 of the FP64 oracle.  Sizes span several pages, chunks and
ring slots with ragged tails; schedules cover the sliding window, the
double-buffer variant, forced streaming and every prediction mode.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import SeraphError
from tests import graphs

pytestmark = pytest.mark.gpu

PR_L1, PR_REL = 1e-5, 1e-4


def rmat(scale, ef=16, weighted=True):
    src, dst = synth.rmat_edges(scale, ef)
    w = synth.weights(src, dst) if weighted else None
    return 1 << scale, src, dst, w


def oracle_graph(n, src, dst, w=None, symmetrize=False):
    if symmetrize:
        src, dst, w = oracle.symmetrize(src, dst, w)
    return oracle.build_csr(n, src, dst, w)


def slot_bytes(g, use_w=True):
    i = g.info()
    return ((i["max_page_struct_bytes"] + 255) // 256) * 256 + (i["max_page_weight_bytes"] if use_w else 0)


def budget(g, window, pages_per_slot=1.0, use_w=True):
    return int((window + 1) * slot_bytes(g, use_w) * pages_per_slot) + 256 * (window + 1)


def pr_errors(x, ref):
    x = x.astype(np.float64)
    return np.abs(x - ref).sum(), np.max(np.abs(x - ref) / ref)


# ------------------------------------------------------------ partitioner

PART_CASES = [
    ("rmat12-P1", lambda: rmat(12), 1, False),
    ("rmat12-P7", lambda: rmat(12), 7, False),
    ("rmat14-sym-P16", lambda: rmat(14, weighted=False), 16, True),
    ("random-P64", lambda: (300,) + graphs.random_graph(300, 5000, seed=5), 64, False),
    ("tiny-P16", lambda: (5,) + graphs.random_graph(5, 12, seed=1), 16, False),
    ("noedges", lambda: (9, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32)), 3, False),
]


@pytest.mark.parametrize("name,make,P,sym", PART_CASES, ids=[c[0] for c in PART_CASES])
def test_partitioner_matches_oracle(name, make, P, sym):
    n, src, dst, w = make()
    g = seraph.Graph.from_edges(n, src, dst, w, symmetrize=sym, num_pages=P)
    col_off, row, wc, od = g.export_csc()
    og = oracle_graph(n, src, dst, w, symmetrize=sym)
    ocol_off, orow, ow = oracle.csc(og)
    assert g.info()["m"] == og.m
    assert np.array_equal(col_off, ocol_off)
    assert np.array_equal(row, orow)
    if w is not None:
        assert np.array_equal(wc, ow)
    assert np.array_equal(od, og.out_degree().astype(np.uint32))
    assert np.array_equal(g.page_bounds(), oracle.page_cut(n, ocol_off, P))
    assert g.info()["max_in_degree"] == int(np.diff(ocol_off).max(initial=0))


@pytest.mark.parametrize("wmax,width", [(255, 1), (1000, 2), (70000, 4)])
def test_weight_width_and_sssp(wmax, width):
    """Weights are stored in the narrowest lossless width; SSSP reads each."""
    src, dst, w = graphs.random_graph(3000, 40000, seed=wmax, wmax=wmax)
    g = seraph.Graph.from_edges(3000, src, dst, w, num_pages=9)
    assert g.info()["weight_width"] == width
    og = oracle_graph(3000, src, dst, w)
    _, _, wc, _ = g.export_csc()
    assert np.array_equal(wc, oracle.csc(og)[2])
    for window, mx in ((2, 0), (3, 5)):
        got, st = seraph.run(g, "sssp", source=1, window=window, max_passes=mx,
                             budget_bytes=budget(g, window, 1.3))
        assert st["resident"] == 0
        assert np.array_equal(got, oracle.sssp(og, 1))


def test_partitioner_device_input_and_csr_input():
    import torch
    n, src, dst, w = rmat(12)
    og = oracle_graph(n, src, dst, w)
    ref = oracle.csc(og)
    gd = seraph.Graph.from_edges(n, torch.from_numpy(src.view(np.int32)).cuda(),
                                 torch.from_numpy(dst.view(np.int32)).cuda(),
                                 torch.from_numpy(w.view(np.int32)).cuda(), num_pages=5)
    gc = seraph.Graph.from_csr(n, og.row_off, og.col, og.w, num_pages=5)
    for g in (gd, gc):
        col_off, row, wc, _ = g.export_csc()
        assert np.array_equal(col_off, ref[0]) and np.array_equal(row, ref[1])
        assert np.array_equal(wc, ref[2])


def test_device_generator_matches_host_generator():
    import torch
    cfg = synth.rmat_config(13)
    src_h, dst_h = synth.rmat_edges(13)
    w_h = synth.weights(src_h, dst_h)
    s = torch.empty(cfg.m, dtype=torch.int32, device="cuda")
    d = torch.empty_like(s)
    w = torch.empty_like(s)
    synth.rmat_edges_device(13, s.data_ptr(), d.data_ptr(), w.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(s.cpu().numpy().view(np.uint32), src_h)
    assert np.array_equal(d.cpu().numpy().view(np.uint32), dst_h)
    assert np.array_equal(w.cpu().numpy().view(np.uint32), w_h)


# ------------------------------------------------------------ algorithms

@pytest.fixture(scope="module")
def r16():
    """RMAT-16, EF16, 4 pages: the small plain-method configuration."""
    n, src, dst, w = rmat(16)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=4)
    gs = seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, num_pages=4)
    og = oracle_graph(n, src, dst, w)
    return dict(n=n, g=g, gs=gs, og=og, sssp=oracle.sssp(og, 0), bfs=oracle.bfs(og, 0),
                cc=oracle.cc(og), pr=oracle.pagerank(og)[0])


def cfg1(g, use_w=True):
    # 4 pages, one page per ring slot, window of 3 resident pages: every
    # page gets 3 local iterations per sweep.
    return dict(window=3, passes=1, budget_bytes=budget(g, 3, 1.0, use_w))


def test_rmat16_sssp(r16):
    d, st = seraph.run(r16["g"], "sssp", source=0, **cfg1(r16["g"]))
    assert np.array_equal(d, r16["sssp"])
    assert st["converged"] == 1 and st["chunks"] == 4


def test_rmat16_bfs(r16):
    d, _ = seraph.run(r16["g"], "bfs", source=0, **cfg1(r16["g"], False))
    assert np.array_equal(d, r16["bfs"])


def test_rmat16_cc(r16):
    lab, _ = seraph.run(r16["gs"], "cc", **cfg1(r16["gs"], False))
    assert np.array_equal(lab, r16["cc"])


@pytest.mark.parametrize("kahan", [1, 0])
def test_rmat16_pagerank(r16, kahan):
    x, st = seraph.run(r16["g"], "pagerank", kahan=kahan, **cfg1(r16["g"], False))
    l1, rel = pr_errors(x, r16["pr"])
    assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel, st)
    assert st["converged"] == 1 and st["residual"] < 1e-7


@pytest.mark.parametrize("pr_normalize", [0, 1])
def test_rmat16_pagerank_mass_scaling(r16, pr_normalize):
    """Scaling x back to unit sum at sweep ends leaves the fixpoint (which sums
    to 1) in place and removes the slow mode of the lagged dangling mass: on
    R-MAT (about 40 % dangling vertices) far fewer sweeps reach the same
    tolerance."""
    x, st = seraph.run(r16["g"], "pagerank", pr_normalize=pr_normalize, **cfg1(r16["g"], False))
    l1, rel = pr_errors(x, r16["pr"])
    assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel, st)
    assert st["converged"] == 1 and st["residual"] < 1e-7
    assert abs(float(x.astype(np.float64).sum()) - 1.0) < 1e-5
    if pr_normalize:
        _, st0 = seraph.run(r16["g"], "pagerank", pr_normalize=0, **cfg1(r16["g"], False))
        assert st["sweeps"] * 3 <= st0["sweeps"] * 2, (st["sweeps"], st0["sweeps"])


@pytest.mark.parametrize("omega", [1.15, 1.3])
def test_rmat16_pagerank_over_relaxed(r16, omega):
    """Over-relaxed steps (x + omega (x_new - x) while the sweep change is above
    pr_pvu_off_below, plain updates after) reach the same fixpoint."""
    x, st = seraph.run(r16["g"], "pagerank", pr_omega=omega, **cfg1(r16["g"], False))
    l1, rel = pr_errors(x, r16["pr"])
    assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel, st)
    assert st["converged"] == 1 and st["residual"] < 1e-7
    if omega == 1.15:
        _, st1 = seraph.run(r16["g"], "pagerank", **cfg1(r16["g"], False))
        assert st["sweeps"] <= st1["sweeps"], (st["sweeps"], st1["sweeps"])


def test_pagerank_over_relaxation_out_of_range_is_rejected(r16):
    for omega in (2.0, -0.5):
        with pytest.raises(SeraphError, match="EINVAL"):
            seraph.run(r16["g"], "pagerank", pr_omega=omega, **cfg1(r16["g"], False))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1027, 4099])
def test_pagerank_ragged_vertex_counts(n):
    """Vertex counts that are not a multiple of four take the close kernels'
    element-wise tail; a chain plus random edges with dangling vertices."""
    rng = np.random.default_rng(n)
    m = 4 * n
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    keep = src % 7 != 3  # vertices with id % 7 == 3 keep no out-edge (dangling)
    src, dst = src[keep], dst[keep]
    og = oracle_graph(n, src, dst, None)
    ref = oracle.pagerank(og)[0]
    g = seraph.Graph.from_edges(n, src, dst, None, num_pages=min(3, n))
    for nm in (0, 1):
        x, st = seraph.run(g, "pagerank", pr_normalize=nm, window=1, budget_bytes=1 << 20)
        l1, rel = pr_errors(x, ref)
        assert l1 <= PR_L1 and rel <= PR_REL, (n, nm, l1, rel, st)


def test_idle_passes_only_while_a_copy_is_in_flight(r16):
    """Idle-slot passes (Sec. 3.2) run only while the next chunk's copy is
    pending: once every chunk is resident (after the first sweep) a step runs
    its base passes only, so the later sweeps run exactly one pass per chunk."""
    g = r16["g"]
    kw = dict(window=1, slots=8, passes=1, pvu="off", budget_bytes=8 * (slot_bytes(g, False) + 256))
    x, st = seraph.run(g, "pagerank", max_passes=6, **kw)
    assert st["resident"] == 1 and st["converged"] == 1
    C, S = st["chunks"], st["sweeps"]
    later = (S - 1) * C                       # steps after the first sweep: one pass each
    assert C + later <= st["passes_run"] + st["passes_skipped"] <= 6 * C + later, st
    l1, rel = pr_errors(x, r16["pr"])
    assert l1 <= PR_L1 and rel <= PR_REL
    d, st2 = seraph.run(g, "sssp", source=0, max_passes=6,
                        **dict(kw, budget_bytes=8 * (slot_bytes(g, True) + 512)))
    assert st2["resident"] == 1 and np.array_equal(d, r16["sssp"])
    assert st2["passes_run"] + st2["passes_skipped"] <= 6 * st2["chunks"] + (st2["sweeps"] - 1) * st2["chunks"]


def test_pagerank_is_deterministic(r16):
    a, _ = seraph.run(r16["g"], "pagerank", **cfg1(r16["g"], False))
    b, _ = seraph.run(r16["g"], "pagerank", **cfg1(r16["g"], False))
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


SCHEDULES = [
    dict(window=1, passes=3),                       # double-buffer variant
    dict(window=2, passes=1),
    dict(window=3, passes=1, order="zigzag"),
    dict(window=2, passes=1, order="zigzag", max_passes=6),
    dict(window=4, passes=1, order="cyclic", max_passes=4, pvu="weak"),
    dict(window=3, passes=2, order="zigzag", pvu="strong"),
    dict(window=1, passes=1, order="zigzag", slots=7),
    dict(window=2, passes=1, order="cyclic", slots=9, max_passes=3),
    dict(window=4, passes=2),
    dict(window=3, passes=1, pvu="strong"),
    dict(window=3, passes=1, pvu="weak"),
    dict(window=2, passes=4, pvu="weak"),
    dict(window=1, passes=1, thread_max_deg=0, group4_max_deg=0, group8_max_deg=0,
         warp_max_deg=0),                                              # every vertex on a CTA
    dict(window=2, passes=1, thread_max_deg=4096, group4_max_deg=4096, group8_max_deg=4096,
         warp_max_deg=4096),                                           # every vertex on a thread
    dict(window=2, passes=1, thread_max_deg=0, group4_max_deg=0, group8_max_deg=0,
         warp_max_deg=1 << 30),                                        # every vertex on a warp
    dict(window=2, passes=1, thread_max_deg=0, group4_max_deg=1 << 30, group8_max_deg=1 << 30,
         warp_max_deg=1 << 30),                                        # every vertex on 4 lanes
    dict(window=2, passes=1, thread_max_deg=0, group4_max_deg=0, group8_max_deg=1 << 30,
         warp_max_deg=1 << 30),                                        # every vertex on 8 lanes
]


@pytest.fixture(scope="module")
def r13_paged():
    """RMAT-13 in 48 pages; budgets below force re-streaming every sweep."""
    n, src, dst, w = rmat(13)
    og = oracle_graph(n, src, dst, w)
    return dict(n=n, g=seraph.Graph.from_edges(n, src, dst, w, num_pages=48),
                gs=seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, num_pages=48),
                og=og, sssp=oracle.sssp(og, 5), bfs=oracle.bfs(og, 5), cc=oracle.cc(og),
                pr=oracle.pagerank(og)[0])


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc"])
def test_schedule_invariance_streamed(r13_paged, algo, sched):
    g = r13_paged["gs"] if algo == "cc" else r13_paged["g"]
    kw = dict(sched)
    nslot = kw.get("slots", kw["window"] + 1)
    kw["budget_bytes"] = budget(g, nslot - 1, 1.7, algo == "sssp")
    got, st = seraph.run(g, algo, source=5, **kw)
    assert st["resident"] == 0 and st["chunks"] > nslot
    assert np.array_equal(got, r13_paged[algo])
    if kw.get("pvu") in ("strong", "weak"):
        assert st["verify_sweeps"] >= 1


@pytest.mark.parametrize("sched", SCHEDULES[:8], ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_pagerank_streamed(r13_paged, sched):
    g = r13_paged["g"]
    kw = dict(sched)
    kw["budget_bytes"] = budget(g, kw.get("slots", kw["window"] + 1) - 1, 1.7, False)
    if kw.get("pvu") == "strong":
        with pytest.raises(SeraphError):
            seraph.run(g, "pagerank", **kw)
        return
    x, st = seraph.run(g, "pagerank", **kw)
    l1, rel = pr_errors(x, r13_paged["pr"])
    assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel, st)


STRONG_ALONE = [dict(window=2), dict(window=1, slots=32), dict(window=1, slots=7, order="zigzag"),
                dict(window=3, passes=2, order="zigzag"), dict(window=1, slots=6, max_passes=4)]


@pytest.mark.parametrize("sched", STRONG_ALONE, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc"])
def test_strong_prediction_alone_is_exact(r13_paged, algo, sched):
    """Strong conditions of Table 1 (as read for asynchronous sweeps) without
    the final prediction-off sweep still give the exact fixpoint, in every
    schedule that processes every chunk in every sweep."""
    g = r13_paged["gs"] if algo == "cc" else r13_paged["g"]
    kw = dict(sched)
    kw["budget_bytes"] = budget(g, kw.get("slots", kw["window"] + 1) - 1, 1.7, algo == "sssp")
    got, st = seraph.run(g, algo, source=5, pvu="strong", verify=0, **kw)
    assert np.array_equal(got, r13_paged[algo])
    assert st["vertices_skipped"] > 0


# ------------------------------------------------------- adversarial shapes

def run_all_min(n, src, dst, w, P, window=2, source=0, pages_per_slot=1.0):
    og = oracle_graph(n, src, dst, w)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=P)
    gs = seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, num_pages=P)
    for algo, gg, ref in (("sssp", g, oracle.sssp(og, source)), ("bfs", g, oracle.bfs(og, source)),
                          ("cc", gs, oracle.cc(og))):
        for pvu in ("off", "strong", "weak"):
            got, _ = seraph.run(gg, algo, source=source, window=window, pvu=pvu,
                                budget_bytes=budget(gg, window, pages_per_slot, algo == "sssp"))
            assert np.array_equal(got, ref), (algo, pvu)
    x, _ = seraph.run(g, "pagerank", window=window, budget_bytes=budget(g, window, pages_per_slot, False))
    l1, rel = pr_errors(x, oracle.pagerank(og)[0])
    assert l1 <= PR_L1 and rel <= PR_REL


def test_path_forward():
    run_all_min(400, *graphs.path_graph(400, w=7), P=8)


def test_path_reverse_worst_order():
    run_all_min(300, *graphs.reverse_path_graph(300, w=3), P=6, source=299)


def test_star_with_hub_larger_than_other_pages():
    run_all_min(5000, *graphs.star_graph(5000, center=17), P=8)


def test_more_pages_than_vertices():
    run_all_min(5, *graphs.random_graph(5, 14, seed=3), P=16, window=3)


def test_isolated_vertices_and_max_weights():
    src, dst, _ = graphs.random_graph(10, 40, seed=4)
    w = np.full(len(src), 255, np.uint32)
    run_all_min(2000, src, dst, w, P=4)


def test_single_vertex_no_edges():
    e = np.zeros(0, np.uint32)
    run_all_min(1, e, e, e, P=1)


def test_hub_page_over_budget_is_rejected():
    src, dst, w = graphs.star_graph(5000, center=0)
    g = seraph.Graph.from_edges(5000, src, dst, w, num_pages=8)
    with pytest.raises(SeraphError, match="EBUDGET"):
        seraph.run(g, "sssp", window=2, budget_bytes=3 * 4096)


def test_sssp_overflow_is_reported():
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 3], np.uint32)
    w = np.array([0xFFFFFF00, 0xFF, 0x10], np.uint32)
    g = seraph.Graph.from_edges(4, src, dst, w, num_pages=2)
    with pytest.raises(SeraphError, match="EOVERFLOW"):
        seraph.run(g, "sssp", window=1)


def test_invalid_arguments():
    src, dst, w = graphs.random_graph(10, 30, seed=2)
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.Graph.from_edges(5, src, dst, w, num_pages=2)   # ids >= n
    g = seraph.Graph.from_edges(10, src, dst, w, num_pages=2)
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.run(g, "sssp", source=10)
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.run(g, "pagerank", pvu="strong")
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.run(g, "sssp", window=17)


def test_output_to_device_tensor(r16):
    import torch
    out = torch.empty(r16["n"], dtype=torch.int32, device="cuda")
    seraph.run(r16["g"], "sssp", out=out, **cfg1(r16["g"]))
    assert np.array_equal(out.cpu().numpy().view(np.uint32), r16["sssp"])


def test_runs_reuse_and_release_kept_buffers(r16):
    """Consecutive runs on one graph borrow the buffers the previous run kept
    (different algorithms and ring sizes in turn); releasing them between runs
    changes nothing in the results."""
    g = r16["g"]
    for k in range(2):
        d, _ = seraph.run(g, "sssp", **cfg1(g))
        x, _ = seraph.run(g, "pagerank", window=1, slots=3, budget_bytes=budget(g, 2, 1.0, False))
        b, _ = seraph.run(g, "bfs", window=2, pvu="weak", budget_bytes=budget(g, 2, 1.0, False))
        assert np.array_equal(d, r16["sssp"]) and np.array_equal(b, r16["bfs"])
        assert pr_errors(x, r16["pr"])[0] <= PR_L1
        if k == 0:
            g.release_buffers()
