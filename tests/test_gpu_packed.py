"""Packed page columns (SERAPH_COMPRESS: LEB128 gaps of each destination's
sources): the streams are byte-exact against the oracle's encoding, and every
algorithm decodes them to the same results as the plain pages -- bit-exact
for SSSP/BFS/CC, within tolerance for PageRank -- on every lane mapping
(thread, 4 lanes, 8 lanes, warp, CTA), with codes of 1 to 5 bytes."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import SeraphError
from tests import graphs
from tests.test_gpu_parity import PR_L1, PR_REL, budget, oracle_graph, pr_errors, rmat

pytestmark = pytest.mark.gpu

PART_CASES = [
    ("rmat12-P7", lambda: rmat(12), 7, False, False),
    ("rmat12-P7-reorder", lambda: rmat(12), 7, False, True),
    ("rmat14-sym-P16-reorder", lambda: rmat(14, weighted=False), 16, True, True),
    ("random-P64", lambda: (300,) + graphs.random_graph(300, 5000, seed=5), 64, False, False),
    ("tiny-P16", lambda: (5,) + graphs.random_graph(5, 12, seed=1), 16, False, False),
    ("noedges", lambda: (9, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32)), 3, False, False),
]


def packed_budget(g, slots, use_w=True, per_slot=1.7):
    i = g.info()
    slot = (i["max_page_packed_bytes"] + 255) // 256 * 256 + (i["max_page_weight_bytes"] if use_w else 0)
    return int(slots * slot * per_slot) + 256 * slots


@pytest.mark.parametrize("name,make,P,sym,reorder", PART_CASES, ids=[c[0] for c in PART_CASES])
def test_packed_streams_match_oracle(name, make, P, sym, reorder):
    n, src, dst, w = make()
    g = seraph.Graph.from_edges(n, src, dst, w, symmetrize=sym, num_pages=P, reorder=reorder,
                                compress=True)
    og = oracle_graph(n, src, dst, w, symmetrize=sym)
    if reorder:
        og = oracle.relabel(og, oracle.degree_order(og))
    ocol_off, orow, _ = oracle.csc(og)
    oboff, odata = oracle.pack_gaps(ocol_off, orow)
    info = g.info()
    assert info["packed"] == 1 and info["packed_data_bytes"] == len(odata)
    boff, data = g.export_packed()
    assert np.array_equal(boff, oboff)
    assert np.array_equal(data, odata)
    col_off, row, _, _ = g.export_csc()      # the plain pages are kept as well
    assert np.array_equal(row, orow)


@pytest.fixture(scope="module")
def r13p():
    n, src, dst, w = rmat(13)
    og = oracle_graph(n, src, dst, w)
    ogs = oracle_graph(n, src, dst, None, symmetrize=True)
    mk = dict(num_pages=48, compress=True)
    return dict(n=n, g=seraph.Graph.from_edges(n, src, dst, w, **mk),
                gr=seraph.Graph.from_edges(n, src, dst, w, reorder=True, **mk),
                gs=seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, reorder=True, **mk),
                sssp=oracle.sssp(og, 5), bfs=oracle.bfs(og, 5), cc=oracle.cc(ogs),
                pr=oracle.pagerank(og)[0])


BIG = 1 << 30
MAPPINGS = {
    "thread": dict(thread_max_deg=BIG, group4_max_deg=BIG, group8_max_deg=BIG, warp_max_deg=BIG),
    "lanes4": dict(thread_max_deg=0, group4_max_deg=BIG, group8_max_deg=BIG, warp_max_deg=BIG),
    "lanes8": dict(thread_max_deg=0, group4_max_deg=0, group8_max_deg=BIG, warp_max_deg=BIG),
    "warp": dict(thread_max_deg=0, group4_max_deg=0, group8_max_deg=0, warp_max_deg=BIG),
    "cta": dict(thread_max_deg=0, group4_max_deg=0, group8_max_deg=0, warp_max_deg=0),
    "default": dict(),
}


@pytest.mark.parametrize("mapping", list(MAPPINGS))
@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc", "pagerank"])
@pytest.mark.parametrize("which", ["g", "gr"])
def test_packed_results_every_mapping(r13p, algo, mapping, which):
    g = r13p["gs"] if algo == "cc" else r13p[which]
    kw = dict(MAPPINGS[mapping], window=2, columns="packed",
              budget_bytes=packed_budget(g, 3, algo == "sssp"))
    got, st = seraph.run(g, algo, source=5, **kw)
    assert st["converged"] == 1 and st["resident"] == 0
    if algo == "pagerank":
        l1, rel = pr_errors(got, r13p["pr"])
        assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel)
    else:
        assert np.array_equal(got, r13p[algo])


SCHEDULES = [
    dict(window=1, order="cyclic", slots=32, pvu="strong", verify=0),
    dict(window=1, order="zigzag", slots=32, pvu="weak"),
    dict(window=3, passes=2, order="zigzag", max_passes=4),
]


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc", "pagerank"])
def test_packed_schedules_match_plain(r13p, algo, sched):
    g = r13p["gs"] if algo == "cc" else r13p["gr"]
    kw = dict(sched)
    if algo == "pagerank" and kw.get("pvu") == "strong":
        kw.update(pvu="weak", verify=1)
    nslot = kw.get("slots", kw["window"] + 1)
    a, sa = seraph.run(g, algo, source=5, columns="packed",
                       budget_bytes=packed_budget(g, nslot, algo == "sssp", 1.2), **kw)
    b, sb = seraph.run(g, algo, source=5, columns="plain",
                       budget_bytes=budget(g, nslot - 1, 1.2, algo == "sssp"), **kw)
    assert sa["bytes_streamed"] < sb["bytes_streamed"]
    if algo == "pagerank":
        assert pr_errors(a, r13p["pr"])[0] <= PR_L1 and pr_errors(b, r13p["pr"])[0] <= PR_L1
    else:
        assert np.array_equal(a, r13p[algo]) and np.array_equal(b, r13p[algo])


def test_packed_form_needs_compressed_graph():
    n, src, dst, w = rmat(9)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=3)
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.run(g, "sssp", columns="packed", budget_bytes=budget(g, 2, 1.7))
    with pytest.raises(SeraphError, match="EINVAL"):
        g.export_packed()


def test_five_byte_codes_and_hub_lists():
    """Ids at and above 2^28 need 5-byte codes; one destination with 5000
    sources (CTA mapping) and sources spread over the whole id range."""
    n = (1 << 28) + 4096
    rng = np.random.default_rng(11)
    hi = rng.integers((1 << 28) - 4096, n, size=6000, dtype=np.int64)
    lo = rng.integers(0, n, size=6000, dtype=np.int64)
    hub = np.full(5000, n - 1, dtype=np.int64)
    src = np.concatenate([hi, lo, rng.integers(0, n, 5000)]).astype(np.uint32)
    dst = np.concatenate([lo, hi, hub]).astype(np.uint32)
    w = synth.weights(src, dst)
    src = np.concatenate([src, np.array([7], np.uint32)])
    dst = np.concatenate([dst, src[:1]])
    w = np.concatenate([w, np.array([3], np.uint32)])
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=8, compress=True)
    og = oracle_graph(n, src, dst, w)
    ocol_off, orow, _ = oracle.csc(og)
    oboff, odata = oracle.pack_gaps(ocol_off, orow)
    boff, data = g.export_packed()
    assert np.array_equal(data, odata) and np.array_equal(boff, oboff)
    assert (odata[oboff[:-1][np.diff(oboff) > 0]] & 0x80).any()
    s = int(src[0])
    d, _ = seraph.run(g, "sssp", source=s, window=2, columns="packed",
                      budget_bytes=packed_budget(g, 3))
    assert np.array_equal(d, oracle.sssp(og, s))


@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc", "pagerank"])
def test_hybrid_forms_keep_every_chunk_resident(r13p, algo):
    """columns="hybrid" packs the fewest leading pages with which every chunk
    fits the ring: with a budget between the plain and the packed totals the
    plain form must stream every sweep, the hybrid one stays resident, and both
    give the oracle's results."""
    g = r13p["gs"] if algo == "cc" else r13p["gr"]
    i = g.info()
    use_w = algo == "sssp"
    wb = i["weight_bytes"] if use_w else 0
    budget = int(((i["struct_bytes"] + i["packed_bytes"]) / 2 + wb) * 1.25)
    kw = dict(source=5, window=1, slots=12, budget_bytes=budget)
    if algo == "pagerank":
        kw["pvu"] = "weak"
    h, sh = seraph.run(g, algo, columns="hybrid", **kw)
    p, sp = seraph.run(g, algo, columns="plain", **kw)
    assert sh["resident"] == 1 and sp["resident"] == 0
    assert sh["bytes_streamed"] < sp["bytes_streamed"]
    for got in (h, p):
        if algo == "pagerank":
            l1, rel = pr_errors(got, r13p["pr"])
            assert l1 <= PR_L1 and rel <= PR_REL
        else:
            assert np.array_equal(got, r13p[algo])


def test_hybrid_needs_window_one(r13p):
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.run(r13p["gr"], "bfs", columns="hybrid", window=2,
                   budget_bytes=packed_budget(r13p["gr"], 3, False))


def test_hybrid_packs_pages_too_big_for_a_plain_slot():
    """A hub page whose plain form exceeds a slot while its packed form fits
    (its in-list is 1-byte gaps): the plain form is refused (SERAPH_EBUDGET),
    the hybrid form packs the leading pages and runs.  (Pages of many small
    in-lists can be larger packed than plain: the byte offsets cost 4 bytes
    per vertex, which is why only leading pages are packed.)"""
    n = 4096
    rng = np.random.default_rng(2)
    src = np.concatenate([np.arange(1, n), rng.integers(0, n, 3000)]).astype(np.uint32)
    dst = np.concatenate([np.zeros(n - 1), rng.integers(1, n, 3000)]).astype(np.uint32)
    w = synth.weights(src, dst)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=6, compress=True)
    og = oracle_graph(n, src, dst, w)
    col_off, _, _ = oracle.csc(og)
    i = g.info()
    pages = g.page_bounds()
    first_plain = 4 * (int(pages[1]) + 1) + 4 * int(col_off[pages[1]])
    assert first_plain > 12000
    kw = dict(source=1, window=1, slots=8, budget_bytes=8 * 12288)
    with pytest.raises(SeraphError, match="EBUDGET"):
        seraph.run(g, "bfs", columns="plain", **kw)
    got, _ = seraph.run(g, "bfs", columns="hybrid", **kw)
    assert np.array_equal(got, oracle.bfs(og, 1))
    d, _ = seraph.run(g, "sssp", columns="hybrid", source=1, window=1, slots=8,
                      budget_bytes=8 * (12288 + (i["max_page_weight_bytes"] + 255) // 256 * 256))
    assert np.array_equal(d, oracle.sssp(og, 1))
