"""The plain method at a size that fits in HBM but is made to stream: R-MAT-24
(2^24 vertices, edge factor 16, 268 M raw edges), 64 destination-range pages
in pinned host memory, a 2 GB device edge budget, the pipelined schedule with
k = 4 local iterations per chunk (a window of 4 chunks over 5 slots, Fig. 4)
and no prediction.  Checked against the oracle:

- PageRank against the FP64 power iteration (L1 <= 1e-5, per-vertex relative
  <= 1e-4);
- SSSP from vertex 0 and BFS from 8 seeded sources by the oracle's
  shortest-path certificate over the raw edge stream (triangle inequality on
  every raw edge, a tight in-edge for every reached vertex: the exact values);
- CC on the symmetrised graph against the oracle's union-find labels
  (bit-exact).

The library stores R-MAT's weights in one byte, so at 2 GB the whole graph
fits the ring and runs resident after its first sweep; SSSP and PageRank run a
second time under a 600 MB budget, where every sweep streams."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SCALE = 24
N = 1 << SCALE
PLAIN = dict(order="cyclic", window=4, slots=5, passes=1, pvu="off")
BUDGETS = (2 << 30, 600 << 20)
PR_L1, PR_REL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def r24():
    src, dst = synth.rmat_edges(SCALE)
    w = synth.weights(src, dst)
    g = seraph.Graph.from_edges(N, src, dst, w, num_pages=64)
    yield dict(src=src, dst=dst, w=w, g=g)
    g.free()


def certificate(src, dst, w, dist, source):
    tight = np.zeros(N, np.uint8)
    bad = oracle.sp_check_edges(src, dst, w, dist, tight)
    return bad + oracle.sp_check_tight(source, dist, tight)


def test_rmat24_sssp_certificate(r24):
    for budget in BUDGETS:
        dist, st = seraph.run(r24["g"], "sssp", source=0, budget_bytes=budget, **PLAIN)
        assert st["converged"] == 1
        if budget == BUDGETS[1]:
            assert st["resident"] == 0
        assert certificate(r24["src"], r24["dst"], r24["w"], dist, 0) == 0, budget


def test_rmat24_bfs_eight_sources_certificate(r24):
    has_out = synth.has_out_edge(N, r24["src"], r24["dst"])
    for s in synth.pick_sources(N, has_out, 8):
        lvl, st = seraph.run(r24["g"], "bfs", source=s, budget_bytes=BUDGETS[0], **PLAIN)
        assert st["converged"] == 1
        assert certificate(r24["src"], r24["dst"], None, lvl, s) == 0, s


def test_rmat24_cc_against_union_find(r24):
    gs = seraph.Graph.from_edges(N, r24["src"], r24["dst"], None, symmetrize=True, num_pages=64)
    try:
        lab, st = seraph.run(gs, "cc", budget_bytes=BUDGETS[0], **PLAIN)
    finally:
        gs.free()
    assert st["converged"] == 1
    assert np.array_equal(lab, oracle.cc_edges(N, r24["src"], r24["dst"]))


def test_rmat24_pagerank_against_fp64_oracle(r24):
    og = oracle.build_csr(N, r24["src"], r24["dst"])
    ref, _, _ = oracle.pagerank(og)
    del og
    for budget in BUDGETS:
        x, st = seraph.run(r24["g"], "pagerank", budget_bytes=budget, **PLAIN)
        assert st["converged"] == 1
        xd = x.astype(np.float64)
        l1 = float(np.abs(xd - ref).sum())
        rel = float(np.max(np.abs(xd - ref) / ref))
        assert l1 <= PR_L1 and rel <= PR_REL, (budget, l1, rel, st["sweeps"])
