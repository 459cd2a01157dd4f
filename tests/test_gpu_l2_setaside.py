"""The persisting-L2 set-aside behind the evict-last hot range: a graph's
first run that keeps its hot range in L2 raises the context's limit, later
runs on the graph leave it alone (so a run calls nothing that would wait for
other work in flight in the context, such as the read-back of an earlier
run's values), and freeing the graph -- or releasing its buffers -- puts the
earlier value back.  Results are the same with and without the hint."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = pytest.mark.gpu


def test_setaside_held_per_graph_then_restored():
    import torch
    torch.cuda.set_device(0)
    n = 1 << 14
    src, dst = synth.rmat_edges(14)
    w = synth.weights(src, dst)
    og = oracle.build_csr(n, src, dst, w)
    before = seraph.debug_l2_setaside()
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=8, reorder=True)
    d1, _ = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
    raised = seraph.debug_l2_setaside()
    assert raised >= before
    d2, _ = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
    x, _ = seraph.run(g, "pagerank", budget_bytes=1 << 20)
    assert seraph.debug_l2_setaside() == raised
    d0, _ = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20, l2_hot_bytes=0)
    ref = oracle.sssp(og, 0)
    assert np.array_equal(d1, ref) and np.array_equal(d2, ref) and np.array_equal(d0, ref)
    g.release_buffers()
    assert seraph.debug_l2_setaside() == before
    seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
    assert seraph.debug_l2_setaside() == raised
    g.free()
    assert seraph.debug_l2_setaside() == before
