"""Runs on one graph from several host threads at once: the first to start
borrows the graph's kept buffers, the others allocate their own, each run
has its own streams, and every result is exact (SSSP, BFS and CC against the
oracle, PageRank within the stated tolerance); afterwards the graph's kept
buffers and the L2 set-aside are still consistent for a normal run."""
import threading

import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from tests.test_gpu_parity import PR_L1, PR_REL, pr_errors

pytestmark = pytest.mark.gpu


def test_concurrent_runs_on_one_graph():
    import torch
    torch.cuda.set_device(0)
    n = 1 << 14
    src, dst = synth.rmat_edges(14)
    w = synth.weights(src, dst)
    og = oracle.build_csr(n, src, dst, w)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=12, reorder=True, compress=True,
                                out_edges=True)
    srcs = synth.pick_sources(n, synth.has_out_edge(n, src, dst), 3)
    jobs = [("sssp", s) for s in srcs] + [("bfs", s) for s in srcs] + [("pagerank", 0)]
    results, errors = {}, []

    def work(i, algo, s):
        try:
            torch.cuda.set_device(0)
            kw = dict(window=1, slots=4, budget_bytes=1 << 21, columns="hybrid", stream_packed=1)
            if algo != "pagerank":
                kw.update(source=s, push=1, pvu="strong")
            else:
                kw.update(pvu="weak", pr_omega=1.15)
            for _ in range(3):
                results[i] = seraph.run(g, algo, **kw)[0]
        except Exception as e:  # reported below, in the main thread
            errors.append((algo, s, repr(e)))

    threads = [threading.Thread(target=work, args=(i, a, s)) for i, (a, s) in enumerate(jobs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, (algo, s) in enumerate(jobs):
        if algo == "sssp":
            assert np.array_equal(results[i], oracle.sssp(og, s)), (algo, s)
        elif algo == "bfs":
            assert np.array_equal(results[i], oracle.bfs(og, s)), (algo, s)
        else:
            l1, rel = pr_errors(results[i], oracle.pagerank(og)[0])
            assert l1 <= PR_L1 and rel <= PR_REL, (l1, rel)
    d, _ = seraph.run(g, "sssp", source=srcs[0], budget_bytes=1 << 21)
    assert np.array_equal(d, oracle.sssp(og, srcs[0]))
    g.free()
