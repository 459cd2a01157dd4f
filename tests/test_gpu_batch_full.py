"""The batched workload at full size (16 graphs, scales 14-22, 256 queries)
in the launch configuration bench.py times (autotuned mapping, CUDA graph),
checked query by query with the oracle's shortest-path certificate over the
raw edge stream (triangle inequality on every edge + a tight in-edge for every
reached vertex, which pins the exact distances) on a sample of queries."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_batch_workload_full_size_sampled_certificates():
    import torch
    import bench
    graphs, queries, _, specs = bench.build_batch(seraph, synth, torch)
    outs = [torch.empty(graphs[g].n, dtype=torch.int32, device="cuda") for g, _, _ in queries]
    _, st = seraph.batch_run(graphs, queries, outs=outs, mapping="auto")
    assert st["graph_captured"] == 1
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(queries), 24, replace=False))
    by_graph = {}
    for i in sample:
        by_graph.setdefault(queries[i][0], []).append(i)
    for g, idx in by_graph.items():
        sp = specs[g]
        src, dst = synth.rmat_edges(sp["scale"], sp["edge_factor"], sp["abcd"], sp["seed"])
        w = synth.weights(src, dst)
        for i in idx:
            _, algo, s = queries[i]
            dist = outs[i].cpu().numpy().view(np.uint32)
            tight = np.zeros(len(dist), np.uint8)
            bad = oracle.sp_check_edges(src, dst, w if algo == "sssp" else None, dist, tight)
            bad += oracle.sp_check_tight(s, dist, tight)
            assert bad == 0, (g, algo, s)
