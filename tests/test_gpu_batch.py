"""Batched multi-query BFS/SSSP (one persistent kernel over many resident
graphs): every query bit-exact against the oracle, for every tile mapping,
tile size, with and without CUDA-graph capture, host and device outputs."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import SeraphError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def work():
    specs, qspecs = synth.batch_workload(n_graphs=6, n_queries=48, min_scale=9, max_scale=13)
    graphs, ogs, queries, refs = [], [], [], []
    for i, sp in enumerate(specs):
        n = 1 << sp["scale"]
        src, dst = synth.rmat_edges(sp["scale"], sp["edge_factor"], sp["abcd"], sp["seed"])
        w = synth.weights(src, dst)
        graphs.append(seraph.BGraph(n, src, dst, w))
        ogs.append(oracle.build_csr(n, src, dst, w))
        srcs = iter(synth.pick_sources(n, synth.has_out_edge(n, src, dst), 64, seed=100 + i))
        for q in qspecs:
            if q["graph"] == i:
                s = next(srcs)
                queries.append((i, q["algo"], s))
    for g, algo, s in queries:
        refs.append(oracle.bfs(ogs[g], s) if algo == "bfs" else oracle.sssp(ogs[g], s))
    return graphs, queries, refs


CASES = [dict(mapping="thread", tile=64), dict(mapping="warp", tile=64),
         dict(mapping="cta", tile=256), dict(mapping="thread", tile=1),
         dict(mapping="cta", tile=2048), dict(mapping="warp", tile=1024, use_graph=0),
         dict(mapping="auto")]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_batch_matches_oracle(work, kw):
    graphs, queries, refs = work
    outs, st = seraph.batch_run(graphs, queries, **kw)
    for o, r in zip(outs, refs):
        assert np.array_equal(o, r)
    assert st["edges"] > 0 and st["rounds_max"] >= 1
    if kw.get("use_graph", 1):
        assert st["graph_captured"] == 1


@pytest.mark.parametrize("delta", [1, 7, 64, 1000, 1 << 30])
@pytest.mark.parametrize("mapping", ["thread", "warp", "cta"])
def test_near_far_bucket_widths(work, delta, mapping):
    """SSSP near-far ordering: any bucket width (1 = a filter round after
    nearly every round, 2^30 = plain label-correcting rounds) gives the exact
    distances."""
    graphs, queries, refs = work
    outs, st = seraph.batch_run(graphs, queries, mapping=mapping, tile=64, delta=delta)
    for o, r in zip(outs, refs):
        assert np.array_equal(o, r)


@pytest.mark.parametrize("pull_div", [1, 2, 20, 0xFFFFFFFF])
@pytest.mark.parametrize("mapping", ["thread", "cta"])
def test_bfs_direction_switch(work, pull_div, mapping):
    """BFS rounds whose frontier exceeds n / pull_div run bottom-up (every
    unvisited vertex looks for a parent in the frontier): never (1), on large
    frontiers (2, 20) or after the first round always (2^32-1) -- the levels
    stay exact, and SSSP queries in the same batch are unaffected."""
    graphs, queries, refs = work
    outs, _ = seraph.batch_run(graphs, queries, mapping=mapping, tile=64, bfs_pull_div=pull_div)
    for o, r in zip(outs, refs):
        assert np.array_equal(o, r)


def test_autotune_result_is_cached_and_device_outputs(work):
    import torch
    graphs, queries, refs = work
    _, st1 = seraph.batch_run(graphs, queries, mapping="auto")
    outs = [torch.empty(graphs[g].n, dtype=torch.int32, device="cuda") for g, _, _ in queries]
    _, st2 = seraph.batch_run(graphs, queries, outs=outs, mapping="auto", replays=3)
    assert st2["tune_ms"] < st1["tune_ms"] + 1.0 and st2["mapping"] == st1["mapping"]
    for o, r in zip(outs, refs):
        assert np.array_equal(o.cpu().numpy().view(np.uint32), r)


def test_batch_edge_cases():
    e = np.zeros(0, np.uint32)
    g0 = seraph.BGraph(5, e, e, e)                       # no edges
    src = np.array([0, 1, 2, 2], np.uint32)
    dst = np.array([1, 2, 3, 3], np.uint32)
    w = np.array([7, 255, 1, 9], np.uint32)
    g1 = seraph.BGraph(6, src, dst, w)                   # vertex 5 isolated, a duplicate edge
    outs, _ = seraph.batch_run([g0, g1], [(0, "bfs", 3), (1, "sssp", 0), (1, "bfs", 5), (1, "sssp", 4)])
    INF = seraph.INF
    assert list(outs[0]) == [INF, INF, INF, 0, INF]
    assert list(outs[1]) == [0, 7, 262, 263, INF, INF]
    assert list(outs[2]) == [INF] * 5 + [0]
    assert list(outs[3]) == [INF, INF, INF, INF, 0, INF]


def test_batch_invalid_arguments(work):
    graphs, _, _ = work
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.batch_run(graphs, [(0, "bfs", graphs[0].n)])
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.batch_run(graphs, [(0, "cc", 0)])
    with pytest.raises(SeraphError, match="EINVAL"):
        seraph.batch_run(graphs, [(len(graphs), "bfs", 0)])


@pytest.mark.parametrize("group", [0, 1])
@pytest.mark.parametrize("kw", [dict(mapping="cta", tile=64), dict(mapping="thread", tile=32),
                                dict(mapping="cta", tile=512, delta=1),
                                dict(mapping="cta", tile=128, bfs_pull_div=0xFFFFFFFF)],
                         ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_grouped_and_single_records_agree_with_the_oracle(work, group, kw):
    """Queries of one graph and algorithm run as lockstep groups (group = 1:
    one frontier for the group, interleaved distances, a shared near-far
    split; BFS groups pulling bottom-up too) or one record each (group = 0):
    exact either way."""
    graphs, queries, refs = work
    outs, st = seraph.batch_run(graphs, queries, group=group, **kw)
    for o, r in zip(outs, refs):
        assert np.array_equal(o, r)


def test_groups_of_eight_with_duplicate_sources_and_a_remainder(work):
    """17 SSSP and 11 BFS queries on one graph: groups of 8 and remainders of
    1 and 3, several queries sharing a source (one frontier entry for all of
    them), in one launch with queries of other graphs."""
    graphs, _, _ = work
    g = 5
    n = graphs[g].n
    spec = synth.batch_workload(n_graphs=6, n_queries=48, min_scale=9, max_scale=13)[0][g]
    src, dst = synth.rmat_edges(spec["scale"], spec["edge_factor"], spec["abcd"], spec["seed"])
    w = synth.weights(src, dst)
    og = oracle.build_csr(n, src, dst, w)
    s = synth.pick_sources(n, synth.has_out_edge(n, src, dst), 12, seed=55)
    qs = [(g, "sssp", x) for x in s + s[:5]] + [(g, "bfs", x) for x in s[:8] + [s[0]] * 3]
    qs += [(0, "bfs", 0), (1, "sssp", 3)]
    outs, _ = seraph.batch_run(graphs, qs, mapping="cta", tile=64)
    for (gi, algo, x), o in zip(qs[:-2], outs):
        ref = oracle.sssp(og, x) if algo == "sssp" else oracle.bfs(og, x)
        assert np.array_equal(o, ref), (algo, x)
    single, _ = seraph.batch_run(graphs, qs[-2:], mapping="cta", tile=64, group=0)
    assert np.array_equal(outs[-2], single[0]) and np.array_equal(outs[-1], single[1])
