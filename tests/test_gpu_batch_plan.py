"""Prepared batches (seraph_batch_plan_*): planned once, run many times.
Every run is bit-exact against the oracle -- with the sources given at
creation, with new sources (including repeated ones), for several mappings
and tile sizes, grouped or one record per query, captured or not -- and
back-to-back runs reuse the plan's device memory; bad arguments are rejected
before anything runs."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def work():
    import torch
    torch.cuda.set_device(0)
    specs, qspecs = synth.batch_workload(n_graphs=4, n_queries=32, min_scale=9, max_scale=12)
    graphs, ogs, queries, pools = [], [], [], []
    for i, sp in enumerate(specs):
        n = 1 << sp["scale"]
        src, dst = synth.rmat_edges(sp["scale"], sp["edge_factor"], sp["abcd"], sp["seed"])
        w = synth.weights(src, dst)
        graphs.append(seraph.BGraph(n, src, dst, w))
        ogs.append(oracle.build_csr(n, src, dst, w))
        pool = synth.pick_sources(n, synth.has_out_edge(n, src, dst), 64, seed=300 + i)
        pools.append(pool)
        it = iter(pool)
        for q in qspecs:
            if q["graph"] == i:
                queries.append((i, q["algo"], next(it)))
    yield graphs, ogs, queries, pools
    for g in graphs:
        g.free()


def ref(ogs, g, algo, s):
    return oracle.bfs(ogs[g], s) if algo == "bfs" else oracle.sssp(ogs[g], s)


CASES = [dict(mapping="cta", tile=256), dict(mapping="thread", tile=1), dict(mapping="warp", tile=64),
         dict(mapping="cta", tile=256, group=0), dict(mapping="cta", tile=64, use_graph=0),
         dict(mapping="auto")]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()))
def test_plan_runs_bit_exact_with_new_sources(work, kw):
    import torch
    graphs, ogs, queries, pools = work
    outs = [torch.empty(graphs[g].n, dtype=torch.int32, device="cuda") for g, _, _ in queries]
    plan = seraph.BatchPlan(graphs, queries, outs, **kw)
    rng = np.random.default_rng(5)
    for it in range(4):
        if it == 0:
            srcs = [s for _, _, s in queries]
            st = plan.run()
        else:
            # new sources from each graph's pool; the last run repeats one
            # source across a graph's queries (groups then hold duplicates)
            srcs = [int(pools[g][0] if it == 3 else rng.choice(pools[g])) for g, _, _ in queries]
            st = plan.run(srcs)
        assert st["tune_ms"] == 0
        for (g, algo, _), s, o in zip(queries, srcs, outs):
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref(ogs, g, algo, s)), (kw, it, g, algo, s)
    plan.free()


def test_plan_reuses_its_memory_and_rejects_bad_input(work):
    import torch
    graphs, ogs, queries, pools = work
    outs = [torch.empty(graphs[g].n, dtype=torch.int32, device="cuda") for g, _, _ in queries]
    plan = seraph.BatchPlan(graphs, queries, outs, mapping="cta", tile=256)
    plan.run()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pinned0 = seraph.debug_pinned_bytes()
    srcs = [int(pools[g][1]) for g, _, _ in queries]
    for _ in range(3):
        plan.run(srcs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and seraph.debug_pinned_bytes() == pinned0
    for (g, algo, _), s, o in zip(queries, srcs, outs):
        assert np.array_equal(o.cpu().numpy().view(np.uint32), ref(ogs, g, algo, s))
    bad = list(srcs)
    bad[0] = graphs[queries[0][0]].n
    with pytest.raises(seraph.SeraphError) as ei:
        plan.run(bad)
    assert ei.value.code == C.SERAPH_EINVAL
    # nothing ran: the outputs still hold the last run
    g, algo, _ = queries[0]
    assert np.array_equal(outs[0].cpu().numpy().view(np.uint32), ref(ogs, g, algo, srcs[0]))
    with pytest.raises(ValueError):
        plan.run(srcs[:-1])
    plan.free()
    with pytest.raises(ValueError):
        seraph.BatchPlan(graphs, queries, [o.cpu() for o in outs])
