"""PageRank in the benchmark's exact configuration against the FP64 oracle.

The graph is built the way the benchmark builds its R-MAT-28 graph -- raw
R-MAT edges generated on the device, vertices renumbered by out-degree
(SERAPH_REORDER), every page kept both plain and packed (SERAPH_COMPRESS),
512 destination-range pages -- and PageRank runs with the benchmark's own
schedule string (cyclic order, one chunk per step, 14 ring slots, weak
prediction, hybrid page forms, unit-sum scaling at sweep ends, steps
over-relaxed by 1.15).  The edge budget is the benchmark's 16 GB scaled by the
vertex count (2^(scale-28)), so the pages of a chunk and the packed share stay
close to the full-size run's.  Both summations (compensated and plain FP32)
are compared with oracle.pagerank (FP64 power iteration to an L1 change below
1e-15) on the host copy of the same generator's edges: L1 <= 1e-5 and
per-vertex relative error <= 1e-4 (the PageRank tolerance of the parity
tests).  The errors are printed (run with -s to see them)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = pytest.mark.gpu

PR_L1, PR_REL = 1e-5, 1e-4


@pytest.fixture(scope="module", params=[20, 22])
def bench_graph(request):
    import torch
    import bench
    torch.cuda.set_device(0)
    scale = request.param
    g = bench.build_graph(seraph, synth, torch, scale, 512, reorder=True, compress=True)
    src, dst = synth.rmat_edges(scale)
    ref, _, _ = oracle.pagerank(oracle.build_csr(1 << scale, src, dst))
    del src, dst
    yield scale, g, ref
    g.free()


@pytest.mark.parametrize("kahan", [1, 0])
def test_bench_pagerank_schedule_matches_fp64_oracle(bench_graph, kahan):
    import bench
    scale, g, ref = bench_graph
    budget = int(16 * (1 << 30) * 2.0 ** (scale - 28))
    kw = bench.parse_sched(bench.DEFAULT_PAGERANK)
    x, st = seraph.run(g, "pagerank", budget_bytes=budget, kahan=kahan, **kw)
    assert st["converged"] == 1 and st["residual"] < 1e-7
    assert st["resident"] == 1  # as at full size: every chunk stays in the ring
    xd = x.astype(np.float64)
    l1 = float(np.abs(xd - ref).sum())
    rel = float(np.max(np.abs(xd - ref) / ref))
    print(f"\nPAGERANK_ERROR scale={scale} kahan={kahan} l1={l1:.3e} max_rel={rel:.3e} "
          f"sweeps={st['sweeps']} chunks={st['chunks']}")
    assert l1 <= PR_L1 and rel <= PR_REL, (scale, kahan, l1, rel)


def test_bench_pagerank_schedule_streams_packed_and_plain_pages(bench_graph):
    """The hybrid form really mixes the two page forms at this budget (fewer
    bytes streamed than all-plain, more than all-packed)."""
    import bench
    scale, g, _ = bench_graph
    budget = int(16 * (1 << 30) * 2.0 ** (scale - 28))
    kw = dict(bench.parse_sched(bench.DEFAULT_PAGERANK), stream_packed=0)  # page forms as stored
    _, hy = seraph.run(g, "pagerank", budget_bytes=budget, max_sweeps=1, **kw)
    _, pk = seraph.run(g, "pagerank", budget_bytes=budget, max_sweeps=1, **dict(kw, columns="packed"))
    _, pl = seraph.run(g, "pagerank", budget_bytes=budget, max_sweeps=1, **dict(kw, columns="plain"))
    assert pk["bytes_streamed"] < hy["bytes_streamed"] < pl["bytes_streamed"]
