"""The streamed benchmark workload at full size -- R-MAT-28 (2^28 vertices,
4.29 G raw edges), 512 pages, a 16 GB edge budget, the benchmark's schedules
and graph build -- checked without a full-size oracle run:

- SSSP with the oracle's shortest-path certificate over the raw generator
  stream, in chunks: every raw edge satisfies the triangle inequality and
  every reached vertex other than the source has a tight in-edge, which
  fixes the exact distances.
- PageRank by properties of its fixpoint that hold at any size: unit sum,
  every value at least the teleport term (1-d)/n, and the same fixpoint
  (within the PageRank tolerances) as the paper's plain update on the same
  graph -- no unit-sum scaling, no over-relaxation, no prediction.
- PageRank against FP64 by the oracle's step certificate: one FP64 map
  application T(x) of the library's result x, assembled from the raw
  generator stream (destinations in hash classes, duplicates dropped per
  class, kept out-degrees from a first round).  T is a d-contraction in L1,
  so ||x - x*||_1 <= ||T(x) - x||_1 / (1 - d), which must be <= 1e-5 for the
  compensated and the plain FP32 sums alike."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SCALE = 28
BUDGET = 16 << 30


@pytest.fixture(scope="module")
def g28():
    import torch
    import bench
    torch.cuda.set_device(0)
    g = bench.build_graph(seraph, synth, torch, SCALE, 512, reorder=True, compress=True)
    yield g
    g.free()


def test_sssp_rmat28_bench_schedule_certificate(g28):
    import bench
    n = 1 << SCALE
    dist, st = seraph.run(g28, "sssp", source=0, budget_bytes=BUDGET,
                          **bench.parse_sched(bench.DEFAULT_SSSP))
    assert st["converged"] == 1 and st["resident"] == 1
    tight = np.zeros(n, np.uint8)
    m = synth.rmat_config(SCALE).m
    step = 1 << 28
    bad = 0
    for e0 in range(0, m, step):
        src, dst = synth.rmat_edges(SCALE, e0=e0, count=min(step, m - e0))
        bad += oracle.sp_check_edges(src, dst, synth.weights(src, dst), dist, tight)
    bad += oracle.sp_check_tight(0, dist, tight)
    assert bad == 0
    assert dist[0] == 0 and int((dist != 0xFFFFFFFF).sum()) > n // 4


def test_pagerank_rmat28_bench_schedule_fixpoint_properties(g28):
    import bench
    n = 1 << SCALE
    d = 0.85
    x, st = seraph.run(g28, "pagerank", budget_bytes=BUDGET,
                       **bench.parse_sched(bench.DEFAULT_PAGERANK))
    assert st["converged"] == 1 and st["residual"] < 1e-7
    xd = x.astype(np.float64)
    assert abs(xd.sum() - 1.0) < 1e-5
    assert float(xd.min()) >= (1.0 - d) / n * (1.0 - 1e-5)
    plain = dict(order="zigzag", window=1, slots=14, pvu="off", columns="hybrid",
                 pr_normalize=0, pr_omega=1.0)
    y, st2 = seraph.run(g28, "pagerank", budget_bytes=BUDGET, **plain)
    assert st2["converged"] == 1 and st2["sweeps"] > st["sweeps"]
    yd = y.astype(np.float64)
    l1 = float(np.abs(xd - yd).sum())
    rel = float(np.max(np.abs(xd - yd) / yd))
    assert l1 <= 1e-5 and rel <= 1e-4, (l1, rel)


def _host_mem_gb() -> float:
    for line in open("/proc/meminfo"):
        if line.startswith("MemAvailable:"):
            return int(line.split()[1]) / (1 << 20)
    return 0.0


def test_pagerank_rmat28_bench_schedule_fp64_step_certificate(g28):
    """The benchmark's PageRank (compensated sums) and the same schedule with
    plain FP32 sums, certified in FP64 over all 4.29 G raw edges."""
    import torch
    import bench
    n = 1 << SCALE
    d = 0.85
    kw = bench.parse_sched(bench.DEFAULT_PAGERANK)
    xs = []
    for kahan in (1, 0):
        x, st = seraph.run(g28, "pagerank", budget_bytes=BUDGET, kahan=kahan, **kw)
        assert st["converged"] == 1
        xs.append(x.astype(np.float64))
    g28.release_buffers()
    X = np.stack(xs)
    del xs
    m = synth.rmat_config(SCALE).m
    step = 1 << 27
    dsrc = torch.empty(step, dtype=torch.int32, device="cuda")
    ddst = torch.empty_like(dsrc)
    hsrc = torch.empty(step, dtype=torch.int32, pin_memory=True)
    hdst = torch.empty(step, dtype=torch.int32, pin_memory=True)

    def chunks():
        # the raw generator stream (the seeded input module), chunk by chunk
        for e0 in range(0, m, step):
            c = min(step, m - e0)
            synth.rmat_edges_device(SCALE, dsrc.data_ptr(), ddst.data_ptr(), None, e0=e0, count=c)
            hsrc[:c].copy_(dsrc[:c])
            hdst[:c].copy_(ddst[:c])
            yield hsrc[:c].numpy().view(np.uint32), hdst[:c].numpy().view(np.uint32)

    nb = 8 if _host_mem_gb() > 64 else 16
    Y, E = oracle.pagerank_step_edges(n, chunks, X, d=d, nbuckets=nb, m_hint=m)
    assert E == g28.info()["m"]
    for kahan, x, y in zip((1, 0), X, Y):
        r = float(np.abs(y - x).sum())
        rel = float(np.max(np.abs(y - x) / x))
        print(f"\nPAGERANK_CERT scale=28 kahan={kahan} step_l1={r:.3e} "
              f"l1_bound={r / (1 - d):.3e} max_rel_step={rel:.3e}")
        assert r / (1 - d) <= 1e-5, (kahan, r)
        assert rel <= 1e-4, (kahan, rel)
