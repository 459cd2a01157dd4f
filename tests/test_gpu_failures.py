"""Failure paths on the GPU, each made without faulting or hanging the device:

- a bounded device wait that runs out: the batched kernel's task-ring waits
  get an iteration limit of zero (timeout_ms = 0), so the first CTA that finds
  no task yet gives up, sets the error flag, and every CTA leaves; the call
  returns SERAPH_ETIMEOUT, and the next normal call on the same graphs is
  exact;
- a failed pinned host allocation, injected on the host at each allocation
  of a graph build and of a run: SERAPH_ENOMEM, no pinned or device memory
  kept, and the next call is exact;
- CSR offsets in device memory that do not start at 0 or that decrease:
  SERAPH_EINVAL before they are used."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r14():
    import torch
    torch.cuda.set_device(0)
    n = 1 << 14
    src, dst = synth.rmat_edges(14)
    w = synth.weights(src, dst)
    return n, src, dst, w, oracle.build_csr(n, src, dst, w)


def test_batch_bounded_wait_runs_out_then_next_call_is_exact(r14):
    n, src, dst, w, og = r14
    bg = seraph.BGraph(n, src, dst, w)
    qs = [(0, "sssp", 0), (0, "bfs", 5)]
    for use_graph in (0, 1):
        with pytest.raises(seraph.SeraphError) as ei:
            seraph.batch_run([bg], qs, mapping="cta", tile=64, timeout_ms=0, use_graph=use_graph)
        assert ei.value.code == C.SERAPH_ETIMEOUT
        assert b"bounded wait" in C.lib().seraph_last_error()
        outs, _ = seraph.batch_run([bg], qs, mapping="cta", tile=64, use_graph=use_graph)
        assert np.array_equal(outs[0], oracle.sssp(og, 0))
        assert np.array_equal(outs[1], oracle.bfs(og, 5))
    bg.free()


def _free_device_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_failed_pinned_allocation_in_graph_build_returns_enomem_and_keeps_nothing(r14):
    n, src, dst, w, og = r14
    # one full build first, so lazily created driver state is not counted
    seraph.Graph.from_edges(n, src, dst, w, num_pages=8, compress=True).free()
    pinned0, free0 = seraph.debug_pinned_bytes(), _free_device_bytes()
    # the build pins page structures, weights, packed pages and the packed
    # pages' streamed headers: fail each
    for k in (1, 2, 3, 4):
        seraph.debug_fail_pinned_alloc(k)
        try:
            with pytest.raises(seraph.SeraphError) as ei:
                seraph.Graph.from_edges(n, src, dst, w, num_pages=8, compress=True)
        finally:
            seraph.debug_fail_pinned_alloc(0)
        assert ei.value.code == C.SERAPH_ENOMEM
        assert b"injected" in C.lib().seraph_last_error()
        assert seraph.debug_pinned_bytes() == pinned0
        assert _free_device_bytes() >= free0 - (8 << 20)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=8, compress=True)
    dist, _ = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20, columns="packed")
    assert np.array_equal(dist, oracle.sssp(og, 0))
    g.free()
    assert seraph.debug_pinned_bytes() == pinned0


def test_failed_pinned_allocation_in_a_run_returns_enomem_and_next_run_is_exact(r14):
    """A graph's first run pins its small read-back buffers (kept with the
    graph): failing that allocation gives SERAPH_ENOMEM and keeps nothing.
    Once a run has succeeded, later runs allocate nothing, so an armed
    failure does not touch them."""
    n, src, dst, w, og = r14
    base = seraph.debug_pinned_bytes()
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=8)
    ref = oracle.sssp(og, 0)
    pinned0 = seraph.debug_pinned_bytes()
    seraph.debug_fail_pinned_alloc(1)
    try:
        with pytest.raises(seraph.SeraphError) as ei:
            seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
    finally:
        seraph.debug_fail_pinned_alloc(0)
    assert ei.value.code == C.SERAPH_ENOMEM
    assert seraph.debug_pinned_bytes() == pinned0
    dist, st = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
    assert st["converged"] == 1 and np.array_equal(dist, ref)
    pinned1 = seraph.debug_pinned_bytes()
    seraph.debug_fail_pinned_alloc(1)
    try:
        dist, _ = seraph.run(g, "sssp", source=0, budget_bytes=1 << 20)
        x, _ = seraph.run(g, "bfs", source=0, budget_bytes=1 << 20)
    finally:
        seraph.debug_fail_pinned_alloc(0)
    assert np.array_equal(dist, ref) and np.array_equal(x, oracle.bfs(og, 0))
    assert seraph.debug_pinned_bytes() == pinned1
    g.free()
    assert seraph.debug_pinned_bytes() == base


def test_from_csr_rejects_bad_device_offsets(r14):
    import torch
    n, src, dst, w, og = r14
    ro = torch.from_numpy(og.row_off.astype(np.int64)).cuda()
    col = torch.from_numpy(og.col.astype(np.int32)).cuda()
    g = seraph.Graph.from_csr(n, ro, col, num_pages=4)
    lvl, _ = seraph.run(g, "bfs", source=0, budget_bytes=4 << 20)
    assert np.array_equal(lvl, oracle.bfs(og, 0))
    g.free()
    bad = ro.clone()
    bad[n // 2] = bad[n // 2 + 1] + 1          # decreases once
    bad0 = ro.clone()
    bad0[0] = 1                                # does not start at 0
    for b in (bad, bad0):
        with pytest.raises(seraph.SeraphError) as ei:
            seraph.Graph.from_csr(n, b, col, num_pages=4)
        assert ei.value.code == C.SERAPH_EINVAL
        assert b"non-decreasing" in C.lib().seraph_last_error()
