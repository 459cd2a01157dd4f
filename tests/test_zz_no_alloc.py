"""The no-allocation pull fixpoint, called through the C ABI.

seraph_pull_fixpoint_noalloc serves callers that cannot call cudaMalloc
(device memory owned by a framework's allocator or planner, or a serving loop
where allocation would synchronise the device).  It must give the same
distances / levels / labels as seraph_run on the same graph and as the
oracle (Dijkstra, FIFO BFS, union-find), on two calls in a row (its static
scratch keeps the previous call's contents, which each call must clear),
report an SSSP distance that does not fit below 2^32-1 as the oracle does,
reject a CSC whose source ids reach n before reading through it, and reject
graphs larger than its static scratch.

This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C

pytestmark = pytest.mark.gpu


def _budget(g, window, use_w):
    i = g.info()
    slot = (i["max_page_struct_bytes"] + 255) // 256 * 256 + (i["max_page_weight_bytes"] if use_w else 0)
    return (window + 1) * slot + 4096


def _device_csc(g):
    import torch
    col_off, row, w, _ = g.export_csc()
    d_off = torch.from_numpy(col_off.view(np.int64).copy()).cuda()
    d_row = torch.from_numpy(row.view(np.int32).copy()).cuda()
    d_w = None if w is None else torch.from_numpy(w.view(np.int32).copy()).cuda()
    return d_off, d_row, d_w


def _call(algo, n, d_off, d_row, d_w, source, out):
    passes = ctypes.c_uint32(0)
    rc = C.lib().seraph_pull_fixpoint_noalloc(algo, n, d_off.data_ptr(), d_row.data_ptr(),
                                              None if d_w is None else d_w.data_ptr(), source,
                                              out.data_ptr(), ctypes.byref(passes), None)
    return rc, passes.value


@pytest.fixture(scope="module")
def rmat15():
    n = 1 << 15
    src, dst = synth.rmat_edges(15)
    w = synth.weights(src, dst)
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=4)
    gs = seraph.Graph.from_edges(n, src, dst, None, symmetrize=True, num_pages=4)
    og = oracle.build_csr(n, src, dst, w)
    want = {"sssp": oracle.sssp(og, 3), "bfs": oracle.bfs(og, 3), "cc": oracle.cc_edges(n, src, dst)}
    return n, g, gs, want


@pytest.mark.parametrize("algo", ["sssp", "bfs", "cc"])
def test_noalloc_matches_seraph_run_and_oracle_twice(rmat15, algo):
    import torch
    n, g, gs, want = rmat15
    gg = gs if algo == "cc" else g
    ref, _ = seraph.run(gg, algo, source=3, window=3, budget_bytes=_budget(gg, 3, algo == "sssp"))
    assert np.array_equal(ref, want[algo])
    d_off, d_row, d_w = _device_csc(gg)
    if algo != "sssp":
        d_w = None
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out.fill_(0x5A5A5A5A)
        rc, passes = _call(C.ALGOS[algo], n, d_off, d_row, d_w, 3, out)
        assert rc == C.SERAPH_OK, C.lib().seraph_last_error()
        assert passes >= 1
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref) and np.array_equal(got, want[algo])


def _tiny_csc(col_off, row, w=None):
    import torch
    d_off = torch.tensor(col_off, dtype=torch.int64, device="cuda")
    d_row = torch.tensor(row, dtype=torch.int32, device="cuda")
    d_w = None if w is None else torch.tensor(np.array(w, dtype=np.uint32).view(np.int32),
                                              device="cuda")
    return d_off, d_row, d_w


def test_noalloc_reports_sssp_overflow_like_the_oracle():
    """Path 0 -> 1 -> 2 with weights 2^31: vertex 2's distance 2^32 does not
    fit below 2^32-1."""
    import torch
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 2], np.uint32)
    w = np.array([1 << 31, 1 << 31], np.uint32)
    with pytest.raises(oracle.OverflowError_):
        oracle.sssp(oracle.build_csr(3, src, dst, w), 0)
    d_off, d_row, d_w = _tiny_csc([0, 0, 1, 2], [0, 1], [1 << 31, 1 << 31])
    out = torch.empty(3, dtype=torch.int32, device="cuda")
    for _ in range(2):
        rc, _ = _call(C.SSSP, 3, d_off, d_row, d_w, 0, out)
        assert rc == C.SERAPH_EOVERFLOW
    # the next call without the overflow is exact (the flag is cleared)
    d_off, d_row, d_w = _tiny_csc([0, 0, 1, 2], [0, 1], [5, 7])
    rc, _ = _call(C.SSSP, 3, d_off, d_row, d_w, 0, out)
    assert rc == C.SERAPH_OK
    assert out.cpu().numpy().tolist() == [0, 5, 12]


def test_noalloc_rejects_a_bad_csc_before_reading_through_it():
    import torch
    out = torch.full((4,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    bad = [([0, 1, 2, 3, 3], [1, 2, 4]),      # source id == n
           ([0, 2, 1, 3, 3], [1, 2, 0]),      # offsets decrease
           ([1, 1, 2, 3, 3], [1, 2, 0])]      # offsets do not start at 0
    for col_off, row in bad:
        d_off, d_row, _ = _tiny_csc(col_off, row)
        rc, _ = _call(C.BFS, 4, d_off, d_row, None, 0, out)
        assert rc == C.SERAPH_EINVAL
        assert C.lib().seraph_last_error()
        assert (out.cpu().numpy() == 0x5A5A5A5A).all()   # values untouched
    d_off, d_row, _ = _tiny_csc([0, 1, 2, 3, 3], [1, 2, 0])
    rc, _ = _call(C.BFS, 4, d_off, d_row, None, 0, out)
    assert rc == C.SERAPH_OK
    # in-edges 1 -> 0, 2 -> 1, 0 -> 2; vertex 3 has none
    og = oracle.build_csr(4, np.array([1, 2, 0], np.uint32), np.array([0, 1, 2], np.uint32))
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.bfs(og, 0))


def test_noalloc_rejects_graphs_beyond_its_scratch():
    import torch
    n = C.NOALLOC_MAX_VERTICES + 1
    d_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    passes = ctypes.c_uint32(0)
    rc = C.lib().seraph_pull_fixpoint_noalloc(C.SSSP, n, d_off.data_ptr(), None, None, 0,
                                              out.data_ptr(), ctypes.byref(passes), None)
    assert rc == C.SERAPH_EINVAL
    assert b"SERAPH_NOALLOC_MAX_VERTICES" in C.lib().seraph_last_error()
