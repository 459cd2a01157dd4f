"""Measurement for active-page skipping (Graphie-style, Sec. 2): with
count_clean, every sweep close counts the pages none of whose in-edge
sources (grouped in 1024 blocks of consecutive ids) changed in that sweep.

Checked on a graph of two disjoint R-MAT-13 halves, SSSP from vertex 0: the
second half is unreachable and never changes, so every page whose
destinations all lie in it (its sources then do too) is clean in every
sweep, and in the final sweep (no change at all) every page is; the first
half's pages are dirty in the first sweep.  Results stay bit-exact."""
import numpy as np
import pytest

import oracle
import synth
import paper_1806_00762_b300 as seraph

pytestmark = pytest.mark.gpu


def two_halves():
    h = 1 << 13
    s1, d1 = synth.rmat_edges(13)
    s2, d2 = synth.rmat_edges(13, seed=9)
    src = np.concatenate([s1, s2 + h]).astype(np.uint32)
    dst = np.concatenate([d1, d2 + h]).astype(np.uint32)
    return 2 * h, src, dst, synth.weights(src, dst)


@pytest.mark.parametrize("algo", ["sssp", "bfs"])
def test_clean_pages_of_an_untouched_half(algo):
    import torch
    torch.cuda.set_device(0)
    n, src, dst, w = two_halves()
    P = 16
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=P)
    vb = g.page_bounds()
    second = int(((vb[:-1] >= n // 2)).sum())  # pages with every destination in the second half
    assert second >= 4
    i = g.info()
    budget = 3 * ((i["max_page_struct_bytes"] + 255) // 256 * 256 + i["max_page_weight_bytes"] + 256)
    og = oracle.build_csr(n, src, dst, w)
    ref = oracle.sssp(og, 0) if algo == "sssp" else oracle.bfs(og, 0)
    got, st = seraph.run(g, algo, source=0, window=2, slots=3, pvu="off", budget_bytes=budget,
                         count_clean=1)
    assert np.array_equal(got, ref)
    sweeps = st["sweeps"]
    assert sweeps >= 2
    # the last sweep changed nothing: all P pages clean; before it, at least
    # the second half's pages; the first sweep dirtied the first half's pages
    assert st["clean_pages"] >= P + second * (sweeps - 1)
    assert st["clean_pages"] <= P * sweeps - (P - second) // 2
    # the measurement is off by default and changes no result
    got2, st2 = seraph.run(g, algo, source=0, window=2, slots=3, pvu="off", budget_bytes=budget)
    assert np.array_equal(got2, ref) and st2["clean_pages"] == 0
    g.free()
