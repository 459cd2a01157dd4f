"""Host logic of bench.py (no GPU): schedule strings, the algorithmic-byte
counts of the relax roofline, the pipeline roofline, and the rule that the
measured relax DRAM traffic is reported only for the kernel source and the
schedules it was captured on."""
import hashlib
import os
from types import SimpleNamespace

import pytest

import bench


def test_parse_sched_types_and_defaults():
    pr = bench.parse_sched(bench.DEFAULT_PAGERANK)
    assert pr["pvu"] == "weak" and pr["columns"] == "hybrid"
    assert isinstance(pr["slots"], int) and isinstance(pr["pr_omega"], float)
    assert pr["pr_omega"] == 1.15 and pr["pr_normalize"] == 1
    ss = bench.parse_sched(bench.DEFAULT_SSSP)
    assert ss == dict(order="cyclic", window=1, slots=16, pvu="strong", verify=0, columns="hybrid",
                      push=1, stream_packed=1)
    assert bench.parse_sched("") == {}


def test_algo_bytes_counts():
    st = dict(edges_relaxed=100, vertices_attempted=10, changes=3)
    # SSSP with 1-byte weights: 9 B per edge + 16 B per vertex + 4 B per change
    assert bench.algo_bytes("sssp", st, 1) == 9 * 100 + 16 * 10 + 4 * 3
    assert bench.algo_bytes("sssp", st, 4, weak=True) == 12 * 100 + 16 * 10 + 4 * 3 + 2 * 10
    # PageRank: 8 B per edge + 20 B per vertex
    assert bench.algo_bytes("pagerank", st) == 8 * 100 + 20 * 10
    # packed pages: their edges' column bytes are the code bytes, not 4 B each
    pk = dict(st, packed_edges=60, code_bytes=90)
    assert bench.algo_bytes("pagerank", pk) == 4 * 40 + 90 + 4 * 100 + 20 * 10
    assert bench.algo_bytes("sssp", pk, 1) == 4 * 40 + 90 + 5 * 100 + 16 * 10 + 4 * 3


def test_pipeline_roofline_takes_the_slower_side():
    r = bench.pipeline_roofline(hbm_bytes=6.5e12, link_bytes=27.5e9, seconds=2.0, hbm_gbs=6500.0,
                                link_gbs=55.0)
    assert r["bound"] == "hbm" and r["t_roof_s"] == pytest.approx(1.0)
    assert r["frac"] == pytest.approx(0.5)
    r = bench.pipeline_roofline(hbm_bytes=6.5e9, link_bytes=110e9, seconds=4.0, hbm_gbs=6500.0,
                                link_gbs=55.0)
    assert r["bound"] == "link" and r["t_link_s"] == pytest.approx(2.0)
    assert r["frac"] == pytest.approx(0.5)
    assert bench.pipeline_roofline(1.0, 1.0, 0.0, 1.0, 1.0)["frac"] == 0.0


def _args(**kw):
    a = dict(scale=28, pages=512, budget_gb=16.0, vertex_order="degree",
             sssp=bench.RELAX_TRAFFIC["sssp"], pagerank=bench.RELAX_TRAFFIC["pagerank"],
             algos="sssp,pagerank")
    a.update(kw)
    return SimpleNamespace(**a)


def test_relax_traffic_only_for_the_captured_source_and_schedules():
    h = hashlib.sha256()
    for name in bench.RELAX_SOURCES:
        h.update(open(os.path.join(bench.ROOT, "paper_1806_00762_b300", "csrc", name), "rb").read())
    got = bench.relax_traffic(_args())
    if h.hexdigest()[:16] == bench.RELAX_TRAFFIC["kernel_sha256"]:
        assert got == bench.RELAX_TRAFFIC["bytes_per_launch"]
    else:
        assert got is None
    # any other workload or schedule: no figure
    for change in (dict(scale=26), dict(pages=256), dict(budget_gb=8.0),
                   dict(vertex_order="natural"), dict(algos="pagerank"),
                   dict(pagerank=bench.RELAX_TRAFFIC["pagerank"] + ",max_passes=2"),
                   dict(sssp=bench.RELAX_TRAFFIC["sssp"].replace("slots=16", "slots=12"))):
        assert bench.relax_traffic(_args(**change)) is None, change


def test_default_schedules_are_the_captured_ones():
    """The committed traffic figure belongs to the default step."""
    assert bench.DEFAULT_SSSP == bench.RELAX_TRAFFIC["sssp"]
    assert bench.DEFAULT_PAGERANK == bench.RELAX_TRAFFIC["pagerank"]
