"""Benchmark: time-to-fixpoint and effective GTEPS of the streamed Seraph hot
path on R-MAT-28 (2^28 vertices, edge factor 16, a,b,c,d = .57,.19,.19,.05),
512 destination-range pages in pinned host memory, a 16 GB device edge-buffer
budget, vertex arrays resident in HBM, SSSP (weights in [1,255], from vertex
0) and PageRank (FP32 Kahan sums, FP64 residual, L1 < 1e-7 or 100 sweeps),
predictive vertex updating on (strong conditions for SSSP, the weak state
machine for PageRank; PageRank's values rescaled to unit sum at sweep ends
and its steps over-relaxed by 1.15 until the sweep change falls below 1e-6),
fixed (non-learned) schedules per algorithm.

Besides the timed steps, one run of each algorithm with the paper's plain
schedule -- a sliding window of k = 4 chunks over a ring of 5 slots, cyclic
order, weak prediction -- is reported as `paper_schedule` for comparison.

One step = SSSP to its fixpoint + PageRank to its stop rule.  `value` is the
effective GTEPS of the step (edges of the graph, counted once per algorithm,
over the device-measured time from the first page copy to the stop
decision).  `e2e` is the same through the public call, timed on the host
over the whole timed loop: every run streams its pages from pinned host
memory and its values are read back into pinned host memory (each read-back
overlapping the next run, whose pages travel the other way).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl seraph|reference]

Under torchrun every rank runs an independent replica (the method runs on one
GPU; there is no exchange step to shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-fixpoint and effective GTEPS, RMAT-28 streamed; learned vs fixed sched"


DEFAULT_SSSP = ("order=cyclic,window=1,slots=16,pvu=strong,verify=0,columns=hybrid,push=1,"
                "stream_packed=1")
DEFAULT_PAGERANK = ("order=cyclic,window=1,slots=14,pvu=weak,columns=hybrid,pr_normalize=1,"
                    "pr_omega=1.15,stream_packed=1")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="seraph", choices=["seraph", "reference"])
    ap.add_argument("--scale", type=int, default=28)
    ap.add_argument("--pages", type=int, default=512)
    ap.add_argument("--budget-gb", type=float, default=16.0)
    ap.add_argument("--sssp", default=DEFAULT_SSSP,
                    help="SSSP schedule: comma-separated seraph_params overrides")
    ap.add_argument("--pagerank", default=DEFAULT_PAGERANK,
                    help="PageRank schedule: comma-separated seraph_params overrides")
    ap.add_argument("--vertex-order", default="degree", choices=["degree", "natural"],
                    help="degree: vertices numbered by non-increasing out-degree before the "
                         "page cut (SERAPH_REORDER); natural: the generator's ids")
    ap.add_argument("--no-paper-schedule", action="store_true")
    ap.add_argument("--ablation", action="store_true",
                    help="also run the paper's ablation ladder (Fig. 9 style) on the same graph: "
                         "baseline, pipelined subgraph iteration, + predictive updating, + the "
                         "library's resident chunks, packed pages and PageRank accelerations")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-scheduler comparison run")
    ap.add_argument("--workload", default="streamed", choices=["streamed", "batch"],
                    help="streamed: the R-MAT-28 headline; batch: 256 BFS/SSSP queries over "
                         "16 resident R-MAT graphs (scales 14-22) in one persistent launch")
    ap.add_argument("--batch-mapping", default="auto", choices=["auto", "thread", "warp", "cta"],
                    help="batch: lane mapping of every graph (auto = the autotuner's choice)")
    ap.add_argument("--batch-tile", type=int, default=0, help="batch: tile with a fixed mapping")
    ap.add_argument("--batch-graph", type=int, default=-1,
                    help="batch: keep only the queries of this graph (profiling one graph)")
    ap.add_argument("--algos", default="sssp,pagerank",
                    help="algorithms of a step (profiling runs may use one)")
    ap.add_argument("--cpu-scale", type=int, default=22, help="R-MAT scale of the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stream-budget-gb", type=float, default=-1.0,
                    help="also run both algorithms once under this budget, too small for the "
                         "graph to become resident (-1 = half of --budget-gb; 0 = skip)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self) -> dict:
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------- setup

def link_gbps(torch, nbytes=1 << 30, reps=5, chunks=4) -> float:
    """Pinned host->device copy bandwidth: 4 x 1 GiB, best of 5."""
    h = torch.empty(chunks * nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(chunks * nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        with torch.cuda.stream(s):
            for i in range(chunks):
                d[i * nbytes:(i + 1) * nbytes].copy_(h[i * nbytes:(i + 1) * nbytes], non_blocking=True)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del h, d
    return chunks * nbytes / (best / 1e3) / 1e9


def build_graph(seraph, synth, torch, scale, pages, reorder=True, compress=True, out_edges=True):
    n = 1 << scale
    m = synth.rmat_config(scale).m
    src = torch.empty(m, dtype=torch.int32, device="cuda")
    dst = torch.empty_like(src)
    w = torch.empty_like(src)
    synth.rmat_edges_device(scale, src.data_ptr(), dst.data_ptr(), w.data_ptr())
    torch.cuda.synchronize()
    g = seraph.Graph.from_edges(n, src, dst, w, num_pages=pages, reorder=reorder, compress=compress,
                                out_edges=out_edges)
    del src, dst, w
    torch.cuda.empty_cache()
    return g


# DRAM traffic of the relax kernels per launch on this workload, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass) on six launches of
# the default step at full size -- three PageRank launches (plain columns, the
# resident sweeps) and three SSSP launches (packed columns, the resident
# sweeps) -- weighted by the step's 154 PageRank and 64 SSSP relax launches
# (profiles/relax_kernel_dram_rmat28.md); valid only for the kernel sources
# (engine.cu and leb128.cuh) and the two schedules it was taken on.
RELAX_TRAFFIC = {"kernel_sha256": "2c17ecc59c18a7bb", "bytes_per_launch": 6.4224e+09,
                 "sssp": DEFAULT_SSSP,
                 "pagerank": DEFAULT_PAGERANK,
                 "workload": "rmat28 default step"}
RELAX_SOURCES = ("engine.cu", "leb128.cuh")


def relax_traffic(args) -> float | None:
    import hashlib
    h = hashlib.sha256()
    for name in RELAX_SOURCES:
        with open(os.path.join(ROOT, "paper_1806_00762_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    default = (args.scale == 28 and args.pages == 512 and args.budget_gb == 16.0 and
               args.vertex_order == "degree" and args.sssp == RELAX_TRAFFIC["sssp"] and
               args.pagerank == RELAX_TRAFFIC["pagerank"] and args.algos == "sssp,pagerank")
    if h.hexdigest()[:16] != RELAX_TRAFFIC["kernel_sha256"] or not default:
        return None
    return RELAX_TRAFFIC["bytes_per_launch"]


def gather_ceiling(seraph) -> float:
    """Random 4-byte gathers per second when every gather hits L2: 2^29 reads
    of 2^28 values, all inside an 8 MB evict-last range (seraph_gather_probe,
    best of 5 launches).  It bounds a pull pass whose gathers all hit L2."""
    n_gathers = 1 << 29
    return n_gathers / seraph.gather_probe(1 << 28, n_gathers, (8 << 20) // 4, 1.0, reps=5)


def pipeline_roofline(hbm_bytes: float, link_bytes: float, seconds: float, hbm_gbs: float,
                      link_gbs: float) -> dict:
    """The pipeline's roofline time, the slower of its relax bytes over HBM and
    its streamed bytes over the host link (a lower bound of the per-step sum of
    the two maxima), as a fraction of the measured time."""
    t_hbm = hbm_bytes / (hbm_gbs * 1e9)
    t_link = link_bytes / (link_gbs * 1e9) if link_gbs else 0.0
    t_roof = max(t_hbm, t_link)
    return {"bound": "link" if t_link >= t_hbm else "hbm", "t_roof_s": t_roof,
            "t_hbm_s": t_hbm, "t_link_s": t_link, "frac": t_roof / seconds if seconds else 0.0}


def max_over_ranks(vals, world: int, device: str):
    """Each value's maximum over the ranks (the slowest replica times the job);
    the identity for one process."""
    if world == 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_units(units_per_rank: float, world: int) -> float:
    """Whole-job work: every rank runs an independent replica of the step."""
    return units_per_rank * world


def parse_sched(text: str) -> dict:
    out = {}
    for item in filter(None, text.split(",")):
        k, v = item.split("=")
        k, v = k.strip(), v.strip()
        out[k] = v if k in ("order", "pvu", "columns") else (float(v) if "." in v else int(v))
    return out


def algo_bytes(algo, st, weight_width=4, weak=False) -> float:
    """Algorithmic bytes of the relax kernels of a run.  Column stream: 4 B per
    edge on plain pages, the LEB128 code bytes of the edges on packed pages
    (stats code_bytes).  Then SSSP (4 + w) B/edge (stored weight of w bytes,
    gathered distance) + 16 B per attempted vertex (list entry, offset pair,
    old value) + 4 B per change; PageRank 4 B/edge (gathered contribution) +
    20 B per attempted vertex (list entry, offset pair, old value, new
    value); +2 B per attempted vertex when the weak prediction state is read
    and written."""
    E, V, ch = st["edges_relaxed"], st["vertices_attempted"], st["changes"]
    col = 4 * (E - st.get("packed_edges", 0)) + st.get("code_bytes", 0)
    extra = 2 * V if weak else 0
    if algo == "sssp":
        return col + (4 + weight_width) * E + 16 * V + 4 * ch + extra
    return col + 4 * E + 20 * V + extra


# ------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(scale, steps=1):
    """The oracle as it stands on an R-MAT sample of the same family:
    Dijkstra (1 thread) and FP64 PageRank with the same stop rule as the GPU
    (OpenMP over vertices).  Returns (GTEPS, seconds, description, threads)."""
    import oracle
    import synth
    n = 1 << scale
    src, dst = synth.rmat_edges(scale)
    w = synth.weights(src, dst)
    og = oracle.build_csr(n, src, dst, w)
    del src, dst, w
    total_t, total_e = 0.0, 0
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.sssp(og, 0)
        t1 = time.perf_counter()
        oracle.pagerank(og, tol=1e-7, maxit=100)
        t2 = time.perf_counter()
        total_t += t2 - t0
        total_e += 2 * og.m
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"RMAT-{scale} sample, not the RMAT-28 workload (same generator and shape, "
            f"{og.m} edges): oracle Dijkstra from vertex 0 (1 thread) + FP64 PageRank to "
            f"L1<1e-7 ({threads} OpenMP threads); GTEPS = edges per algorithm / time on the "
            f"sample -- an extrapolation that flatters the CPU, whose per-edge cost grows "
            f"with the graph (cache misses)")
    return total_e / total_t / 1e9, total_t, desc, threads


def pagerank_error_vs_oracle(seraph, synth, torch, scale, pages, sched_kw) -> dict:
    """PageRank error of the benchmark's schedule against the FP64 oracle, on
    the CPU sample's graph size (part of the cpu_baseline leg, which runs the
    oracle's PageRank anyway): the graph built as build_graph builds it, the
    edge budget scaled from 16 GB at 2^28 vertices, compensated and plain
    FP32 sums, each against oracle.pagerank to an L1 change < 1e-15."""
    import oracle
    n = 1 << scale
    src, dst = synth.rmat_edges(scale)
    ref, _, _ = oracle.pagerank(oracle.build_csr(n, src, dst))
    del src, dst
    g = build_graph(seraph, synth, torch, scale, pages)
    budget = int(16 * (1 << 30) * 2.0 ** (scale - 28))
    out = {"workload": f"rmat{scale}-ef16, {pages} pages, budget {budget} B, the benchmark's "
                       f"PageRank schedule", "reference": "oracle FP64 power iteration, L1 change "
                       "< 1e-15", "tolerance": {"l1": 1e-5, "max_rel": 1e-4}}
    try:
        for name, kahan in (("kahan", 1), ("plain", 0)):
            x, st = seraph.run(g, "pagerank", budget_bytes=budget, kahan=kahan, **sched_kw)
            xd = x.astype(np.float64)
            out[name] = {"l1": float(np.abs(xd - ref).sum()),
                         "max_rel": float(np.max(np.abs(xd - ref) / ref)), "sweeps": st["sweeps"]}
    finally:
        g.free()
    return out


# ------------------------------------------------------------ batch workload

def build_batch(seraph, synth, torch, seed=7):
    """The 16 graphs and 256 queries of synth.batch_workload, generated on the
    device; sources drawn over vertices with an out-edge."""
    specs, qspecs = synth.batch_workload(seed=seed)
    graphs, queries, edges_of = [], [], []
    for i, sp in enumerate(specs):
        n = 1 << sp["scale"]
        m = synth.rmat_config(sp["scale"], sp["edge_factor"], sp["abcd"], sp["seed"]).m
        src = torch.empty(m, dtype=torch.int32, device="cuda")
        dst = torch.empty_like(src)
        w = torch.empty_like(src)
        synth.rmat_edges_device(sp["scale"], src.data_ptr(), dst.data_ptr(), w.data_ptr(),
                                edge_factor=sp["edge_factor"], abcd=sp["abcd"], seed=sp["seed"])
        has_out = torch.zeros(n, dtype=torch.bool, device="cuda")
        keep = src != dst
        has_out[src[keep].long()] = True
        g = seraph.BGraph(n, src, dst, w)
        srcs = iter(synth.pick_sources(n, has_out.cpu().numpy(), 64, seed=100 + i))
        for q in qspecs:
            if q["graph"] == i:
                queries.append((i, q["algo"], next(srcs)))
        graphs.append(g)
        edges_of.append(int(keep.sum()))
        del src, dst, w, has_out, keep
    torch.cuda.empty_cache()
    return graphs, queries, edges_of, specs


def main_batch(args, world, rank):
    import torch
    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    import paper_1806_00762_b300 as seraph
    graphs, queries, edges_of, specs = build_batch(seraph, synth, torch)
    if args.batch_graph >= 0:
        queries = [q for q in queries if q[0] == args.batch_graph]
    kw = dict(mapping=args.batch_mapping)
    if args.batch_tile:
        kw["tile"] = args.batch_tile
    outs = [torch.empty(graphs[g].n, dtype=torch.int32, device="cuda") for g, _, _ in queries]
    _, tune = seraph.batch_run(graphs, queries, outs=outs, **kw)  # autotune (cached)
    for _ in range(args.warmup):
        seraph.batch_run(graphs, queries, outs=outs, **kw)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        _, st = seraph.batch_run(graphs, queries, outs=outs, replays=args.steps, **kw)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    raw_edges = sum(edges_of[g] for g, _, _ in queries)
    t = max_over_ranks([st["time_ms"] / 1e3], world, "cuda")[0]
    # end to end, as a serving loop: two prepared plans (seraph_batch_plan,
    # each with its own device outputs) run alternately; every step uploads
    # its query sources and its distances are read back into pinned host
    # memory on a copy stream while the next step computes
    srcs = [s for _, _, s in queries]
    sizes = [graphs[g].n for g, _, _ in queries]
    # each plan's outputs are views of one device block, read back in one copy
    blocks = [torch.empty(sum(sizes), dtype=torch.int32, device="cuda") for _ in range(2)]
    douts = [list(torch.split(b, sizes)) for b in blocks]
    plans = [seraph.BatchPlan(graphs, queries, d, **kw) for d in douts]
    hblock = torch.empty(sum(sizes), dtype=torch.int32, pin_memory=True)
    read_back = torch.cuda.Stream()
    read_done = [None, None]
    for pl in plans:
        pl.run(srcs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        k = i % 2
        if read_done[k] is not None:
            read_done[k].synchronize()
        plans[k].run(srcs)
        with torch.cuda.stream(read_back):
            hblock.copy_(blocks[k], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(read_back)
        read_done[k] = ev
    torch.cuda.synchronize()
    te2e = max_over_ranks([(time.perf_counter() - t0) / args.steps], world, "cuda")[0]
    for pl in plans:
        pl.free()
    d2h = sum(4 * graphs[g].n for g, _, _ in queries)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    # work-efficient algorithmic bytes per query over its graph's E edges and n
    # vertices: BFS 8 B per edge (column, destination level) + 12 B per vertex,
    # SSSP 12 B per edge (column, weight, destination distance)
    alg_bytes = sum((8 * edges_of[g] + 12 * graphs[g].n) if a == "bfs" else 12 * edges_of[g]
                    for g, a, _ in queries)
    achieved = alg_bytes / t / 1e9  # per replica: the kernel of one GPU
    nq_job = replica_units(len(queries), world)
    line = {"metric": "batched BFS/SSSP: queries per second and effective GTEPS",
            "value": nq_job / t, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": st["time_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batch-256q-16g-rmat14-22" if args.batch_graph < 0 else
                       f"batch-graph{args.batch_graph}-{len(queries)}q", "graphs": specs,
                       "queries": len(queries), "cuda_graph": bool(st["graph_captured"]),
                       "mapping": st["mapping"], "tile": st["tile"],
                       "l2": "inputs larger than L2: all 16 graphs resident, about "
                             f"{sum(5 * e + 8 * g.n for e, g in zip(edges_of, graphs)) / 1e9:.2f} GB"},
            "gteps_effective": replica_units(raw_edges, world) / t / 1e9,
            "gteps_processed": replica_units(st["edges"], world) / t / 1e9,
            "rounds_max": st["rounds_max"], "tune_ms": tune["tune_ms"],
            "e2e": {"value": nq_job / te2e, "unit": "queries/s",
                    "h2d_bytes_per_step": 4 * len(queries), "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "kernel": "batch_kernel", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "algorithmic_bytes_per_step": alg_bytes},
            "edges_processed_per_raw": st["edges"] / raw_edges,
            # per replay: distances init, round-0 init, the persistent kernel and
            # the scatter of grouped queries' distances
            "gpu_launches": 4 * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------- main

def main():
    args = parse()
    if args.workload == "batch":
        return main_batch(args, int(os.environ.get("WORLD_SIZE", "1")),
                          int(os.environ.get("RANK", "0")))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    sched = {"sssp": parse_sched(args.sssp), "pagerank": parse_sched(args.pagerank)}
    config = {"workload": f"rmat{args.scale}-ef16-streamed", "scale": args.scale, "edge_factor": 16,
              "pages": args.pages, "budget_gb": args.budget_gb, "algorithms": ["sssp", "pagerank"],
              "vertex_order": args.vertex_order,
              "schedule": {"kind": "fixed", **sched},
              "inputs": "pinned host pages streamed each sweep (the method)",
              "l2_flush": "inputs larger than L2 (graph >= 2 GB per sweep)",
              "parallelism": f"replicas{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle  # noqa: F401  (the reference arm is the CPU oracle)
        sample_scale = args.cpu_scale
        # the oracle cannot run the RMAT-28 workload within minutes: its line
        # names the sample it timed, not the GPU arm's graph
        config = dict(config, workload=f"rmat{sample_scale}-ef16-oracle-sample",
                      scale=sample_scale, sample_of=f"rmat{args.scale}-ef16-streamed",
                      inputs="host CSR built by the oracle (no streaming)")
        for _ in range(args.warmup):
            cpu_oracle_sample(sample_scale)
        g_s, t_s, desc, thr = cpu_oracle_sample(sample_scale, steps=args.steps)
        line = {"metric": METRIC, "value": g_s, "unit": "GTEPS", "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_s / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+f64",
                "data": "synthetic", "config": config, "impl": "reference",
                "cpu_baseline": {"value": g_s, "unit": "GTEPS", "cores": thr, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": g_s, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import synth
    import paper_1806_00762_b300 as seraph

    t_setup = time.time()
    g = build_graph(seraph, synth, torch, args.scale, args.pages,
                    reorder=args.vertex_order == "degree")
    info = g.info()
    E = info["m"]
    n = info["n"]
    setup_s = time.time() - t_setup
    link = link_gbps(torch)
    budget = int(args.budget_gb * (1 << 30))
    # Results: each run writes its values into a device buffer and returns;
    # the read-back into pinned host buffers runs on a copy stream while the
    # next run streams its graph (the link carries the pages host -> device
    # and the values device -> host at once).  Two device buffer sets, so a
    # run never overwrites values whose read-back may still be in flight.
    out_u = torch.empty(n, dtype=torch.int32, pin_memory=True)
    out_f = torch.empty(n, dtype=torch.float32, pin_memory=True)
    dev_out = [(torch.empty(n, dtype=torch.int32, device="cuda"),
                torch.empty(n, dtype=torch.float32, device="cuda")) for _ in range(2)]
    read_back = torch.cuda.Stream()
    read_done = [None, None]
    step_no = [0]

    algos = args.algos.split(",")
    empty = {k: 0 for k in ("time_ms", "wall_ms", "relax_ms", "compute_ms", "relax_launches", "bytes_streamed",
                            "copy_ms", "kernel_launches", "edges_relaxed", "vertices_attempted",
                            "changes", "sweeps")}

    def read(dst, src):
        with torch.cuda.stream(read_back):
            dst.copy_(src, non_blocking=True)

    def step(sssp_kw=sched["sssp"], pr_kw=sched["pagerank"]):
        s1 = s2 = empty
        k = step_no[0] % 2
        step_no[0] += 1
        if read_done[k] is not None:
            read_done[k].synchronize()
        du, df = dev_out[k]
        if "sssp" in algos:
            _, s1 = seraph.run(g, "sssp", out=du, source=0, budget_bytes=budget, profile=1,
                               **sssp_kw)
            read(out_u, du)
        if "pagerank" in algos:
            _, s2 = seraph.run(g, "pagerank", out=df, budget_bytes=budget, profile=1, **pr_kw)
            read(out_f, df)
        ev = torch.cuda.Event()
        ev.record(read_back)
        read_done[k] = ev
        return s1, s2

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    stats = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            stats.append(step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()

    dev_s = sum(s1["time_ms"] + s2["time_ms"] for s1, s2 in stats) / 1e3
    dev_s, wall_s = max_over_ranks([dev_s, wall], world, "cuda")
    units = replica_units(len(algos) * E * args.steps, world)
    value = units / dev_s / 1e9
    e2e = units / wall_s / 1e9
    ww = info.get("weight_width", 4)
    relax_bytes = sum(algo_bytes("sssp", s1, ww, sched["sssp"].get("pvu") == "weak") +
                      algo_bytes("pagerank", s2, ww, sched["pagerank"].get("pvu") == "weak")
                      for s1, s2 in stats)
    relax_ms = sum(s1["relax_ms"] + s2["relax_ms"] for s1, s2 in stats)
    relax_launches = sum(s1["relax_launches"] + s2["relax_launches"] for s1, s2 in stats)
    streamed = sum(s1["bytes_streamed"] + s2["bytes_streamed"] for s1, s2 in stats)
    copy_ms = sum(s1["copy_ms"] + s2["copy_ms"] for s1, s2 in stats)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = relax_bytes / (relax_ms / 1e3) / 1e9 if relax_ms else 0.0
    gathers = sum(s1["edges_relaxed"] + s2["edges_relaxed"] for s1, s2 in stats)
    gather_rate = gathers / (relax_ms / 1e3) / 1e9 if relax_ms else 0.0
    gather_peak = gather_ceiling(seraph) / 1e9
    s1, s2 = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 (SSSP), f32 Kahan + f64 residual (PR)",
        "data": "synthetic", "config": config,
        "time_to_fixpoint_s": {"sssp": s1["time_ms"] / 1e3, "pagerank": s2["time_ms"] / 1e3},
        "sweeps": {"sssp": s1["sweeps"], "pagerank": s2["sweeps"]},
        "graph": {"n": n, "m": E, "struct_bytes": info["struct_bytes"],
                  "weight_bytes": info["weight_bytes"], "setup_s": setup_s},
        "e2e": {"value": e2e, "unit": "GTEPS",
                "h2d_bytes_per_step": streamed // args.steps,
                "d2h_bytes_per_step": 2 * 4 * n},
        "roofline": {"bound": "hbm", "kernel": "relax_kernel", "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": relax_traffic(args),
                     "algorithmic_bytes_per_launch": relax_bytes / relax_launches if relax_launches else 0,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "gather_roofline": {"bound": "l2_gather_rate", "kernel": "relax_kernel",
                            "achieved": gather_rate, "peak": gather_peak, "unit": "Ggathers/s",
                            "frac": gather_rate / gather_peak if gather_peak else 0.0,
                            "peak_source": "seraph_gather_probe: 2^29 random 4-byte gathers "
                                           "of 2^28 values, all in an 8 MB evict-last range "
                                           "(every gather an L2 hit), best of 5, this process"},
        "link_roofline": {"bound": "link", "achieved": streamed / (dev_s * 1e9) if dev_s else 0,
                          "peak": link, "unit": "GB/s",
                          "frac": (streamed / (link * 1e9)) / dev_s if dev_s else 0,
                          "copy_busy_frac": copy_ms / 1e3 / dev_s if dev_s else 0},
        "pipeline_roofline": pipeline_roofline(relax_bytes, streamed, dev_s, hbm_peak, link),
        "relax": {"launches": relax_launches, "ms": relax_ms, "bytes": relax_bytes},
        # where a step's device time goes (ms per step, CUDA events): the
        # relax kernels, all kernels of the pipeline steps (gate, compaction,
        # relax, PageRank apply), and the copies on the copy stream
        "phases_ms_per_step": {
            "device": 1e3 * dev_s / args.steps,
            "relax": relax_ms / args.steps,
            "step_kernels": sum(s1["compute_ms"] + s2["compute_ms"] for s1, s2 in stats) / args.steps,
            "copies": copy_ms / args.steps},
        "gpu_launches": int(sum(a["kernel_launches"] + b["kernel_launches"] for a, b in stats)),
        "clocks": clk.summary(),
        "wall_s_timed": wall,
    }
    if not args.no_paper_schedule:
        plain = dict(order="cyclic", window=4, slots=5, pvu="weak", columns="plain")
        p1, p2 = step(plain, dict(plain, pr_normalize=0, pr_omega=1.0))
        p_bytes = (algo_bytes("sssp", p1, ww, True) + algo_bytes("pagerank", p2, ww, True))
        p_time = (p1["time_ms"] + p2["time_ms"]) / 1e3
        line["paper_schedule"] = {
            "schedule": {"sssp": plain, "pagerank": dict(plain, pr_normalize=0, pr_omega=1.0)},
            "time_to_fixpoint_s": {"sssp": p1["time_ms"] / 1e3,
                                                       "pagerank": p2["time_ms"] / 1e3},
            "sweeps": {"sssp": p1["sweeps"], "pagerank": p2["sweeps"]},
            "gteps": 2 * E / p_time / 1e9,
            "pipeline_roofline": pipeline_roofline(
                p_bytes, p1["bytes_streamed"] + p2["bytes_streamed"], p_time, hbm_peak, link)}
    if args.ablation:
        # baseline: one pass per streamed page pair (double buffer, no reuse), no prediction;
        # psi: k = 4 local passes over a window of 4 chunks while the next streams (Fig. 4);
        # psi+pvu: with the predictive vertex update (strong for SSSP, weak for PageRank);
        # then the library's resident-chunk schedule without and with packed SSSP pages,
        # hybrid pages, PageRank's unit-sum scaling at sweep ends and its over-relaxation
        # (the scaling only in the last two rows, the over-relaxation only in the last).
        ladder = [
            ("baseline", dict(order="cyclic", window=1, slots=2, pvu="off", columns="plain"),
             dict(order="cyclic", window=1, slots=2, pvu="off", columns="plain")),
            ("psi", dict(order="cyclic", window=4, slots=5, pvu="off", columns="plain"),
             dict(order="cyclic", window=4, slots=5, pvu="off", columns="plain")),
            ("psi+pvu", dict(order="cyclic", window=4, slots=5, pvu="strong", columns="plain"),
             dict(order="cyclic", window=4, slots=5, pvu="weak", columns="plain")),
            # (PageRank's plain pages do not fit this ring: it streams, and
            # without the scaling and over-relaxation of the last rows the
            # zigzag order needs fewer sweeps there than the cyclic one)
            ("resident+pvu", dict(sched["sssp"], slots=32, columns="plain"),
             dict(sched["pagerank"], slots=32, columns="plain", order="zigzag")),
            ("resident+pvu+packed", dict(sched["sssp"], slots=32, columns="packed"),
             dict(sched["pagerank"], slots=32, columns="plain", order="zigzag")),
            ("resident+pvu+hybrid", sched["sssp"], sched["pagerank"]),
        ]
        ladder = [(nm, ks, dict(kp, pr_normalize=0, pr_omega=1.0)) for nm, ks, kp in ladder]
        ladder.append(("resident+pvu+hybrid+pr_unit_sum", sched["sssp"],
                       dict(sched["pagerank"], pr_normalize=1, pr_omega=1.0)))
        nopush = {k: v for k, v in sched["sssp"].items() if k != "push"}
        ladder = [(nm, {k: v for k, v in ks.items() if k != "push"}, kp) for nm, ks, kp in ladder]
        ladder.append(("resident+pvu+hybrid+pr_unit_sum+sor", nopush,
                       dict(sched["pagerank"], pr_normalize=1)))
        ladder.append(("resident+pvu+hybrid+pr_unit_sum+sor+push", dict(nopush, push=1),
                       dict(sched["pagerank"], pr_normalize=1)))
        # every rung so far streams plain chunks as they are stored; the last
        # adds the compact transfer of plain chunks (the benchmark default)
        plain_xfer = lambda d: {k: v for k, v in d.items() if k != "stream_packed"}
        ladder = [(nm, plain_xfer(ks), plain_xfer(kp)) for nm, ks, kp in ladder]
        ladder.append(("resident+pvu+hybrid+pr_unit_sum+sor+push+compact_transfer", sched["sssp"],
                       dict(sched["pagerank"], pr_normalize=1)))
        line["ablation"] = {}
        for name, ks, kp in ladder:
            a1, a2 = step(ks, kp)
            line["ablation"][name] = {
                "time_to_fixpoint_s": {"sssp": a1["time_ms"] / 1e3, "pagerank": a2["time_ms"] / 1e3},
                "sweeps": {"sssp": a1["sweeps"], "pagerank": a2["sweeps"]},
                "streamed_gb": {"sssp": a1["bytes_streamed"] / 1e9, "pagerank": a2["bytes_streamed"] / 1e9},
                "edges_relaxed": {"sssp": a1["edges_relaxed"], "pagerank": a2["edges_relaxed"]},
                "gteps": 2 * E / ((a1["time_ms"] + a2["time_ms"]) / 1e3) / 1e9}
    if not args.no_learned:
        from paper_1806_00762_b300 import train_sched
        params = train_sched.load()
        if params is None:
            line["learned"] = {"unavailable": "no trained weights (run train_sched)"}
        else:
            model = seraph.SchedModel()
            model.set_params(params)
            lk = {"sssp": dict(sched["sssp"], max_passes=4, sched_model=model),
                  "pagerank": dict(sched["pagerank"], max_passes=1, sched_model=model)}
            for d in lk.values():
                d["window"] = 1
            l1, l2 = step(lk["sssp"], lk["pagerank"])
            fixed_t = {"sssp": s1["time_ms"] / 1e3, "pagerank": s2["time_ms"] / 1e3}
            learned_t = {"sssp": l1["time_ms"] / 1e3, "pagerank": l2["time_ms"] / 1e3}
            line["learned"] = {
                "time_to_fixpoint_s": learned_t,
                "sweeps": {"sssp": l1["sweeps"], "pagerank": l2["sweeps"]},
                "fixed_time_to_fixpoint_s": fixed_t,
                # the method without the network: the paper's fixed k = 4 pipeline
                "fixed_k4_time_to_fixpoint_s": (line["paper_schedule"]["time_to_fixpoint_s"]
                                                if "paper_schedule" in line else None),
                "gteps": 2 * E / (sum(learned_t.values())) / 1e9,
                # the fixed schedule is the yardstick: keep the learned one only where it wins
                "chosen": {a: ("learned" if learned_t[a] < fixed_t[a] else "fixed") for a in fixed_t},
                "weights": "paper_1806_00762_b300/sched_weights.f32"}
    if args.stream_budget_gb < 0:
        args.stream_budget_gb = args.budget_gb / 2
    if args.stream_budget_gb > 0:
        # the library's own schedules under a budget too small for the graph to
        # become resident: every sweep streams (the out-of-budget regime)
        sb = int(args.stream_budget_gb * (1 << 30))
        r1 = r2 = empty
        if "sssp" in algos:
            _, r1 = seraph.run(g, "sssp", out=out_u, source=0, budget_bytes=sb, profile=1,
                               **sched["sssp"])
        if "pagerank" in algos:
            _, r2 = seraph.run(g, "pagerank", out=out_f, budget_bytes=sb, profile=1,
                               **sched["pagerank"])
        st_t = (r1["time_ms"] + r2["time_ms"]) / 1e3
        st_b = r1["bytes_streamed"] + r2["bytes_streamed"]
        line["streaming_budget"] = {
            "budget_gb": args.stream_budget_gb,
            "resident": {"sssp": r1["resident"], "pagerank": r2["resident"]},
            "time_to_fixpoint_s": {"sssp": r1["time_ms"] / 1e3, "pagerank": r2["time_ms"] / 1e3},
            "sweeps": {"sssp": r1["sweeps"], "pagerank": r2["sweeps"]},
            "streamed_gb": {"sssp": r1["bytes_streamed"] / 1e9, "pagerank": r2["bytes_streamed"] / 1e9},
            "gteps": len(algos) * E / st_t / 1e9 if st_t else 0.0,
            "pipeline_roofline": pipeline_roofline(
                algo_bytes("sssp", r1, ww, sched["sssp"].get("pvu") == "weak") +
                algo_bytes("pagerank", r2, ww, sched["pagerank"].get("pvu") == "weak"),
                st_b, st_t, hbm_peak, link)}
    if rank == 0 and not args.no_cpu_baseline:
        g_s, t_s, desc, thr = cpu_oracle_sample(args.cpu_scale)
        line["cpu_baseline"] = {"value": g_s, "unit": "GTEPS", "cores": thr, "kind": "oracle",
                                "sample": desc, "seconds": t_s}
        if "pagerank" in algos:
            line["pagerank_error_vs_oracle"] = pagerank_error_vs_oracle(
                seraph, synth, torch, args.cpu_scale, args.pages, sched["pagerank"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
