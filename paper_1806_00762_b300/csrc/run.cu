// Host sweep driver: pipelined subgraph iteration (Sec. 3.2, Fig. 4) with
// predictive vertex updating (Sec. 4) to a fixpoint.
//
// The device edge buffer is a ring of window+1 slots.  Global step t
//   (1) enqueues, on the copy stream, the host->device copy of the chunk of
//       step t+1 into slot (t+1) mod R, after the event of step t-1 (the last
//       step whose window held that slot's previous chunk);
//   (2) enqueues, on the compute stream, `passes` local passes over the
//       window (chunks t-window+1 .. t) once the copy of chunk t is done.
// A sweep is C consecutive steps (C = chunks); every chunk gets
// window * passes passes in it.  At the end of a sweep one small report is
// copied back; the host reads it while the next chunk is already in flight
// and decides: continue, run a prediction-off verification sweep, or stop.
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "graph.hpp"

namespace seraph {
namespace {

struct Chunk {
    uint32_t first_page, end_page;
    uint64_t s_begin, s_bytes;  // structure byte range in the pinned region
    uint64_t w_begin, w_bytes;  // weight byte range (0 bytes if not streamed)
    uint64_t w_slot_off;        // weights start this far into the slot
    uint32_t v_begin, v_end;
};

struct Event {
    cudaEvent_t e = nullptr;
    void create(bool timing) {
        SR_CUDA(cudaEventCreateWithFlags(&e, timing ? cudaEventDefault : cudaEventDisableTiming));
    }
    ~Event() { if (e) cudaEventDestroy(e); }
};

void wait_event(cudaEvent_t e, uint32_t timeout_ms) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t r = cudaEventQuery(e);
        if (r == cudaSuccess) return;
        if (r != cudaErrorNotReady) SR_CUDA(r);
        auto ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        SR_CHECK(ms < timeout_ms, SERAPH_ETIMEOUT, "timed out waiting for the device");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    SR_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
}

}  // namespace

int run_graph(seraph_graph* g, const seraph_params* P, void* out, int out_mem, seraph_stats* st) {
    auto wall0 = std::chrono::steady_clock::now();
    SR_CHECK(g && P, SERAPH_EINVAL, "null graph or params");
    SR_CHECK(P->algo >= SERAPH_SSSP && P->algo <= SERAPH_PAGERANK, SERAPH_EINVAL, "bad algo");
    SR_CHECK(P->window >= 1 && P->window <= kMaxWindow, SERAPH_EINVAL, "window must be in [1,16]");
    SR_CHECK(P->passes >= 1 && P->passes <= 64, SERAPH_EINVAL, "passes must be in [1,64]");
    SR_CHECK(P->pvu >= SERAPH_PVU_OFF && P->pvu <= SERAPH_PVU_WEAK, SERAPH_EINVAL, "bad pvu");
    SR_CHECK(!(P->algo == SERAPH_PAGERANK && P->pvu == SERAPH_PVU_STRONG), SERAPH_EINVAL,
             "PageRank has no strong prediction condition; use weak or off");
    SR_CHECK(!(P->pvu == SERAPH_PVU_WEAK && !P->verify), SERAPH_EINVAL,
             "weak prediction needs the verification sweep");
    SR_CHECK(out_mem == SERAPH_MEM_HOST || out_mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad out_mem");
    SR_CHECK(P->max_sweeps >= 1, SERAPH_EINVAL, "max_sweeps must be >= 1");
    for (int i = 0; i < 12; ++i)
        SR_CHECK(P->fsm_next[i] < 6, SERAPH_EINVAL, "fsm_next entries must be < 6");
    SR_CHECK(P->thread_max_deg <= P->warp_max_deg, SERAPH_EINVAL, "thread_max_deg > warp_max_deg");
    const uint64_t n = g->n;
    int algo = P->algo;
    if ((algo == SERAPH_SSSP || algo == SERAPH_BFS))
        SR_CHECK(P->source < n, SERAPH_EINVAL, "source >= n");
    if (algo == SERAPH_SSSP && !g->weighted) algo = SERAPH_BFS;  // unit weights
    const bool use_w = algo == SERAPH_SSSP;
    const bool is_pr = algo == SERAPH_PAGERANK;
    SR_CUDA(cudaSetDevice(g->device));

    // ------------------------------------------------------------ chunking
    const uint32_t W = P->window;
    const uint32_t R = W + 1;
    const uint64_t slot_bytes = (P->budget_bytes / R) & ~255ull;
    SR_CHECK(slot_bytes >= 256, SERAPH_EBUDGET, "budget too small for the ring");
    std::vector<Chunk> chunks;
    {
        Chunk cur{};
        bool open = false;
        for (uint32_t p = 0; p < g->num_pages; ++p) {
            const PageMeta& pm = g->pages[p];
            const uint64_t wb = use_w ? pm.w_bytes : 0;
            SR_CHECK(align_up(pm.s_bytes, 256) + wb <= slot_bytes, SERAPH_EBUDGET,
                     "page " + std::to_string(p) + " (" + std::to_string(pm.s_bytes + wb) +
                         " B) does not fit a ring slot of " + std::to_string(slot_bytes) + " B");
            if (open && align_up(cur.s_bytes + pm.s_bytes, 256) + cur.w_bytes + wb <= slot_bytes) {
                cur.end_page = p + 1;
                cur.s_bytes += pm.s_bytes;
                cur.w_bytes += wb;
                cur.v_end = (uint32_t)(pm.vb + pm.nv);
                continue;
            }
            if (open) chunks.push_back(cur);
            cur = Chunk{p, p + 1, pm.s_off, pm.s_bytes, pm.w_off, wb, 0, (uint32_t)pm.vb,
                        (uint32_t)(pm.vb + pm.nv)};
            open = true;
        }
        if (open) chunks.push_back(cur);
    }
    for (auto& c : chunks) c.w_slot_off = align_up(c.s_bytes, 256);
    const uint32_t C = (uint32_t)chunks.size();
    const bool resident = C <= R;
    const uint32_t Weff = W < C ? W : C;
    const uint32_t nslots = resident ? C : R;

    // static per-page placement relative to the chunk image
    std::vector<uint64_t> rel_soff(g->num_pages), rel_woff(g->num_pages), offb(g->num_pages);
    for (const Chunk& c : chunks)
        for (uint32_t p = c.first_page; p < c.end_page; ++p) {
            rel_soff[p] = g->pages[p].s_off - c.s_begin;
            rel_woff[p] = c.w_slot_off + (g->pages[p].w_off - c.w_begin);
            offb[p] = g->pages[p].off_bytes;
        }
    uint64_t max_win_v = 1;
    for (uint32_t t = 0; t < C; ++t) {
        uint64_t s = 0;
        for (uint32_t k = 0; k < Weff; ++k) {
            const Chunk& c = chunks[(t + C - k) % C];
            s += c.v_end - c.v_begin;
        }
        max_win_v = std::max<uint64_t>(max_win_v, s);
    }

    // --------------------------------------------------------- allocations
    Stream cs, xs;
    cs.use(P->stream);
    xs.create();
    DevBuf<uint8_t> ebuf(slot_bytes * nslots);
    DevBuf<PageLoc> loc(g->num_pages);
    DevBuf<uint64_t> d_rel_soff(g->num_pages), d_rel_woff(g->num_pages), d_offb(g->num_pages);
    SR_CUDA(cudaMemcpyAsync(d_rel_soff.p, rel_soff.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    SR_CUDA(cudaMemcpyAsync(d_rel_woff.p, rel_woff.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    SR_CUDA(cudaMemcpyAsync(d_offb.p, offb.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    DevBuf<unsigned long long> lists(3 * max_win_v);
    DevBuf<RunState> rs(1);
    DevBuf<SweepReport> d_rep(1);
    PinnedBuf h_rep;
    h_rep.alloc(sizeof(SweepReport));
    DevBuf<uint32_t> val;
    DevBuf<float> x, contrib, x_next, x_prev, inv_out;
    DevBuf<uint8_t> state;
    const int nparts = device_sms() * 4;
    DevBuf<double> partial;
    if (is_pr) {
        x.alloc(n); contrib.alloc(n); x_next.alloc(n); x_prev.alloc(n); inv_out.alloc(n);
        partial.alloc(nparts);
    } else {
        val.alloc(n);
    }
    if (P->pvu == SERAPH_PVU_WEAK) state.alloc(n);

    AlgoArgs a{};
    a.val = val.p;
    a.x = x.p;
    a.contrib = contrib.p;
    a.x_next = x_next.p;
    a.inv_out = inv_out.p;
    a.state = state.p;
    a.rs = rs.p;
    a.loc = loc.p;
    a.vb = g->d_vb.p;
    for (int k = 0; k < 3; ++k) a.list[k] = lists.p + k * max_win_v;
    a.thread_max = P->thread_max_deg;
    a.warp_max = P->warp_max_deg;
    a.damping = (float)P->damping;
    a.fail_eps = (float)P->pr_fail_eps;
    std::memcpy(a.fsm_next, P->fsm_next, 12);
    a.skip_mask = P->fsm_skip_mask;
    a.pvu = (uint8_t)P->pvu;

    uint64_t launches = 0;
    {
        RunState init{};
        init.thr_cur = SERAPH_INF;
        init.thr_prev = 0;  // the initial values count as sweep-0 writes (minimum 0)
        SR_CUDA(cudaMemcpyAsync(rs.p, &init, sizeof(init), cudaMemcpyHostToDevice, cs.s));
        if (is_pr) {
            launch_init_pr(g->d_outdeg.p, a, x_prev.p, n, cs.s);
            launch_close_pr(a, n, x_prev.p, g->d_zero_in.p, P->damping, partial.p, nparts,
                            nullptr, cs.s);
            launches += 4;
            // the init residual pass must not count as a sweep
            SR_CUDA(cudaMemcpyAsync(&rs.p->cur, &init.cur, sizeof(init.cur), cudaMemcpyHostToDevice, cs.s));
        } else {
            launch_init_values(algo, a, n, P->source, cs.s);
            launches += 1;
        }
        SR_CUDA(cudaStreamSynchronize(cs.s));
    }

    // -------------------------------------------------------------- events
    std::vector<Event> copy_done(R), step_done(R);
    for (uint32_t i = 0; i < R; ++i) { copy_done[i].create(false); step_done[i].create(false); }
    Event ev_start, ev_stop, ev_sweep;
    ev_start.create(true);
    ev_stop.create(true);
    ev_sweep.create(false);
    const bool prof = P->profile != 0;
    // per-sweep profiling pools, double-buffered by sweep parity
    std::vector<Event> pc_b, pc_e, pk_b, pk_e, pr_b, pr_e;
    if (prof) {
        for (auto* v : {&pc_b, &pc_e, &pk_b, &pk_e}) {
            v->resize(2 * C);
            for (auto& e : *v) e.create(true);
        }
        for (auto* v : {&pr_b, &pr_e}) {
            v->resize(C * P->passes);
            for (auto& e : *v) e.create(true);
        }
    }

    seraph_stats S{};
    S.chunks = C;
    S.resident = resident;
    std::vector<uint8_t> loaded(C, 0);

    auto load = [&](uint64_t t) {  // chunk for step t into its slot
        const uint32_t c = (uint32_t)(t % C);
        const uint32_t slot = resident ? c : (uint32_t)(t % R);
        if (!resident && t >= R) SR_CUDA(cudaStreamWaitEvent(xs.s, step_done[(t - 2) % R].e, 0));
        const Chunk& ch = chunks[c];
        uint8_t* sb = ebuf.p + (uint64_t)slot * slot_bytes;
        uint8_t* wb = use_w ? sb + ch.w_slot_off : nullptr;
        const int par = (int)((t / C) & 1), i = (int)(t % C);
        if (prof) SR_CUDA(cudaEventRecord(pc_b[par * C + i].e, xs.s));
        SR_CUDA(cudaMemcpyAsync(sb, g->h_struct.p + ch.s_begin, ch.s_bytes, cudaMemcpyHostToDevice, xs.s));
        if (use_w && ch.w_bytes)
            SR_CUDA(cudaMemcpyAsync(wb, g->h_weight.p + ch.w_begin, ch.w_bytes, cudaMemcpyHostToDevice, xs.s));
        if (prof) SR_CUDA(cudaEventRecord(pc_e[par * C + i].e, xs.s));
        launch_set_locs(loc.p, g->d_vb.p, ch.first_page, ch.end_page, d_rel_soff.p, d_rel_woff.p,
                        d_offb.p, sb, use_w ? ebuf.p + (uint64_t)slot * slot_bytes : nullptr, xs.s);
        ++launches;
        SR_CUDA(cudaEventRecord(copy_done[t % R].e, xs.s));
        S.bytes_streamed += ch.s_bytes + (use_w ? ch.w_bytes : 0);
        loaded[c] = 1;
    };

    const unsigned relax_grid = device_sms() * 8;
    uint32_t pass = 0;
    bool predict = P->pvu != SERAPH_PVU_OFF;
    bool pr_predict_off = false;
    int rc = SERAPH_OK;
    std::vector<double> copy_ms_by_sweep;

    SR_CUDA(cudaStreamSynchronize(cs.s));
    SR_CUDA(cudaEventRecord(ev_start.e, xs.s));
    load(0);
    for (uint64_t t = 0;; ++t) {
        const uint32_t c = (uint32_t)(t % C);
        const uint64_t sweep = t / C;
        const int par = (int)(sweep & 1), si = (int)(t % C);
        if (!resident || t + 1 < C) load(t + 1);
        if (!resident || t < C) SR_CUDA(cudaStreamWaitEvent(cs.s, copy_done[t % R].e, 0));
        if (prof) SR_CUDA(cudaEventRecord(pk_b[par * C + si].e, cs.s));

        WindowDesc wd{};
        {
            const uint32_t wn = (uint32_t)std::min<uint64_t>(Weff, t + 1);
            uint32_t blocks = 0;
            for (uint32_t k = 0; k < wn; ++k) {  // oldest first
                const Chunk& ch = chunks[(c + C - (wn - 1 - k)) % C];
                ChunkDesc& d = wd.c[k];
                d.v_begin = ch.v_begin;
                d.v_end = ch.v_end;
                d.first_page = ch.first_page;
                d.end_page = ch.end_page;
                d.block_begin = blocks;
                blocks += (uint32_t)((uint64_t(ch.v_end - ch.v_begin) + 1023) / 1024);
            }
            wd.nchunks = wn;
            wd.nblocks = blocks;
        }
        const bool pred_now = is_pr ? (predict && !pr_predict_off) : predict;
        for (uint32_t j = 0; j < P->passes; ++j) {
            launch_compact(algo, wd, a, pass, j > 0, pred_now ? 1 : 0, cs.s);
            if (prof) SR_CUDA(cudaEventRecord(pr_b[si * P->passes + j].e, cs.s));
            launch_relax(algo, P->kahan, a, pass, j > 0, relax_grid, cs.s);
            if (prof) SR_CUDA(cudaEventRecord(pr_e[si * P->passes + j].e, cs.s));
            launches += 2;
            S.relax_launches += 1;
            if (is_pr) {
                launch_pr_apply(a, pass, j > 0, relax_grid, cs.s);
                ++launches;
            }
            ++pass;
        }
        if (prof) SR_CUDA(cudaEventRecord(pk_e[par * C + si].e, cs.s));
        SR_CUDA(cudaEventRecord(step_done[t % R].e, cs.s));
        S.steps += 1;

        if (c != C - 1) continue;
        // ---------------------------------------------------- sweep close
        if (is_pr)
            launch_close_pr(a, n, x_prev.p, g->d_zero_in.p, P->damping, partial.p, nparts, d_rep.p, cs.s);
        else
            launch_close_min(rs.p, d_rep.p, cs.s);
        launches += is_pr ? 4 : 1;
        SR_CUDA(cudaMemcpyAsync(h_rep.p, d_rep.p, sizeof(SweepReport), cudaMemcpyDeviceToHost, cs.s));
        SR_CUDA(cudaEventRecord(ev_sweep.e, cs.s));
        wait_event(ev_sweep.e, P->timeout_ms);
        SweepReport rep;
        std::memcpy(&rep, h_rep.p, sizeof(rep));
        S.sweeps += 1;
        S.passes_run += rep.passes_run;
        S.passes_skipped += rep.passes_skipped;
        S.edges_relaxed += rep.edges;
        S.vertices_attempted += rep.attempted;
        S.vertices_skipped += rep.skipped;
        S.changes += rep.changed;
        if (!pred_now) S.verify_sweeps += 1;
        if (prof) {
            for (uint32_t i = 0; i < C; ++i) {
                S.compute_ms += elapsed(pk_b[par * C + i].e, pk_e[par * C + i].e);
                for (uint32_t j = 0; j < P->passes; ++j)
                    S.relax_ms += elapsed(pr_b[i * P->passes + j].e, pr_e[i * P->passes + j].e);
                if (!resident || sweep == 0)
                    S.copy_ms += elapsed(pc_b[par * C + i].e, pc_e[par * C + i].e);
            }
        }
        bool stop = false;
        if (is_pr) {
            S.residual = rep.resid;
            if (!pred_now && rep.resid < P->tol) { S.converged = 1; stop = true; }
            else if (pred_now && rep.resid < std::max(P->pr_pvu_off_below, P->tol)) pr_predict_off = true;
            if (!stop && S.sweeps >= P->max_sweeps) stop = true;
        } else {
            if (rep.changed == 0 && (!pred_now || !P->verify)) {
                S.converged = 1;
                stop = true;
                if (rep.overflow) rc = SERAPH_EOVERFLOW;
            } else if (rep.changed == 0) {
                predict = false;  // verification sweep with prediction off
            } else {
                predict = P->pvu != SERAPH_PVU_OFF;
            }
            if (!stop && S.sweeps >= P->max_sweeps) { rc = SERAPH_ENOTCONV; stop = true; }
        }
        if (stop) break;
    }
    SR_CUDA(cudaEventRecord(ev_stop.e, cs.s));
    SR_CUDA(cudaStreamSynchronize(cs.s));
    S.time_ms = elapsed(ev_start.e, ev_stop.e);

    // ------------------------------------------------------------- output
    const void* src = is_pr ? (const void*)x.p : (const void*)val.p;
    if (out) {
        SR_CUDA(cudaMemcpyAsync(out, src, 4 * n,
                                out_mem == SERAPH_MEM_HOST ? cudaMemcpyDeviceToHost
                                                           : cudaMemcpyDeviceToDevice,
                                cs.s));
    }
    SR_CUDA(cudaStreamSynchronize(cs.s));
    SR_CUDA(cudaStreamSynchronize(xs.s));
    S.kernel_launches = launches;
    S.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    if (st) *st = S;
    if (rc == SERAPH_EOVERFLOW)
        throw Error(SERAPH_EOVERFLOW, "an SSSP distance does not fit below 2^32-1");
    if (rc == SERAPH_ENOTCONV)
        throw Error(SERAPH_ENOTCONV, "max_sweeps reached before the fixpoint");
    return rc;
}

}  // namespace seraph
