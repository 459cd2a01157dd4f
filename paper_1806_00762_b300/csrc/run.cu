// Host sweep driver: pipelined subgraph iteration (Sec. 3.2, Fig. 4) with
// predictive vertex updating (Sec. 4) to a fixpoint.
//
// The device edge buffer is a ring of `slots` (>= window+1) slots.  Every
// pipeline step
//   (1) enqueues, on the copy stream, the host->device copy of the chunk the
//       next step needs into the free slot, after the event of the step that
//       last used that slot;
//   (2) enqueues, on the compute stream, `passes` local passes over the
//       window of resident chunks once their copies are done, then up to
//       `max_passes` idle-slot passes that each run only while the copy of
//       (1) is still in flight and the previous pass changed something;
//   (3) evicts one chunk of the window; its slot becomes the next free slot.
// Which chunk comes next is the schedule's choice: the paper's sliding
// window wraps cyclically; the zigzag order reverses at each end so that the
// resident window opens the next sweep without being streamed again.
//
// Per-step change counts live on the device.  At the end of a sweep one
// small report and the step counts are copied back while the next chunk is
// already in flight, and the host decides: continue, turn prediction off, or
// stop.  SSSP/BFS/CC stop once every chunk has been processed with
// prediction off after the last change anywhere; PageRank stops on the FP64
// L1 change between sweep ends.
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include <algorithm>
#include <numeric>

#include "engine.cuh"
#include "graph.hpp"
#include "mlp.cuh"
#include "push.cuh"

namespace seraph {
namespace {

struct Chunk {
    uint32_t first_page, end_page;
    uint64_t s_begin, s_bytes;  // structure byte range in the pinned region
    uint64_t w_begin, w_bytes;  // weight byte range (0 bytes if not streamed)
    uint64_t w_slot_off;        // weights start this far into the slot
    uint32_t v_begin, v_end;
    bool packed;                // pages in the packed form (else plain)
    // stream_packed: the plain chunk streams compact -- each page's streamed
    // header and gap stream, pk_bytes in all -- to slot offset stage_off and
    // is rebuilt in place
    bool decode;
    uint64_t pk_bytes, stage_off;
};

// A typed piece of a larger allocation (not owned).
template <class T>
struct Slice {
    T* p = nullptr;
};

// Bytes a page stages in its slot when its chunk streams compact: its
// streamed header, then its gap stream padded to 16 bytes.
uint64_t staged_bytes(const PageMeta& pm) { return pm.sh_bytes + align_up(pm.pk_data, 16); }

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

// Window schedules over C chunks with a window of W.  window(t) is the set of
// chunks step t processes; it is a pure function of t (a ramp followed by a
// periodic part, both tabulated once) so that the driver can look ahead for
// loads and evictions.
class Schedule {
  public:
    // Dynamic schedule (window of one chunk, a chunk order chosen per sweep;
    // sweeps not chosen yet are assumed to visit every chunk, alternating
    // direction when `zig`).
    Schedule(uint32_t C, bool zig) : C_(C), W_(1), zigzag_(zig), dynamic_(true) {
        for (uint32_t c = 0; c < C; ++c) singles_.push_back({c});
        std::vector<uint32_t> first(C);
        std::iota(first.begin(), first.end(), 0u);
        orders_.push_back(first);
        starts_.push_back(0);
    }
    // The next sweep's order (appended after the last known sweep).
    void append_order(const std::vector<uint32_t>& order) {
        starts_.push_back(starts_.back() + orders_.back().size());
        orders_.push_back(order);
    }

    Schedule(uint32_t C, uint32_t W, int order, bool resident)
        : C_(C), W_(resident ? (W < C ? W : C) : W), zigzag_(!resident && order == SERAPH_ORDER_ZIGZAG) {
        if (!zigzag_) {  // sliding window, cyclic over the chunks
            ramp_ = W_ - 1;
            period_ = C_;
            for (uint64_t t = 0; t < ramp_ + period_; ++t) {
                const uint64_t wn = std::min<uint64_t>(W_, t + 1);
                const uint32_t c = (uint32_t)(t % C_);
                std::vector<uint32_t> w;
                for (uint64_t k = 0; k < wn; ++k) w.push_back((uint32_t)((c + C_ - (wn - 1 - k)) % C_));
                table_.push_back(w);
            }
        } else {  // lowest chunk: 0,1,..,C-W (forward), C-W-1,..,1 (back)
            ramp_ = W_ - 1;
            const uint64_t span = C_ - W_;
            period_ = 2 * span;
            for (uint64_t t = 0; t < ramp_; ++t) {
                std::vector<uint32_t> w;
                for (uint32_t k = 0; k <= t; ++k) w.push_back(k);
                table_.push_back(w);
            }
            for (uint64_t u = 0; u < period_; ++u) {
                const uint32_t lo = (uint32_t)(u <= span ? u : 2 * span - u);
                std::vector<uint32_t> w;
                for (uint32_t k = 0; k < W_; ++k) w.push_back(lo + k);
                table_.push_back(w);
            }
        }
    }

    const std::vector<uint32_t>& window(uint64_t t) const {
        if (dynamic_) {
            bool end;
            return singles_[dyn_chunk(t, &end)];
        }
        return table_[t < ramp_ ? t : ramp_ + (t - ramp_) % period_];
    }

    bool sweep_end(uint64_t t) const {
        if (dynamic_) {
            bool end;
            dyn_chunk(t, &end);
            return end;
        }
        if (!zigzag_) return t % C_ == C_ - 1;
        if (t < ramp_) return false;
        const uint64_t u = t - ramp_, span = C_ - W_;
        return u > 0 && u % span == 0;
    }

  private:
    // sweep j and position i of step t; beyond the known sweeps the last
    // order is assumed to repeat (look-ahead only)
    // Chunk and end-of-sweep flag of dynamic step t.
    uint32_t dyn_chunk(uint64_t t, bool* end) const {
        size_t j = (size_t)(std::upper_bound(starts_.begin(), starts_.end(), t) - starts_.begin()) - 1;
        uint64_t i = t - starts_[j];
        if (i < orders_[j].size()) {
            *end = i + 1 == orders_[j].size();
            return orders_[j][i];
        }
        // beyond the known sweeps: full sweeps in the base direction
        const uint64_t off = i - orders_[j].size();
        const uint64_t js = orders_.size() + off / C_, k = off % C_;
        *end = k + 1 == C_;
        return (uint32_t)(zigzag_ && (js & 1) ? C_ - 1 - k : k);
    }
    uint32_t C_, W_;
    bool zigzag_, dynamic_ = false;
    uint64_t ramp_ = 0, period_ = 1;
    std::vector<std::vector<uint32_t>> table_;
    std::vector<std::vector<uint32_t>> orders_, singles_;
    std::vector<uint64_t> starts_;
};

}  // namespace

int run_graph(seraph_graph* g, const seraph_params* P, void* out, int out_mem, seraph_stats* st) {
    auto wall0 = std::chrono::steady_clock::now();
    SR_CHECK(g && P, SERAPH_EINVAL, "null graph or params");
    SR_CHECK(P->algo >= SERAPH_SSSP && P->algo <= SERAPH_PAGERANK, SERAPH_EINVAL, "bad algo");
    SR_CHECK(P->window >= 1 && P->window <= kMaxWindow, SERAPH_EINVAL, "window must be in [1,16]");
    SR_CHECK(P->passes >= 1 && P->passes <= 64, SERAPH_EINVAL, "passes must be in [1,64]");
    SR_CHECK(P->max_passes <= 64, SERAPH_EINVAL, "max_passes must be <= 64");
    SR_CHECK(P->order == SERAPH_ORDER_CYCLIC || P->order == SERAPH_ORDER_ZIGZAG, SERAPH_EINVAL,
             "bad order");
    SR_CHECK(P->pvu >= SERAPH_PVU_OFF && P->pvu <= SERAPH_PVU_WEAK, SERAPH_EINVAL, "bad pvu");
    SR_CHECK(!(P->algo == SERAPH_PAGERANK && P->pvu == SERAPH_PVU_STRONG), SERAPH_EINVAL,
             "PageRank has no strong prediction condition; use weak or off");
    SR_CHECK(!(P->pvu == SERAPH_PVU_WEAK && !P->verify), SERAPH_EINVAL,
             "weak prediction needs the verification sweep");
    SR_CHECK(out_mem == SERAPH_MEM_HOST || out_mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad out_mem");
    SR_CHECK(P->max_sweeps >= 1, SERAPH_EINVAL, "max_sweeps must be >= 1");
    SR_CHECK(P->pr_omega >= 0.0 && P->pr_omega < 2.0, SERAPH_EINVAL, "pr_omega must be in [0, 2)");
    for (int i = 0; i < 12; ++i)
        SR_CHECK(P->fsm_next[i] < 6, SERAPH_EINVAL, "fsm_next entries must be < 6");
    SR_CHECK(P->thread_max_deg <= P->group4_max_deg && P->group4_max_deg <= P->group8_max_deg &&
                 P->group8_max_deg <= P->warp_max_deg,
             SERAPH_EINVAL, "need thread_max_deg <= group4_max_deg <= group8_max_deg <= warp_max_deg");
    const bool learned = P->sched == SERAPH_SCHED_LEARNED;
    seraph_trace* trace = (seraph_trace*)P->trace;
    SR_CHECK(P->sched == SERAPH_SCHED_FIXED || learned, SERAPH_EINVAL, "bad sched");
    SR_CHECK(!learned || P->sched_model, SERAPH_EINVAL, "learned schedule needs sched_model");
    SR_CHECK(!(learned || trace) || P->window == 1, SERAPH_EINVAL,
             "learned schedules and traces need window = 1");
    const SchedModel* model = learned ? &((seraph_sched_model*)P->sched_model)->model : nullptr;
    SR_CHECK(P->push <= 1, SERAPH_EINVAL, "push must be 0 or 1");
    SR_CHECK(!P->push || P->algo != SERAPH_PAGERANK, SERAPH_EINVAL,
             "the push stage is for SSSP, BFS and CC");
    SR_CHECK(!P->push || g->out_edges, SERAPH_EINVAL,
             "the push stage needs a graph built with SERAPH_OUT_EDGES");
    SR_CHECK(!P->push || !(P->algo == SERAPH_CC && !g->symmetrized), SERAPH_EINVAL,
             "CC with the push stage needs a symmetrized graph");
    const uint64_t n = g->n;
    int algo = P->algo;
    if ((algo == SERAPH_SSSP || algo == SERAPH_BFS))
        SR_CHECK(P->source < n, SERAPH_EINVAL, "source >= n");
    if (algo == SERAPH_SSSP && !g->weighted) algo = SERAPH_BFS;  // unit weights
    const bool use_w = algo == SERAPH_SSSP;
    const bool is_pr = algo == SERAPH_PAGERANK;
    SR_CUDA(cudaSetDevice(g->device));

    // ------------------------------------------------------------ chunking
    SR_CHECK(P->columns <= SERAPH_COLUMNS_HYBRID, SERAPH_EINVAL, "bad columns");
    const bool any_packed = P->columns != SERAPH_COLUMNS_PLAIN &&
                            (P->columns != SERAPH_COLUMNS_AUTO || g->packed);
    SR_CHECK(!any_packed || g->packed, SERAPH_EINVAL, "graph was built without SERAPH_COMPRESS");
    const bool hybrid = P->columns == SERAPH_COLUMNS_HYBRID;
    SR_CHECK(P->stream_packed <= 1, SERAPH_EINVAL, "stream_packed must be 0 or 1");
    const bool stream_packed = P->stream_packed != 0;
    SR_CHECK(!stream_packed || g->packed, SERAPH_EINVAL,
             "stream_packed needs a graph built with SERAPH_COMPRESS");
    SR_CHECK(!hybrid || P->window == 1, SERAPH_EINVAL, "hybrid page forms need window = 1");
    const uint32_t W = P->window;
    const uint32_t R = P->slots ? P->slots : W + 1;
    SR_CHECK(R >= W + 1 && R <= 4096, SERAPH_EINVAL, "slots must be in [window+1, 4096]");
    const uint64_t slot_bytes = (P->budget_bytes / R) & ~255ull;
    SR_CHECK(slot_bytes >= 256, SERAPH_EBUDGET, "budget too small for the ring");
    // Pages [0, npk) stream packed, the rest plain (npk = 0 or P for one form).
    // Chunks are runs of consecutive pages of one form that fit a slot.
    // Returns false (or throws SERAPH_EBUDGET when `strict`) if a page does not
    // fit a slot in its form.
    auto make_chunks = [&](uint32_t npk, std::vector<Chunk>& out, bool strict) {
        out.clear();
        Chunk cur{};
        bool open = false;
        for (uint32_t p = 0; p < g->num_pages; ++p) {
            const PageMeta& pm = g->pages[p];
            const bool pk = p < npk;
            const uint64_t sb = pk ? pm.pk_bytes : pm.s_bytes;
            const uint64_t wb = use_w ? pm.w_bytes : 0;
            // a plain page that may stream packed leaves room for its packed
            // form behind the chunk's plain bytes (the decode's staging)
            const uint64_t slack = stream_packed && !pk ? align_up(staged_bytes(pm), 256) : 0;
            if (align_up(sb, 256) + wb > slot_bytes) {
                SR_CHECK(!strict, SERAPH_EBUDGET,
                         "page " + std::to_string(p) + " (" + std::to_string(sb + wb) +
                             " B) does not fit a ring slot of " + std::to_string(slot_bytes) + " B");
                return false;
            }
            if (open && cur.packed == pk &&
                align_up(cur.s_bytes + sb, 256) + cur.w_bytes + wb + slack <= slot_bytes) {
                cur.end_page = p + 1;
                cur.s_bytes += sb;
                cur.w_bytes += wb;
                cur.v_end = (uint32_t)(pm.vb + pm.nv);
                continue;
            }
            if (open) out.push_back(cur);
            cur = Chunk{p, p + 1, pk ? pm.pk_off : pm.s_off, sb, pm.w_off, wb, 0, (uint32_t)pm.vb,
                        (uint32_t)(pm.vb + pm.nv), pk, false, 0, 0};
            open = true;
        }
        if (open) out.push_back(cur);
        return true;
    };
    std::vector<Chunk> chunks;
    uint32_t npk = any_packed ? g->num_pages : 0;
    if (hybrid) {
        // the fewest packed pages (the first pages hold the most-connected
        // destinations when vertices are in out-degree order, and their gaps
        // are short) with which every chunk stays resident in the ring; never
        // a page from the first one whose packed form is not smaller than its
        // plain form on (the tail of many vertices with few in-edges), so a
        // ring that cannot hold the graph packs exactly the pages that shrink
        uint32_t shrink = 0;
        while (shrink < g->num_pages && g->pages[shrink].pk_bytes < g->pages[shrink].s_bytes) ++shrink;
        std::vector<Chunk> trial;
        uint32_t lo = 0, hi = make_chunks(shrink, trial, false) ? shrink : g->num_pages;
        while (lo < hi) {  // (a split whose plain pages do not fit a slot counts as too few)
            const uint32_t mid = (lo + hi) / 2;
            if (make_chunks(mid, trial, false) && trial.size() <= R) hi = mid; else lo = mid + 1;
        }
        npk = lo;
    }
    make_chunks(npk, chunks, true);
    const bool packed = npk > 0;  // some pages stream packed
    for (auto& c : chunks) c.w_slot_off = align_up(c.s_bytes, 256);
    // Streaming a plain chunk compact: its pages' streamed headers and gap
    // streams go to the far end of the slot and page j is rebuilt into its
    // plain place, which must end before page j's staged bytes start (pages
    // are rebuilt in order, so an earlier page's staged bytes may be
    // overwritten once used).
    for (auto& c : chunks) {
        if (!stream_packed || c.packed) continue;
        c.pk_bytes = 0;
        for (uint32_t p = c.first_page; p < c.end_page; ++p) c.pk_bytes += staged_bytes(g->pages[p]);
        if (c.pk_bytes >= c.s_bytes || c.pk_bytes > slot_bytes) continue;
        c.stage_off = (slot_bytes - c.pk_bytes) & ~255ull;
        bool fits = true;
        uint64_t rel = 0;
        for (uint32_t p = c.first_page; p < c.end_page && fits; ++p) {
            const PageMeta& pm = g->pages[p];
            fits = (pm.s_off - c.s_begin) + pm.s_bytes <= c.stage_off + rel;
            rel += staged_bytes(pm);
        }
        c.decode = fits;
    }
    const uint32_t C = (uint32_t)chunks.size();
    const bool resident = C <= R;
    const uint32_t Weff = W < C ? W : C;
    const uint32_t nslots = resident ? C : R;

    std::vector<uint64_t> rel_soff(g->num_pages), rel_woff(g->num_pages), offb(g->num_pages);
    for (const Chunk& c : chunks)
        for (uint32_t p = c.first_page; p < c.end_page; ++p) {
            rel_soff[p] = (c.packed ? g->pages[p].pk_off : g->pages[p].s_off) - c.s_begin;
            rel_woff[p] = c.w_slot_off + (g->pages[p].w_off - c.w_begin);
            offb[p] = g->pages[p].off_bytes;
        }
    // list capacity: the most vertices any W consecutive chunks hold
    uint64_t max_win_v = 1;
    for (uint32_t t = 0; t < C; ++t) {
        uint64_t s = 0;
        for (uint32_t k = 0; k < Weff; ++k) {
            const Chunk& c = chunks[(t + k) % C];
            s += c.v_end - c.v_begin;
        }
        max_win_v = std::max<uint64_t>(max_win_v, s);
    }
    // step ring (per-step events, change counts and bookkeeping, indexed by
    // step modulo its size): more steps than a sweep plus its look-ahead
    uint32_t ring = 64;
    while (ring < 4 * (uint64_t)C + 8) ring <<= 1;

    // --------------------------------------------------------- allocations
    Stream cs, xs, ds;  // compute, copies, decode of packed-streamed chunks
    cs.use(P->stream);
    xs.create();
    if (stream_packed) ds.create();
    DevBuf<uint8_t> ebuf;
    DevBuf<unsigned long long> lists;
    DevBuf<uint32_t> val, caller_order;
    DevBuf<float> x, contrib, x_next, x_prev, inv_out;
    DevBuf<uint8_t> state;
    DevBuf<uint32_t> stamp, front0, front1, big;
    DevBuf<uint8_t> small;
    PinnedBuf small_h;
    // borrow the graph's kept buffers for this run (given back on every exit)
    struct Lease {
        RunWorkspace* ws = nullptr;
        DevBuf<uint8_t>* ebuf; DevBuf<unsigned long long>* lists; DevBuf<uint32_t>* val;
        DevBuf<uint32_t>* out; DevBuf<float>* f[5]; DevBuf<uint8_t>* state; DevBuf<uint32_t>* pu[4];
        DevBuf<uint8_t>* small; PinnedBuf* small_h;
        ~Lease() {
            if (!ws) return;
            ws->ebuf = std::move(*ebuf); ws->lists = std::move(*lists); ws->val = std::move(*val);
            ws->out = std::move(*out); ws->x = std::move(*f[0]); ws->contrib = std::move(*f[1]);
            ws->x_next = std::move(*f[2]); ws->x_prev = std::move(*f[3]);
            ws->inv_out = std::move(*f[4]); ws->state = std::move(*state);
            ws->stamp = std::move(*pu[0]); ws->front0 = std::move(*pu[1]);
            ws->front1 = std::move(*pu[2]); ws->big = std::move(*pu[3]);
            ws->small = std::move(*small); ws->small_h = std::move(*small_h);
            ws->m.unlock();
        }
    } lease{nullptr, &ebuf, &lists, &val, &caller_order, {&x, &contrib, &x_next, &x_prev, &inv_out}, &state,
            {&stamp, &front0, &front1, &big}, &small, &small_h};
    if (g->ws.m.try_lock()) {
        RunWorkspace& w = g->ws;
        ebuf = std::move(w.ebuf); lists = std::move(w.lists); val = std::move(w.val);
        caller_order = std::move(w.out); x = std::move(w.x); contrib = std::move(w.contrib);
        x_next = std::move(w.x_next); x_prev = std::move(w.x_prev); inv_out = std::move(w.inv_out);
        state = std::move(w.state);
        stamp = std::move(w.stamp); front0 = std::move(w.front0); front1 = std::move(w.front1);
        big = std::move(w.big);
        small = std::move(w.small); small_h = std::move(w.small_h);
        lease.ws = &w;
    }
    auto ensure = [](auto& buf, size_t count) { if (buf.n < count) buf.alloc(count); };
    ensure(ebuf, slot_bytes * nslots);
    // The run's small buffers, carved out of one device and one pinned
    // allocation kept with the graph: after a graph's first run nothing is
    // allocated, so a run issued while other work (say the read-back of the
    // previous run's values) is in flight does not wait for it.
    const int nparts = device_sms() * 4;
    const uint64_t big_cap = std::min<uint64_t>(n, g->m / kPushWarpMax + 1);
    uint64_t dsz = 0, hsz = 0;
    auto carve = [](uint64_t& at, uint64_t bytes) { const uint64_t o = at; at = align_up(at + bytes, 256); return o; };
    const uint64_t o_loc = carve(dsz, sizeof(PageLoc) * g->num_pages);
    const uint64_t o_rel = carve(dsz, 3 * 8ull * g->num_pages);
    const uint64_t o_rs = carve(dsz, sizeof(RunState));
    const uint64_t o_rep = carve(dsz, sizeof(SweepReport));
    const uint64_t o_steps = carve(dsz, 4ull * ring);
    const uint64_t o_part = carve(dsz, 3 * 8ull * nparts);
    const uint64_t o_dirty = carve(dsz, 32 * 4);
    const uint64_t o_ps = carve(dsz, sizeof(PushState));
    const uint64_t oh_rep = carve(hsz, sizeof(SweepReport));
    const uint64_t oh_steps = carve(hsz, 4ull * ring);
    const uint64_t oh_ps = carve(hsz, sizeof(PushState));
    ensure(small, dsz);
    if (small_h.bytes < hsz) small_h.alloc(hsz);
    Slice<PageLoc> loc{(PageLoc*)(small.p + o_loc)};
    Slice<uint64_t> d_rel_soff{(uint64_t*)(small.p + o_rel)};
    Slice<uint64_t> d_rel_woff{d_rel_soff.p + g->num_pages}, d_offb{d_rel_soff.p + 2 * g->num_pages};
    SR_CUDA(cudaMemcpyAsync(d_rel_soff.p, rel_soff.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    SR_CUDA(cudaMemcpyAsync(d_rel_woff.p, rel_woff.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    SR_CUDA(cudaMemcpyAsync(d_offb.p, offb.data(), 8 * g->num_pages, cudaMemcpyHostToDevice, cs.s));
    ensure(lists, (uint64_t)kClasses * max_win_v);
    Slice<RunState> rs{(RunState*)(small.p + o_rs)};
    Slice<SweepReport> d_rep{(SweepReport*)(small.p + o_rep)};
    Slice<unsigned> d_steps{(unsigned*)(small.p + o_steps)};
    SR_CUDA(cudaMemsetAsync(d_steps.p, 0, ring * sizeof(unsigned), cs.s));
    Slice<uint8_t> h_rep{small_h.p + oh_rep}, h_steps{small_h.p + oh_steps}, h_ps{small_h.p + oh_ps};
    Slice<double> partial{(double*)(small.p + o_part)};
    if (is_pr) {
        ensure(x, n); ensure(contrib, n); ensure(x_next, n); ensure(x_prev, n); ensure(inv_out, n);
    } else {
        ensure(val, n);
    }
    if (P->pvu == SERAPH_PVU_WEAK) ensure(state, n);
    const bool push_on = P->push != 0;
    SR_CHECK(P->count_clean <= 1, SERAPH_EINVAL, "count_clean must be 0 or 1");
    const bool count_clean = P->count_clean != 0 && !is_pr;
    Slice<uint32_t> dirty_blocks{count_clean ? (uint32_t*)(small.p + o_dirty) : nullptr};
    Slice<PushState> d_ps{push_on ? (PushState*)(small.p + o_ps) : nullptr};
    if (push_on || count_clean) {
        ensure(stamp, n);
        SR_CUDA(cudaMemsetAsync(stamp.p, 0, n * sizeof(uint32_t), cs.s));
    }
    if (push_on) {
        ensure(front0, n); ensure(front1, n); ensure(big, big_cap);
    }
    const uint64_t push_below = P->push_below ? P->push_below : std::max<uint64_t>(n / 256, 1);

    AlgoArgs a{};
    a.val = is_pr ? nullptr : val.p;  // (borrowed buffers of other algorithms stay unused)
    a.x = is_pr ? x.p : nullptr;
    a.contrib = is_pr ? contrib.p : nullptr;
    a.x_next = is_pr ? x_next.p : nullptr;
    a.inv_out = is_pr ? inv_out.p : nullptr;
    a.state = P->pvu == SERAPH_PVU_WEAK ? state.p : nullptr;
    a.rs = rs.p;
    a.loc = loc.p;
    a.vb = g->d_vb.p;
    for (int k = 0; k < kClasses; ++k) a.list[k] = lists.p + k * max_win_v;
    a.step_changed = d_steps.p;
    a.step_mask = ring - 1;
    a.cls_max[0] = P->thread_max_deg;
    a.cls_max[1] = P->group4_max_deg;
    a.cls_max[2] = P->group8_max_deg;
    a.cls_max[3] = P->warp_max_deg;
    a.damping = (float)P->damping;
    a.fail_eps = (float)P->pr_fail_eps;
    // over-relaxation runs while the last sweep changed the values by at least
    // pr_pvu_off_below (L1); the sweeps after that publish plain updates, so
    // no vertex keeps an overshoot from its last over-relaxed update
    const float omega0 = (P->pr_omega == 0.0 || P->pr_omega == 1.0) ? 1.0f : (float)P->pr_omega;
    a.omega = omega0;
    a.fsm_bits = 0;
    for (int i = 0; i < 12; ++i) a.fsm_bits |= (uint64_t)P->fsm_next[i] << (3 * i);
    a.skip_mask = P->fsm_skip_mask;
    a.pvu = (uint8_t)P->pvu;
    a.wbytes = (uint8_t)g->wbytes;
    a.packed = packed;
    a.n = (uint32_t)n;
    a.chg_stamp = push_on || count_clean ? stamp.p : nullptr;
    a.chg_tag = 1;
    {
        uint64_t hot_bytes = P->l2_hot_bytes;
        if (hot_bytes == SERAPH_L2_HOT_AUTO) {
            int l2 = 0;
            SR_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device));
            hot_bytes = (uint64_t)l2 * 3 / 8;  // measured best at R-MAT-28: 32-48 MB of 126
        }
        a.hints = hot_bytes > 0;
        a.hot = (uint32_t)std::min<uint64_t>(n, hot_bytes / 4);
        // set-aside = the hot range (measured: a larger set-aside starves the
        // normal lines -- 5/3 of 48 MB cost 8 % of PageRank's relax time)
        if (a.hints) l2_setaside_hold(g, g->device, (uint64_t)a.hot * 4);
    }

    uint64_t launches = 0;
    {
        RunState init{};
        init.thr_cur = SERAPH_INF;
        init.thr_prev = 0;  // the initial values count as sweep-0 writes (minimum 0)
        SR_CUDA(cudaMemcpyAsync(rs.p, &init, sizeof(init), cudaMemcpyHostToDevice, cs.s));
        if (is_pr) {
            launch_init_pr(g->d_outdeg.p, a, x_prev.p, n, cs.s);
            launch_close_pr(a, n, x_prev.p, P->damping, partial.p, nparts, nullptr, false, cs.s);
            launches += 3;
        } else {
            uint32_t source = P->source;
            if (g->reordered && algo != SERAPH_CC) {  // the caller's source id -> internal id
                SR_CUDA(cudaMemcpyAsync(h_steps.p, g->d_inv.p + source, 4, cudaMemcpyDeviceToHost, cs.s));
                SR_CUDA(cudaStreamSynchronize(cs.s));
                std::memcpy(&source, h_steps.p, 4);
            }
            launch_init_values(algo, a, n, source, g->reordered ? g->d_perm.p : nullptr, cs.s);
            launches += 1;
        }
        SR_CUDA(cudaStreamSynchronize(cs.s));
    }

    // -------------------------------------------------------------- events
    // staged[p]: page p's compact bytes are in its slot (the rebuild of a
    // page waits for its own copies, not for the whole chunk's)
    std::vector<Event> step_done(ring), copy_done(C), staged(g->num_pages);
    std::vector<uint32_t> npass_of(ring, 0);
    for (auto& e : step_done) e.create(false);
    for (auto& e : copy_done) e.create(false);
    for (const Chunk& c : chunks)
        if (c.decode)
            for (uint32_t p = c.first_page; p < c.end_page; ++p) staged[p].create(false);
    Event ev_start, ev_stop, ev_sweep;
    ev_start.create(true);
    ev_stop.create(true);
    ev_sweep.create(false);
    const bool prof = P->profile != 0;
    // a learned step may run up to 16 passes unless max_passes says otherwise
    const uint32_t max_passes =
        learned && P->max_passes == 0 ? 16u : std::max(P->max_passes, P->passes);
    // profiling pools, indexed by step within the ring
    std::vector<Event> pc_b, pc_e, pk_b, pk_e, pr_b, pr_e;
    if (prof) {
        for (auto* v : {&pc_b, &pc_e, &pk_b, &pk_e}) {
            v->resize(ring);
            for (auto& e : *v) e.create(true);
        }
        for (auto* v : {&pr_b, &pr_e}) {
            v->resize((size_t)ring * max_passes);
            for (auto& e : *v) e.create(true);
        }
    }

    seraph_stats S{};
    S.chunks = C;
    S.resident = resident;

    std::vector<int64_t> slot_of(C, -1);        // chunk -> slot
    std::vector<int64_t> chunk_in(nslots, -1);   // slot -> chunk
    std::vector<int64_t> last_use(nslots, -1);   // slot -> last step that used it
    std::vector<uint8_t> pending(C, 0);          // copied but not yet waited on by compute
    uint32_t load_seq = 0, loads_timed = 0;
    const bool zig_base = !resident && P->order == SERAPH_ORDER_ZIGZAG;
    Schedule sched = learned ? Schedule(C, zig_base) : Schedule(C, W, (int)P->order, resident);
    const bool zig = zig_base;

    // Look-ahead over the deterministic window sequence: next step >= from
    // whose window holds chunk c (or `horizon` if none within it).
    const uint64_t horizon_len = 2 * (uint64_t)C + 2;
    auto next_use = [&](uint32_t c, uint64_t from, uint64_t horizon) -> uint64_t {
        for (uint64_t u = from; u < horizon; ++u)
            for (uint32_t x : sched.window(u))
                if (x == c) return u;
        return horizon;
    };

    // Eviction choices.  Steps <= t are enqueued; steps > t are not.
    //  - demand (chunk needed by step t itself): an empty slot, else the
    //    resident chunk outside window t with the furthest next use;
    //  - cyclic prefetch for step t+1: the chunk outside windows t and t+1
    //    with the furthest next use (the classic ring: the chunk that just
    //    left the window);
    //  - zigzag prefetch for a later step u: exactly the chunk furthest-next-
    //    use eviction would pick when step u arrives, and only if no step in
    //    [t, u) still needs it (otherwise stop prefetching for now).
    auto take = [&](int64_t s) {
        slot_of[chunk_in[s]] = -1;
        chunk_in[s] = -1;
        return s;
    };
    auto empty_slot = [&]() -> int64_t {
        for (uint32_t s = 0; s < nslots; ++s)
            if (chunk_in[s] < 0) return s;
        return -1;
    };
    auto slot_demand = [&](uint64_t t) -> int64_t {
        const int64_t e = empty_slot();
        if (e >= 0) return e;
        const std::vector<uint32_t>& win_t = sched.window(t);
        int64_t best = -1;
        uint64_t best_next = 0;
        for (uint32_t s = 0; s < nslots; ++s) {
            bool in_win = false;
            for (uint32_t c : win_t) in_win |= chunk_in[s] == (int64_t)c;
            if (in_win) continue;
            const uint64_t nu = next_use((uint32_t)chunk_in[s], t, t + horizon_len);
            if (best < 0 || nu > best_next) { best = s; best_next = nu; }
        }
        SR_CHECK(best >= 0, SERAPH_EINVAL, "schedule error: no slot to evict");
        return take(best);
    };
    auto slot_prefetch = [&](uint64_t t, uint64_t u) -> int64_t {
        const int64_t e = empty_slot();
        if (e >= 0) return e;
        const uint64_t horizon = t + horizon_len;
        if (!zig) {  // candidates: not used by steps t..u
            int64_t best = -1;
            uint64_t best_next = 0;
            for (uint32_t s = 0; s < nslots; ++s) {
                const uint64_t nu = next_use((uint32_t)chunk_in[s], t, horizon);
                if (nu <= u) continue;
                if (best < 0 || nu > best_next) { best = s; best_next = nu; }
            }
            return best < 0 ? -1 : take(best);
        }
        int64_t best = -1;
        uint64_t best_next = 0;
        for (uint32_t s = 0; s < nslots; ++s) {
            const uint64_t nu = next_use((uint32_t)chunk_in[s], u, horizon);
            if (best < 0 || nu > best_next) { best = s; best_next = nu; }
        }
        if (best < 0 || best_next <= u) return -1;
        if (next_use((uint32_t)chunk_in[best], t, u) < u) return -1;  // still needed before u
        return take(best);
    };

    // copy chunk c into `slot` on the copy stream, during step t
    // chunk last loaded into each slot: a decode on the side stream may still
    // be writing it when the slot is reloaded without a step having used it
    std::vector<int64_t> slot_load(nslots, -1);
    auto load = [&](uint32_t c, int64_t slot, uint64_t t) {
        if (last_use[slot] >= 0) SR_CUDA(cudaStreamWaitEvent(xs.s, step_done[last_use[slot] % ring].e, 0));
        if (slot_load[slot] >= 0 && chunks[slot_load[slot]].decode)
            SR_CUDA(cudaStreamWaitEvent(xs.s, copy_done[slot_load[slot]].e, 0));
        const Chunk& ch = chunks[c];
        uint8_t* sb = ebuf.p + (uint64_t)slot * slot_bytes;
        if (prof) SR_CUDA(cudaEventRecord(pc_b[(load_seq + 1) % ring].e, xs.s));
        cudaStream_t fin = xs.s;  // the stream that finishes the load
        if (ch.decode) {
            // each page's streamed header and gap stream to the far end of
            // the slot, then (on the decode stream, so the copy engine moves
            // on) each page rebuilt in its plain place as soon as its own
            // bytes have landed, in page order
            uint64_t rel = 0;
            for (uint32_t p = ch.first_page; p < ch.end_page; ++p) {
                const PageMeta& pm = g->pages[p];
                uint8_t* dst = sb + ch.stage_off + rel;
                SR_CUDA(cudaMemcpyAsync(dst, g->h_shdr.p + pm.sh_off, pm.sh_bytes,
                                        cudaMemcpyHostToDevice, xs.s));
                if (pm.pk_data)
                    SR_CUDA(cudaMemcpyAsync(dst + pm.sh_bytes, g->h_pack.p + pm.pk_off + 2 * pm.off_bytes,
                                            align_up(pm.pk_data, 16), cudaMemcpyHostToDevice, xs.s));
                SR_CUDA(cudaEventRecord(staged[p].e, xs.s));
                SR_CUDA(cudaStreamWaitEvent(ds.s, staged[p].e, 0));
                launch_decode_page(dst, sb + (pm.s_off - ch.s_begin), (uint32_t)pm.nv, pm.sh_nesc,
                                   pm.off_bytes, pm.s_bytes, ds.s);
                rel += staged_bytes(pm);
                ++launches;
            }
            fin = ds.s;
        } else {
            SR_CUDA(cudaMemcpyAsync(sb, (ch.packed ? g->h_pack.p : g->h_struct.p) + ch.s_begin,
                                    ch.s_bytes, cudaMemcpyHostToDevice, xs.s));
        }
        // (copy_ms counts the copies on the copy stream: a decoded chunk's
        // weights, copied after its decode, are not in it)
        if (prof && ch.decode) SR_CUDA(cudaEventRecord(pc_e[(load_seq + 1) % ring].e, xs.s));
        // weights after the decode (they may overlap the packed staging bytes)
        if (use_w && ch.w_bytes)
            SR_CUDA(cudaMemcpyAsync(sb + ch.w_slot_off, g->h_weight.p + ch.w_begin, ch.w_bytes,
                                    cudaMemcpyHostToDevice, fin));
        if (prof && !ch.decode) SR_CUDA(cudaEventRecord(pc_e[(load_seq + 1) % ring].e, fin));
        launch_set_locs(loc.p, g->d_vb.p, ch.first_page, ch.end_page, d_rel_soff.p, d_rel_woff.p,
                        d_offb.p, sb, use_w ? sb : nullptr, ch.packed, rs.p, ++load_seq, fin);
        ++launches;
        SR_CUDA(cudaEventRecord(copy_done[c].e, fin));
        slot_load[slot] = (int64_t)c;
        slot_of[c] = slot;
        chunk_in[slot] = c;
        pending[c] = 1;
        S.bytes_streamed += (ch.decode ? ch.pk_bytes : ch.s_bytes) + (use_w ? ch.w_bytes : 0);
    };

    const unsigned relax_grid = device_sms() * 8;
    // learned scheduler / trace state
    const bool track = learned || trace;
    DevBuf<ChunkStatic> d_cs;
    DevBuf<ChunkDyn> d_cd;
    DevBuf<float> rec_feat, d_feats, d_prio;
    DevBuf<unsigned> rec_gain;
    DevBuf<int32_t> d_kp;
    PinnedBuf h_feat, h_gain, h_prio;
    const uint32_t rec_rows = C + W + 2;
    if (track) {
        std::vector<ChunkStatic> cs_h(C);
        for (uint32_t c = 0; c < C; ++c) {
            ChunkStatic x{};
            x.nv = (float)(chunks[c].v_end - chunks[c].v_begin);
            float ne = 0.f, md = 0.f;
            for (uint32_t p = chunks[c].first_page; p < chunks[c].end_page; ++p) {
                ne += (float)g->pages[p].ne;
                md = std::max(md, (float)g->pages[p].maxdeg);
            }
            x.ne = ne;
            x.maxdeg = md;
            x.bytes_frac = (float)(chunks[c].s_bytes + (use_w ? chunks[c].w_bytes : 0)) / (float)slot_bytes;
            cs_h[c] = x;
        }
        d_cs.alloc(C);
        d_cd.alloc(C);
        SR_CUDA(cudaMemcpy(d_cs.p, cs_h.data(), C * sizeof(ChunkStatic), cudaMemcpyHostToDevice));
        SR_CUDA(cudaMemset(d_cd.p, 0, C * sizeof(ChunkDyn)));
        rec_feat.alloc((uint64_t)rec_rows * kSchedIn);
        rec_gain.alloc((uint64_t)rec_rows * 16);
        SR_CUDA(cudaMemset(rec_gain.p, 0, (uint64_t)rec_rows * 16 * sizeof(unsigned)));
        h_feat.alloc((uint64_t)rec_rows * kSchedIn * sizeof(float));
        h_gain.alloc((uint64_t)rec_rows * 16 * sizeof(unsigned));
        if (learned) {
            d_feats.alloc((uint64_t)C * kSchedIn);
            d_prio.alloc(C);
            d_kp.alloc(C);
            h_prio.alloc(C * sizeof(float));
        }
        if (trace) trace->count = 0;
    }
    SchedArgs sa{};
    sa.cs = d_cs.p;
    sa.cd = d_cd.p;
    sa.rs = rs.p;
    sa.inv_n = (float)(1.0 / (double)n);
    sa.is_pr = is_pr ? 1.f : 0.f;
    uint32_t skip_streak = 0;  // consecutive learned sweeps that skipped chunks
    uint32_t pass = 0;
    bool predict = P->pvu != SERAPH_PVU_OFF;
    bool pr_predict_off = false;
    int rc = SERAPH_OK;
    std::vector<int64_t> proc_step(C, -1);  // last prediction-off step that processed a chunk
    // tag of the last sweep in which a chunk was processed with every vertex
    // relaxed or final (prediction off, or strong conditions); 0 = none yet
    std::vector<uint32_t> valid_tag(C, 0);
    int64_t last_change = -1;               // last step with a value change (init = step -1)
    uint64_t sweep_first_step = 0;
    std::vector<uint8_t> pred_in_step(ring, 0);
    std::vector<std::vector<uint32_t>> window_of(ring);
    uint32_t npass = P->passes;

    SR_CUDA(cudaStreamSynchronize(cs.s));
    SR_CUDA(cudaEventRecord(ev_start.e, xs.s));
    std::vector<uint32_t> seq_of(C, 0);  // load sequence number of each chunk
    for (uint64_t t = 0;; ++t) {
        const std::vector<uint32_t>& win = sched.window(t);
        a.chg_tag = S.sweeps + 1;  // value changes of this sweep carry its tag
        // (0) anything step t needs that could not be prefetched
        for (uint32_t c : win)
            if (slot_of[c] < 0) {
                load(c, slot_demand(t), t);
                seq_of[c] = load_seq;
            }
        // (1) prefetch: the next step (cyclic), or as far ahead as the
        // eviction rule allows (zigzag), so the copy engine keeps streaming
        const uint64_t reach = zig ? t + horizon_len : t + 2;
        bool stop_prefetch = false;
        for (uint64_t u = t + 1; u < reach && !stop_prefetch; ++u)
            for (uint32_t c : sched.window(u)) {
                if (slot_of[c] >= 0) continue;
                const int64_t slot = slot_prefetch(t, u);
                if (slot < 0) { stop_prefetch = true; break; }
                load(c, slot, t);
                seq_of[c] = load_seq;
            }
        // idle-slot passes of this step run while the next step's data is in flight
        bool prefetch = false;
        uint32_t want = 0;
        for (uint32_t c : sched.window(t + 1))
            if (pending[c]) { prefetch = true; want = std::max(want, seq_of[c]); }
        // (2) passes over the window
        for (uint32_t c : win) {
            SR_CHECK(slot_of[c] >= 0, SERAPH_EINVAL, "schedule error: window chunk not resident");
            if (pending[c]) {
                SR_CUDA(cudaStreamWaitEvent(cs.s, copy_done[c].e, 0));
                pending[c] = 0;
            }
        }
        if (prof) SR_CUDA(cudaEventRecord(pk_b[t % ring].e, cs.s));
        WindowDesc wd{};
        {
            uint32_t blocks = 0;
            for (size_t k = 0; k < win.size(); ++k) {
                const Chunk& ch = chunks[win[k]];
                ChunkDesc& d = wd.c[k];
                d.v_begin = ch.v_begin;
                d.v_end = ch.v_end;
                d.first_page = ch.first_page;
                d.end_page = ch.end_page;
                d.block_begin = blocks;
                blocks += (uint32_t)((uint64_t(ch.v_end - ch.v_begin) + 1023) / 1024);
            }
            wd.nchunks = (uint32_t)win.size();
            wd.nblocks = blocks;
        }
        const bool pred_now = is_pr ? (predict && !pr_predict_off) : predict;
        npass = max_passes > P->passes && (prefetch || learned) ? max_passes : P->passes;
        const uint64_t row = t - sweep_first_step;
        unsigned* rec_row = track && row < rec_rows ? rec_gain.p + row * 16 : nullptr;
        if (track) {
            sa.predict = pred_now ? 1.f : 0.f;
            sa.sweep = (float)S.sweeps;
            launch_sched_step(sa, rs.p, win[0], rec_row ? rec_feat.p + row * kSchedIn : nullptr,
                              learned ? model : nullptr, cs.s);
            ++launches;
        }
        for (uint32_t j = 0; j < npass; ++j) {
            const bool idle = j >= P->passes && !learned;
            launch_gate(rs.p, pass, j > 0, idle && prefetch, want, j, learned ? 1 : 0,
                        j < 16 ? rec_row : nullptr, cs.s);
            launch_compact(algo, wd, a, pass, pred_now ? 1 : 0, cs.s);
            if (prof) SR_CUDA(cudaEventRecord(pr_b[(t % ring) * max_passes + j].e, cs.s));
            {
                AlgoArgs ap = a;
                ap.packed = chunks[win[0]].packed;  // windows hold one form (hybrid needs W = 1)
                // every vertex with level <= k is final after k sweeps (strong prediction
                // skips them), so an attempted vertex's level is at least k + 1; without
                // prediction only the source has level 0
                ap.bfs_lb = (pred_now && P->pvu == SERAPH_PVU_STRONG) ? (uint32_t)S.sweeps + 1u : 1u;
                launch_relax(algo, P->kahan, ap, pass, (uint32_t)t, relax_grid, cs.s);
            }
            if (prof) SR_CUDA(cudaEventRecord(pr_e[(t % ring) * max_passes + j].e, cs.s));
            launches += 3;
            S.relax_launches += 1;
            if (is_pr) {
                launch_pr_apply(a, pass, relax_grid, cs.s);
                ++launches;
            }
            ++pass;
        }
        if (track) {
            launch_step_epilogue(rs.p, d_cd.p, win[0], pass - 1, std::min<uint32_t>(npass, 16), rec_row, cs.s);
            ++launches;
        }
        if (prof) SR_CUDA(cudaEventRecord(pk_e[t % ring].e, cs.s));
        SR_CUDA(cudaEventRecord(step_done[t % ring].e, cs.s));
        for (uint32_t c : win) last_use[slot_of[c]] = (int64_t)t;
        pred_in_step[t % ring] = pred_now;
        window_of[t % ring] = win;
        npass_of[t % ring] = npass;
        S.steps += 1;
        if (!sched.sweep_end(t)) continue;

        // ---------------------------------------------------- sweep close
        if (is_pr)
            launch_close_pr(a, n, x_prev.p, P->damping, partial.p, nparts, d_rep.p,
                            P->pr_normalize != 0, cs.s);
        else {
            if (count_clean) {
                launch_count_clean(stamp.p, n, S.sweeps + 1, g->src_block, g->d_page_blocks.p,
                                   g->num_pages, dirty_blocks.p, rs.p, cs.s);
                launches += 2;
            }
            launch_close_min(rs.p, d_rep.p, cs.s);
        }
        launches += is_pr ? (P->pr_normalize ? 4 : 2) : 1;
        SR_CUDA(cudaMemcpyAsync(h_rep.p, d_rep.p, sizeof(SweepReport), cudaMemcpyDeviceToHost, cs.s));
        SR_CUDA(cudaMemcpyAsync(h_steps.p, d_steps.p, ring * sizeof(unsigned), cudaMemcpyDeviceToHost, cs.s));
        const uint64_t rows_now = std::min<uint64_t>(t + 1 - sweep_first_step, rec_rows);
        if (trace) {
            SR_CUDA(cudaMemcpyAsync(h_feat.p, rec_feat.p, rows_now * kSchedIn * sizeof(float), cudaMemcpyDeviceToHost, cs.s));
            SR_CUDA(cudaMemcpyAsync(h_gain.p, rec_gain.p, rows_now * 16 * sizeof(unsigned), cudaMemcpyDeviceToHost, cs.s));
        }
        if (learned) {
            sa.predict = predict ? 1.f : 0.f;
            sa.sweep = (float)(S.sweeps + 1);
            launch_sched_features(sa, C, d_feats.p, cs.s);
            model->infer(d_feats.p, C, d_kp.p, d_prio.p, cs.s);
            SR_CUDA(cudaMemcpyAsync(h_prio.p, d_prio.p, C * sizeof(float), cudaMemcpyDeviceToHost, cs.s));
            launches += 2;
        }
        if (track) SR_CUDA(cudaMemsetAsync(rec_gain.p, 0, (uint64_t)rec_rows * 16 * sizeof(unsigned), cs.s));
        SR_CUDA(cudaEventRecord(ev_sweep.e, cs.s));
        wait_event(ev_sweep.e, P->timeout_ms);
        SweepReport rep;
        std::memcpy(&rep, h_rep.p, sizeof(rep));
        const unsigned* steps_changed = (const unsigned*)h_steps.p;
        for (uint64_t s = sweep_first_step; s <= t; ++s) {
            if (steps_changed[s % ring]) last_change = (int64_t)s;
            if (!pred_in_step[s % ring] || !P->verify)
                for (uint32_t c : window_of[s % ring]) proc_step[c] = (int64_t)s;
            // every vertex of the chunk relaxed or final (for the push stage);
            // strong skips count as final where every sweep visits every chunk
            // (not zigzag; the learned mode skips chunks only with verify = 1)
            if (!pred_in_step[s % ring] ||
                (P->pvu == SERAPH_PVU_STRONG && !zig && !(learned && P->verify)))
                for (uint32_t c : window_of[s % ring]) valid_tag[c] = S.sweeps + 1;
        }
        // clear the ring entries of this sweep for reuse
        SR_CUDA(cudaMemsetAsync(d_steps.p, 0, ring * sizeof(unsigned), cs.s));
        S.sweeps += 1;
        S.passes_run += rep.passes_run;
        S.passes_skipped += rep.passes_skipped;
        S.edges_relaxed += rep.edges;
        S.packed_edges += rep.packed_edges;
        S.clean_pages += rep.clean_pages;
        S.code_bytes += rep.code_bytes;
        S.vertices_attempted += rep.attempted;
        S.vertices_skipped += rep.skipped;
        S.changes += rep.changed;
        if (!pred_now) S.verify_sweeps += 1;
        if (prof) {
            for (uint64_t s = sweep_first_step; s <= t; ++s) {
                S.compute_ms += elapsed(pk_b[s % ring].e, pk_e[s % ring].e);
                for (uint32_t j = 0; j < npass_of[s % ring]; ++j) {
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, pr_b[(s % ring) * max_passes + j].e,
                                             pr_e[(s % ring) * max_passes + j].e) == cudaSuccess)
                        S.relax_ms += ms;
                    else
                        (void)cudaGetLastError();
                }
            }
            // every finished load (the prefetch for the next sweep may still run)
            while (loads_timed < load_seq && cudaEventQuery(pc_e[(loads_timed + 1) % ring].e) == cudaSuccess) {
                ++loads_timed;
                S.copy_ms += elapsed(pc_b[loads_timed % ring].e, pc_e[loads_timed % ring].e);
            }
        }
        if (trace) {
            for (uint64_t r = 0; r < rows_now && trace->count < trace->capacity; ++r) {
                const uint64_t o = trace->count++;
                std::memcpy(trace->features + o * kSchedIn, (const float*)h_feat.p + r * kSchedIn,
                            kSchedIn * sizeof(float));
                std::memcpy(trace->gains + o * 16, (const unsigned*)h_gain.p + r * 16, 16 * sizeof(unsigned));
                const Chunk& ch = chunks[sched.window(sweep_first_step + r)[0]];
                if (trace->vertices) trace->vertices[o] = ch.v_end - ch.v_begin;
            }
        }
        sweep_first_step = t + 1;
        bool stop = false;
        if (is_pr) {
            S.residual = rep.resid;
            if (!pred_now && rep.resid < P->tol) { S.converged = 1; stop = true; }
            else if (pred_now && rep.resid < std::max(P->pr_pvu_off_below, P->tol)) pr_predict_off = true;
            if (rep.resid < P->pr_pvu_off_below) a.omega = 1.0f;
            if (!stop && S.sweeps >= P->max_sweeps) stop = true;
        } else {
            bool all_after = true;
            for (uint32_t c = 0; c < C; ++c) all_after &= proc_step[c] > last_change;
            if (all_after) {
                S.converged = 1;
                stop = true;
                if (rep.overflow) rc = SERAPH_EOVERFLOW;
            } else if (rep.changed == 0) {
                predict = false;  // a predicted sweep changed nothing: retrieve with all-pull
            } else {
                predict = P->pvu != SERAPH_PVU_OFF;
            }
            // dense -> sparse switch.  Every chunk was last processed with all of
            // its vertices relaxed or final in sweep valid_tag[c] or later, so an
            // edge can be violated only if its source changed since the earliest
            // of those sweeps (tag_first): those vertices start the push stage.
            // (Zigzag orders skip a sweep's boundary chunk in the next sweep, so
            // tag_first may lie one sweep back.)
            const uint32_t tag_first = *std::min_element(valid_tag.begin(), valid_tag.end());
            if (!stop && push_on && !S.push_sweep && rep.changed > 0 && rep.changed <= push_below &&
                tag_first > 0) {
                S.push_sweep = S.sweeps;
                PushArgs pa{};
                pa.out_off = g->h_out_off.device_ptr<uint64_t>();
                pa.out_col = g->h_out_col.device_ptr<uint32_t>();
                pa.out_w = use_w ? g->h_out_w.device_ptr<uint8_t>() : nullptr;
                pa.wbytes = g->wbytes;
                pa.n = (uint32_t)n;
                pa.val = val.p;
                pa.stamp = stamp.p;
                pa.front[0] = front0.p;
                pa.front[1] = front1.p;
                pa.big = big.p;
                pa.big_cap = (uint32_t)big_cap;
                pa.ps = d_ps.p;
                const uint32_t tag_last = S.sweeps;  // the tag of the sweep that just closed
                launch_push_frontier(pa, tag_first, cs.s);
                launches += 1;
                PushState hps{};
                const int ialgo = algo == SERAPH_SSSP ? ALG_SSSP : algo == SERAPH_BFS ? ALG_BFS : ALG_CC;
                for (uint32_t r = 0;;) {
                    // rounds in batches of 8 (a round after the frontier ran dry does nothing)
                    for (int k = 0; k < 8; ++k, ++r) launch_push_round(ialgo, pa, r, tag_last + 1 + r, cs.s);
                    launches += 8 * 3;
                    SR_CUDA(cudaMemcpyAsync(h_ps.p, d_ps.p, sizeof(PushState), cudaMemcpyDeviceToHost, cs.s));
                    SR_CUDA(cudaEventRecord(ev_sweep.e, cs.s));
                    wait_event(ev_sweep.e, P->timeout_ms);
                    std::memcpy(&hps, h_ps.p, sizeof(hps));
                    if (hps.cnt[r & 1] == 0) break;
                    SR_CHECK(r < n + 16, SERAPH_ENOTCONV, "push stage: no fixpoint after n rounds");
                }
                S.push_rounds = hps.rounds;
                S.push_edges = hps.edges;
                S.changes += hps.changes;
                if (!hps.ovf) {
                    S.converged = 1;
                    stop = true;
                } else {
                    // a candidate overflowed: a prediction-off pull sweep over every
                    // chunk decides SERAPH_EOVERFLOW as without the push stage
                    predict = false;
                    last_change = (int64_t)t;
                }
            }
            if (!stop && S.sweeps >= P->max_sweeps) { rc = SERAPH_ENOTCONV; stop = true; }
        }
        if (stop) break;
        if (learned) {  // the next sweep's order, without chunks predicted idle
            const float* pr = (const float*)h_prio.p;
            std::vector<uint32_t> ord(C);
            std::iota(ord.begin(), ord.end(), 0u);
            if (zig_base && (S.sweeps & 1)) std::reverse(ord.begin(), ord.end());
            // SSSP/BFS/CC: the chunks already in the ring first, in the base
            // order (they cost no copy, and the base order -- out-degree order
            // from the hubs -- is how improvements propagate); the chunks to
            // be streamed after them in order of predicted gain (which
            // partition to stream next).  PageRank keeps the base order
            // (forward Gauss-Seidel blocks).
            if (!is_pr)
                std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
                    const bool rx = slot_of[x] >= 0, ry = slot_of[y] >= 0;
                    if (rx != ry) return rx;
                    return !rx && pr[x] > pr[y];
                });
            // SSSP/BFS/CC: skip chunks predicted to change nothing, except after
            // a sweep without changes and at least every fourth sweep (the
            // stop rule needs every chunk processed after the last change)
            // (never without the prediction-off check: a skipped chunk breaks
            // the every-chunk-every-sweep premise of the strong conditions)
            const bool may_skip = !is_pr && P->verify && rep.changed > 0 && skip_streak < 3;
            if (may_skip) {
                std::vector<uint32_t> keep;
                for (uint32_t c : ord)
                    if (pr[c] >= 0.02f) keep.push_back(c);
                if (!keep.empty() && keep.size() < C) ord.swap(keep);
            }
            skip_streak = ord.size() < C ? skip_streak + 1 : 0;
            sched.append_order(ord);
        }
    }
    SR_CUDA(cudaEventRecord(ev_stop.e, cs.s));
    SR_CUDA(cudaStreamSynchronize(cs.s));
    S.time_ms = elapsed(ev_start.e, ev_stop.e);

    // ------------------------------------------------------------- output
    const void* src = is_pr ? (const void*)x.p : (const void*)val.p;
    if (out && g->reordered) {  // back to the caller's vertex ids
        uint32_t* dst = out_mem == SERAPH_MEM_DEVICE ? (uint32_t*)out : nullptr;
        if (!dst) {
            ensure(caller_order, n);
            dst = caller_order.p;
        }
        launch_unpermute((const uint32_t*)src, g->d_inv.p, n, dst, cs.s);
        ++launches;
        src = dst;
    }
    if (out && src != out) {
        SR_CUDA(cudaMemcpyAsync(out, src, 4 * n,
                                out_mem == SERAPH_MEM_HOST ? cudaMemcpyDeviceToHost
                                                           : cudaMemcpyDeviceToDevice,
                                cs.s));
    }
    SR_CUDA(cudaStreamSynchronize(cs.s));
    SR_CUDA(cudaStreamSynchronize(xs.s));
    if (stream_packed) SR_CUDA(cudaStreamSynchronize(ds.s));
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
