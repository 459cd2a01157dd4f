// Batched multi-query BFS/SSSP over many resident graphs in one persistent
// kernel (not in the paper: a serving pattern for many sources and many
// small graphs).
//
// Each query keeps its own distances and two frontier lists and advances in
// rounds; a round's frontier is cut into tiles of T vertices, and every tile
// is one task.  Tasks of all queries share one ring of task slots.  A block
// claims the next task index, waits until that slot is published, processes
// the tile (push relaxation over the out-edge CSR: atomicMin on the
// destination's distance, improved vertices go to the next frontier once per
// round), then counts the tile done; the block that finishes a query's last
// tile of a round publishes the query's next round.  No block ever waits for
// a block that has not started, so the kernel needs no co-residency; every
// wait has an iteration limit after which the kernel records an error and
// returns.  Label-correcting relaxation reaches the exact distances / levels
// whatever the interleaving.
//
// Mappings of a tile (picked per graph by the autotuner): one thread per
// frontier vertex, one warp per frontier vertex, or the whole CTA over the
// tile's edges (edge-balanced: a block scan of the tile's degrees, then one
// thread per edge).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "graph.hpp"


namespace seraph {
namespace {

constexpr int kNT = 256;
constexpr unsigned long long kConsumed = ~0ull;

struct BGraphDev {
    const uint64_t* off;
    const uint32_t* col;
    const uint8_t* w;
    uint32_t n, wbytes;
    const uint64_t* in_off;   // in-edge rows (bottom-up BFS)
    const uint32_t* in_col;
};

// SSSP queries order their work near-far: improved vertices whose distance is
// below `split` join the next round's (near) frontier, the others a far pile
// (once per epoch).  When the near frontier runs dry, a filter round raises
// split to (smallest far distance) + delta and moves the far vertices now
// below it to the near frontier, keeping the rest in the other far pile.
// BFS queries keep split = infinity (plain level-synchronous push).
//
// A record may also run a group of up to kMaxGroup queries of one graph and
// one algorithm in lockstep (gsz > 1): distances interleaved (dist[v * gsz +
// j] for sub-query j), one frontier of vertices for all of them, and per
// vertex a word (round << 8 | sub-query bits) telling which sub-queries hold
// it in the frontier of a round (mword, double-buffered by round parity) or
// in a far pile of an epoch (fword).  One read of a frontier vertex's
// out-edges then serves every sub-query that holds it, and the sub-queries'
// distances of a destination share one 32-byte sector.  The group shares
// one near-far split.
constexpr uint32_t kMaxGroup = 8;
constexpr uint32_t kMaxGroupTile = 512;

struct BQuery {
    uint32_t graph, algo, source, mapping, tile;
    uint32_t round, cur_n, next_n, tiles_total, tiles_done, done, pull_min;
    uint32_t split, delta, phase, fsel, epoch, far_min, far_n[2];
    uint32_t* dist;
    uint32_t* stamp;
    uint32_t* front[2];
    uint32_t* far[2];
    uint32_t* fstamp;
    uint32_t gsz;              // sub-queries (1: a single query, the fields above)
    uint32_t* mword[2];        // group: near-frontier words by round parity
    uint32_t* fword[2];        // group (SSSP): far-pile words by pile
};

// A group's sources and per-sub-query outputs (n distances each), read only
// at the start and the end of a launch.
struct BGroupIO {
    uint32_t src[kMaxGroup];
    uint32_t* gout[kMaxGroup];
    uint32_t tiles0;           // tiles of round 0 (every record)
};

constexpr uint32_t kPhaseNear = 0, kPhaseFilter = 1, kPhasePull = 2;
constexpr uint32_t kPullTile = 1024;  // vertices per bottom-up task
constexpr uint32_t kDefaultPullDiv = 5;  // pull when the frontier exceeds n / 5 (measured best of 1..100)
constexpr uint32_t kDefaultDelta = 64;  // near-far bucket width when the caller gives none

struct BGlobal {
    unsigned long long head, tail, edges, tasks;
    unsigned active, err, max_round, pad;
};

struct TaskSlot {
    unsigned long long seq;  // task index + 1 once published, kConsumed once read, 0 initially
    uint32_t q, tile, part, pad;
};

// A CTA-mapped tile whose frontier vertices have more than kPartEdges out-edges
// in all is processed in parts of kPartEdges edges: the task of part 0 spawns
// the others into the ring (raising the round's task count before its own
// completion is counted), so one hub no longer holds a round to one CTA.
constexpr uint64_t kPartEdges = 16384;

// What a task needs to spawn further tasks.
struct RingCtx {
    TaskSlot* ring;
    unsigned long long mask, spin_limit;
    BGlobal* gl;
};

__device__ __forceinline__ uint32_t weight_at(const BGraphDev& g, uint64_t e) {
    if (!g.w) return 1u;
    if (g.wbytes == 1) return g.w[e];
    if (g.wbytes == 2) return ((const uint16_t*)g.w)[e];
    return ((const uint32_t*)g.w)[e];
}

constexpr int kPushNone = 0, kPushNear = 1, kPushFar = 2;

// Relax edge (u -> v) with candidate distance cand.  `seen` is v's distance
// as last read: a candidate that does not beat it takes no atomic (most
// edges, and every edge into a hub that is already settled -- atomics on one
// address would serialise in L2).  An improvement pushes v once per round to
// the near frontier (cand < split) or once per epoch to the far pile.
__device__ __forceinline__ int relax(const BQuery& Q, uint32_t v, uint32_t cand, uint32_t seen) {
    if (cand >= seen) return kPushNone;
    const uint32_t old = atomicMin(&Q.dist[v], cand);
    if (cand >= old) return kPushNone;
    if (cand < Q.split)
        return atomicMax(&Q.stamp[v], Q.round + 1) < Q.round + 1 ? kPushNear : kPushNone;
    return atomicMax(&Q.fstamp[v], Q.epoch + 1) < Q.epoch + 1 ? kPushFar : kPushNone;
}

// Warp-aggregated append of the `push` lanes' vertices to list[*count].
__device__ __forceinline__ void append(uint32_t* list, uint32_t* count, bool push, uint32_t v) {
    const unsigned m = __ballot_sync(kFull, push);
    if (!m) return;
    const unsigned leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane_id() == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (push) list[base + __popc(m & lanemask_lt())] = v;
}

constexpr int kEdgeIlp = 4;  // edges per lane in flight per step
static_assert(kEdgeIlp == 4, "relax_edges tests four far-push slots");

// Warp-aggregated append of the kEdgeIlp slots of every lane whose push kind
// is `kind`: one atomic per warp for all of them.
__device__ __forceinline__ void append_many(uint32_t* list, uint32_t* count, const int push[kEdgeIlp],
                                            int kind, const uint32_t v[kEdgeIlp]) {
    unsigned m[kEdgeIlp], tot = 0;
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) {
        m[j] = __ballot_sync(kFull, push[j] == kind);
        tot += __popc(m[j]);
    }
    if (!tot) return;
    unsigned base = 0;
    if (lane_id() == 0) base = atomicAdd(count, tot);
    base = __shfl_sync(kFull, base, 0);
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) {
        if (push[j] == kind) list[base + __popc(m[j] & lanemask_lt())] = v[j];
        base += __popc(m[j]);
    }
}

__device__ __forceinline__ uint32_t cand_of(const BQuery& Q, uint32_t du, uint32_t w, bool& ok) {
    const uint32_t c = du + (Q.algo == SERAPH_SSSP ? w : 1u);
    ok = c >= du && c != SERAPH_INF;  // overflowing candidates are dropped
    return c;
}

// Query record as last published (read through L2: L1 is not coherent
// across SMs and this kernel outlives many rounds).
__device__ __forceinline__ BQuery load_query(const BQuery* p) {
    BQuery Q;
    const volatile BQuery* v = p;
    Q.graph = v->graph; Q.algo = v->algo; Q.source = v->source; Q.mapping = v->mapping;
    Q.tile = v->tile; Q.round = v->round; Q.cur_n = v->cur_n; Q.next_n = 0;
    Q.tiles_total = 0; Q.tiles_done = 0; Q.done = 0; Q.pull_min = v->pull_min;
    Q.split = v->split; Q.delta = v->delta; Q.phase = v->phase; Q.fsel = v->fsel;
    Q.epoch = v->epoch; Q.far_min = 0; Q.far_n[0] = Q.far_n[1] = 0;
    Q.dist = v->dist; Q.stamp = v->stamp; Q.front[0] = v->front[0]; Q.front[1] = v->front[1];
    Q.far[0] = v->far[0]; Q.far[1] = v->far[1]; Q.fstamp = v->fstamp;
    Q.gsz = v->gsz;
    Q.mword[0] = v->mword[0]; Q.mword[1] = v->mword[1];
    Q.fword[0] = v->fword[0]; Q.fword[1] = v->fword[1];
    return Q;
}

// Sets `bits` in a (tag << 8 | bits) word for `tag`: a word of an older tag
// starts over.  Returns true if this call opened the tag (the vertex enters
// the list of that round or epoch).  Each retry follows another thread's
// change of the word, and a word changes at most kMaxGroup + 1 times per tag.
__device__ __forceinline__ bool tag_or(uint32_t* w, uint32_t tag, uint32_t bits) {
    uint32_t old = *(volatile uint32_t*)w;
    for (;;) {
        const bool same = (old >> 8) == tag;
        const uint32_t want = same ? (old | bits) : ((tag << 8) | bits);
        if (want == old) return false;
        const uint32_t prev = atomicCAS(w, old, want);
        if (prev == old) return !same;
        old = prev;
    }
}

__device__ __forceinline__ uint32_t tag_bits(uint32_t w, uint32_t tag) {
    return (w >> 8) == tag ? (w & 0xFFu) : 0u;
}


// kEdgeIlp edges per lane: columns and weights first, then the distance
// reads, then the atomics of the candidates that improve, then the pushes.
// Edge j of this lane is (u_j -> col[e_j]) with source distance du_j; lanes
// with act_j false carry nothing (but still take part in the ballots).
// Block-aggregated append (all threads of the block call): one atomic per
// block for the near and far pushes of all its warps.
// Slot j of a lane goes to the near frontier when pn[j] == kPushNear and to
// the far pile when pf[j] == kPushFar (a group's edge may do both).
__device__ __forceinline__ void append_block(BQuery* qs, uint32_t q, const BQuery& Q,
                                             const int pn[kEdgeIlp], const int pf[kEdgeIlp],
                                             const uint32_t v[kEdgeIlp]) {
    __shared__ unsigned s_cnt[2][kNT / 32], s_base[2];
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    unsigned mn[kEdgeIlp], mf[kEdgeIlp], tn = 0, tf = 0;
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) {
        mn[j] = __ballot_sync(kFull, pn[j] == kPushNear);
        mf[j] = __ballot_sync(kFull, pf[j] == kPushFar);
        tn += __popc(mn[j]);
        tf += __popc(mf[j]);
    }
    if (lane == 0) { s_cnt[0][warp] = tn; s_cnt[1][warp] = tf; }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned tot = 0;
        for (int w = 0; w < kNT / 32; ++w) tot += s_cnt[threadIdx.x][w];
        s_base[threadIdx.x] = tot ? atomicAdd(threadIdx.x == 0 ? &qs[q].next_n : &qs[q].far_n[Q.fsel], tot) : 0u;
    }
    __syncthreads();
    unsigned bn = s_base[0], bf = s_base[1];
    for (unsigned w = 0; w < warp; ++w) { bn += s_cnt[0][w]; bf += s_cnt[1][w]; }
    uint32_t* near = Q.front[(Q.round + 1) & 1];
    uint32_t* far = Q.far[Q.fsel];
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) {
        if (pn[j] == kPushNear) near[bn + __popc(mn[j] & lanemask_lt())] = v[j];
        if (pf[j] == kPushFar) far[bf + __popc(mf[j] & lanemask_lt())] = v[j];
        bn += __popc(mn[j]);
        bf += __popc(mf[j]);
    }
    __syncthreads();  // s_cnt is reused by the next call
}

template <bool BLOCK>
__device__ __forceinline__ void relax_edges(BQuery* qs, uint32_t q, const BQuery& Q,
                                            const BGraphDev& G, const bool act[kEdgeIlp],
                                            const uint64_t e[kEdgeIlp],
                                            const uint32_t du[kEdgeIlp]) {
    uint32_t v[kEdgeIlp], c[kEdgeIlp], seen[kEdgeIlp];
    bool ok[kEdgeIlp];
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) {
        v[j] = act[j] ? G.col[e[j]] : 0u;
        c[j] = act[j] ? cand_of(Q, du[j], weight_at(G, e[j]), ok[j]) : 0u;
        ok[j] = act[j] && ok[j];
    }
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) seen[j] = ok[j] ? __ldcg(Q.dist + v[j]) : 0u;
    int push[kEdgeIlp];
#pragma unroll
    for (int j = 0; j < kEdgeIlp; ++j) push[j] = ok[j] ? relax(Q, v[j], c[j], seen[j]) : kPushNone;
    if (BLOCK) {
        append_block(qs, q, Q, push, push, v);
        return;
    }
    append_many(Q.front[(Q.round + 1) & 1], &qs[q].next_n, push, kPushNear, v);
    if (__any_sync(kFull, push[0] == kPushFar || push[1] == kPushFar || push[2] == kPushFar ||
                              push[3] == kPushFar))
        append_many(Q.far[Q.fsel], &qs[q].far_n[Q.fsel], push, kPushFar, v);
}

// A filter task: far-pile entries [t0, t0 + cnt) of query q.  Vertices whose
// distance is now below split join the near frontier (once per round), the
// others the other far pile (once per epoch).
__device__ void filter_tile(BQuery* qs, uint32_t q, const BQuery& Q, uint32_t t0, uint32_t cnt) {
    const uint32_t* src = Q.far[Q.fsel];
    const uint32_t dst = Q.fsel ^ 1u;
    for (uint32_t base = 0; base < cnt; base += kNT) {
        const uint32_t i = base + threadIdx.x;
        uint32_t v = 0, d = SERAPH_INF;
        if (i < cnt) {
            v = __ldcg(src + t0 + i);
            d = __ldcg(Q.dist + v);
        }
        const bool near = i < cnt && d < Q.split &&
                          atomicMax(&Q.stamp[v], Q.round + 1) < Q.round + 1;
        const bool far = i < cnt && d >= Q.split &&
                         atomicMax(&Q.fstamp[v], Q.epoch + 1) < Q.epoch + 1;
        append(Q.front[(Q.round + 1) & 1], &qs[q].next_n, near, v);
        append(Q.far[dst], &qs[q].far_n[dst], far, v);
        const uint32_t mn = __reduce_min_sync(kFull, far ? d : SERAPH_INF);
        if (lane_id() == 0 && mn != SERAPH_INF) atomicMin(&qs[q].far_min, mn);
    }
}

// Publish tasks [t0, t0 + count) of query q; the whole block helps.  Task i
// is tile i, part 0 (a round), or tile `tile`, part i + 1 (spawned parts).
__device__ bool publish(TaskSlot* ring, unsigned long long mask, unsigned long long t0,
                        uint32_t count, uint32_t q, unsigned long long spin_limit,
                        bool parts = false, uint32_t tile = 0) {
    bool ok = true;
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
        TaskSlot* sl = &ring[(t0 + i) & mask];
        unsigned long long spins = 0;
        for (;;) {  // the slot's previous task must have been read
            const unsigned long long s = *(volatile unsigned long long*)&sl->seq;
            if (s == 0 || s == kConsumed) break;
            if (++spins > spin_limit) { ok = false; break; }
            __nanosleep(32);
        }
        if (!ok) break;
        sl->q = q;
        sl->tile = parts ? tile : i;
        sl->part = parts ? i + 1 : 0;
        __threadfence();
        *(volatile unsigned long long*)&sl->seq = t0 + i + 1;
    }
    return ok;
}

// A bottom-up BFS task: vertices [t0, t0 + cnt) of the graph.  Each unvisited
// vertex scans its in-neighbours for one in the current frontier (level =
// round) and stops at the first; only this thread writes its level, so no
// atomics.  Found vertices form the next frontier.  Returns in-edges read.
__device__ unsigned long long pull_tile(BQuery* qs, uint32_t q, const BQuery& Q,
                                        const BGraphDev& G, uint32_t t0, uint32_t cnt) {
    unsigned long long edges = 0;
    for (uint32_t base = 0; base < cnt; base += kNT) {
        const uint32_t v = t0 + base + threadIdx.x;
        bool found = false;
        if (base + threadIdx.x < cnt && __ldcg(Q.dist + v) == SERAPH_INF) {
            const uint64_t b = G.in_off[v], e = G.in_off[v + 1];
            for (uint64_t k = b; k < e; ++k) {
                ++edges;
                if (__ldcg(Q.dist + G.in_col[k]) == Q.round) { found = true; break; }
            }
            if (found) Q.dist[v] = Q.round + 1;
        }
        append(Q.front[(Q.round + 1) & 1], &qs[q].next_n, found, v);
    }
    return edges;
}

// ------------------------------------------------------------ query groups

// Out-edge (u -> v) of weight w for the sub-queries in `bits` (u's distances
// du[j]): `near` / `far` receive the sub-queries it improved below / at or
// above the group's split.
__device__ __forceinline__ void group_relax(const BQuery& Q, uint32_t v, uint32_t w, uint32_t bits,
                                            const uint32_t* du, uint32_t& near, uint32_t& far) {
    near = far = 0;
    uint32_t* row = Q.dist + (uint64_t)v * Q.gsz;
    for (uint32_t m = bits; m; m &= m - 1) {
        const uint32_t j = __ffs(m) - 1;
        const uint32_t d = du[j];
        if (d == SERAPH_INF) continue;
        const uint32_t c = d + (Q.algo == SERAPH_SSSP ? w : 1u);
        if (c < d || c == SERAPH_INF) continue;  // overflowing candidates are dropped
        if (c >= __ldcg(row + j)) continue;
        if (c >= atomicMin(row + j, c)) continue;
        if (c < Q.split) near |= 1u << j;
        else far |= 1u << j;
    }
}

// A group's frontier tile, edge-balanced over the CTA like the CTA mapping of
// single queries (parts of kPartEdges edges included): each frontier vertex
// brings its sub-query bits and distances, each edge is read once for all
// of them.
__device__ unsigned long long group_near_tile(const BGraphDev& G, BQuery* qs, uint32_t q,
                                              const BQuery& Q, uint32_t tile, uint32_t part,
                                              const RingCtx& rc, uint64_t* s_pref, uint64_t* s_e0,
                                              uint32_t* s_gdu, uint32_t* s_gm) {
    __shared__ uint64_t ws[kNT / 32 + 1];
    const uint32_t GS = Q.gsz;
    const uint32_t* cur = Q.front[Q.round & 1];
    const uint32_t* mw = Q.mword[Q.round & 1];
    uint32_t* mw_next = Q.mword[(Q.round + 1) & 1];
    uint32_t* fw = Q.fword[Q.fsel];
    const uint32_t t0 = tile * Q.tile;
    const uint32_t cnt = min(Q.tile, Q.cur_n - t0);
    for (uint32_t base = 0; base < cnt; base += kNT) {
        const uint32_t i = base + threadIdx.x;
        uint64_t d = 0;
        if (i < cnt) {
            const uint32_t u = __ldcg(cur + t0 + i);
            const uint64_t b = G.off[u];
            s_e0[i] = b;
            s_gm[i] = tag_bits(__ldcg(mw + u), Q.round);
            for (uint32_t j = 0; j < GS; ++j) s_gdu[i * kMaxGroup + j] = __ldcg(Q.dist + (uint64_t)u * GS + j);
            d = G.off[u + 1] - b;
        }
        uint64_t tot;
        const uint64_t ex = block_excl_scan<kNT>(d, ws, &tot);
        const uint64_t run = base ? s_pref[base] : 0;
        if (i < cnt) s_pref[i] = run + ex;
        if (threadIdx.x == 0) s_pref[min(base + kNT, cnt)] = run + tot;
        __syncthreads();
    }
    const uint64_t total = s_pref[cnt];
    const uint64_t lo = (uint64_t)part * kPartEdges;
    const uint64_t hi = total < lo + kPartEdges ? total : lo + kPartEdges;
    if (part == 0 && total > kPartEdges) {  // spawn parts 1.. of this tile
        __shared__ unsigned long long s_t0;
        __shared__ uint32_t s_n;
        if (threadIdx.x == 0) {
            s_n = (uint32_t)((total - 1) / kPartEdges);
            atomicAdd(&qs[q].tiles_total, s_n);  // before this task counts as done
            s_t0 = atomicAdd(&rc.gl->tail, (unsigned long long)s_n);
            atomicAdd(&rc.gl->tasks, (unsigned long long)s_n);
        }
        __syncthreads();
        if (!publish(rc.ring, rc.mask, s_t0, s_n, q, rc.spin_limit, true, tile))
            atomicOr(&rc.gl->err, 4u);
        __syncthreads();
    }
    for (uint64_t k0 = lo; k0 < hi; k0 += (uint64_t)kNT * kEdgeIlp) {
        int pn[kEdgeIlp], pf[kEdgeIlp];
        uint32_t vv[kEdgeIlp];
#pragma unroll
        for (int j = 0; j < kEdgeIlp; ++j) {
            const uint64_t k = k0 + (uint64_t)j * kNT + threadIdx.x;
            pn[j] = pf[j] = kPushNone;
            vv[j] = 0;
            if (k < hi) {
                uint32_t a = 0, z = cnt - 1;  // largest i with s_pref[i] <= k
                while (a < z) {
                    const uint32_t mid = (a + z + 1) >> 1;
                    if (s_pref[mid] <= k) a = mid; else z = mid - 1;
                }
                const uint64_t e = s_e0[a] + (k - s_pref[a]);
                const uint32_t v = G.col[e];
                uint32_t near, far;
                group_relax(Q, v, weight_at(G, e), s_gm[a], s_gdu + a * kMaxGroup, near, far);
                vv[j] = v;
                if (near && tag_or(mw_next + v, Q.round + 1, near)) pn[j] = kPushNear;
                if (far && tag_or(fw + v, Q.epoch + 1, far)) pf[j] = kPushFar;
            }
        }
        append_block(qs, q, Q, pn, pf, vv);
    }
    __syncthreads();
    return threadIdx.x == 0 ? hi - lo : 0;
}

// A group's filter task over far-pile entries [t0, t0 + cnt): each entry's
// sub-queries now below the split join the near frontier, the others the
// other far pile.
__device__ void group_filter_tile(BQuery* qs, uint32_t q, const BQuery& Q, uint32_t t0, uint32_t cnt) {
    const uint32_t* src = Q.far[Q.fsel];
    const uint32_t dst = Q.fsel ^ 1u, GS = Q.gsz;
    for (uint32_t base = 0; base < cnt; base += kNT) {
        const uint32_t i = base + threadIdx.x;
        uint32_t v = 0, fmin = SERAPH_INF;
        bool pn = false, pf = false;
        if (i < cnt) {
            v = __ldcg(src + t0 + i);
            const uint32_t bits = tag_bits(__ldcg(Q.fword[Q.fsel] + v), Q.epoch);
            uint32_t near = 0, far = 0;
            for (uint32_t m = bits; m; m &= m - 1) {
                const uint32_t j = __ffs(m) - 1;
                const uint32_t d = __ldcg(Q.dist + (uint64_t)v * GS + j);
                if (d < Q.split) {
                    near |= 1u << j;
                } else {
                    far |= 1u << j;
                    fmin = min(fmin, d);
                }
            }
            pn = near && tag_or(Q.mword[(Q.round + 1) & 1] + v, Q.round + 1, near);
            pf = far && tag_or(Q.fword[dst] + v, Q.epoch + 1, far);
        }
        append(Q.front[(Q.round + 1) & 1], &qs[q].next_n, pn, v);
        append(Q.far[dst], &qs[q].far_n[dst], pf, v);
        const uint32_t mn = __reduce_min_sync(kFull, fmin);
        if (lane_id() == 0 && mn != SERAPH_INF) atomicMin(&qs[q].far_min, mn);
    }
}

// A group's bottom-up BFS task over vertices [t0, t0 + cnt): a vertex still
// unvisited by some sub-queries scans its in-neighbours for ones at level
// `round` in those sub-queries, and stops once it found all of them.
__device__ unsigned long long group_pull_tile(BQuery* qs, uint32_t q, const BQuery& Q,
                                              const BGraphDev& G, uint32_t t0, uint32_t cnt) {
    const uint32_t GS = Q.gsz, r = Q.round;
    uint32_t* mw_next = Q.mword[(r + 1) & 1];
    unsigned long long edges = 0;
    for (uint32_t base = 0; base < cnt; base += kNT) {
        const uint32_t v = t0 + base + threadIdx.x;
        uint32_t found = 0;
        if (base + threadIdx.x < cnt) {
            uint32_t need = 0;
            for (uint32_t j = 0; j < GS; ++j)
                if (__ldcg(Q.dist + (uint64_t)v * GS + j) == SERAPH_INF) need |= 1u << j;
            if (need) {
                const uint64_t b = G.in_off[v], e = G.in_off[v + 1];
                for (uint64_t k = b; k < e && need; ++k) {
                    ++edges;
                    const uint32_t u = G.in_col[k];
                    for (uint32_t m = need; m; m &= m - 1) {
                        const uint32_t j = __ffs(m) - 1;
                        if (__ldcg(Q.dist + (uint64_t)u * GS + j) == r) found |= 1u << j;
                    }
                    need &= ~found;
                }
                for (uint32_t m = found; m; m &= m - 1)
                    Q.dist[(uint64_t)v * GS + (__ffs(m) - 1)] = r + 1;
                if (found) mw_next[v] = ((r + 1) << 8) | found;
            }
        }
        append(Q.front[(r + 1) & 1], &qs[q].next_n, found != 0, v);
    }
    return edges;
}

// One task: tile `tile` of query q's current frontier.  Returns edges relaxed.
// Frontier entries and distances are mutable across rounds: read via L2.
__device__ unsigned long long process_tile(const BGraphDev* graphs, BQuery* qs, uint32_t q,
                                           uint32_t tile, uint32_t part, const RingCtx& rc,
                                           uint64_t* s_pref, uint64_t* s_e0, uint32_t* s_du,
                                           uint32_t* s_gdu, uint32_t* s_gm) {
    const BQuery Q = load_query(qs + q);
    const BGraphDev G = graphs[Q.graph];
    const uint32_t* cur = Q.front[Q.round & 1];
    const uint32_t t0 = tile * Q.tile;
    const uint32_t cnt = min(Q.tile, Q.cur_n - t0);
    unsigned long long edges = 0;
    if (Q.gsz > 1) {
        if (Q.phase == kPhaseFilter) {
            group_filter_tile(qs, q, Q, t0, cnt);
            return 0;
        }
        if (Q.phase == kPhasePull) {
            const uint32_t p0 = tile * kPullTile;
            return group_pull_tile(qs, q, Q, G, p0, min(kPullTile, G.n - p0));
        }
        return group_near_tile(G, qs, q, Q, tile, part, rc, s_pref, s_e0, s_gdu, s_gm);
    }
    if (Q.phase == kPhaseFilter) {
        filter_tile(qs, q, Q, t0, cnt);
        return 0;
    }
    if (Q.phase == kPhasePull) {
        const uint32_t p0 = tile * kPullTile;
        return pull_tile(qs, q, Q, G, p0, min(kPullTile, G.n - p0));
    }
    if (Q.mapping == SERAPH_MAP_THREAD) {
        for (uint32_t base = 0; base < cnt; base += kNT) {  // warps stay converged for the ballot
            const uint32_t i = base + threadIdx.x;
            uint32_t du = 0;
            uint64_t b = 0, e = 0;
            if (i < cnt) {
                const uint32_t u = __ldcg(cur + t0 + i);
                du = __ldcg(Q.dist + u);
                b = G.off[u];
                e = G.off[u + 1];
            }
            edges += e - b;
            for (uint64_t k = b;; k += kEdgeIlp) {
                if (!__any_sync(kFull, k < e)) break;
                bool act[kEdgeIlp];
                uint64_t ek[kEdgeIlp];
                uint32_t dk[kEdgeIlp];
#pragma unroll
                for (int j = 0; j < kEdgeIlp; ++j) { act[j] = k + j < e; ek[j] = k + j; dk[j] = du; }
                relax_edges<false>(qs, q, Q, G, act, ek, dk);
            }
        }
    } else if (Q.mapping == SERAPH_MAP_WARP) {
        const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
        for (uint32_t i = warp; i < cnt; i += kNT / 32) {
            const uint32_t u = __ldcg(cur + t0 + i);
            const uint32_t du = __ldcg(Q.dist + u);
            const uint64_t b = G.off[u], e = G.off[u + 1];
            if (lane == 0) edges += e - b;
            for (uint64_t k0 = b; k0 < e; k0 += 32 * kEdgeIlp) {
                bool act[kEdgeIlp];
                uint64_t ek[kEdgeIlp];
                uint32_t dk[kEdgeIlp];
#pragma unroll
                for (int j = 0; j < kEdgeIlp; ++j) {
                    ek[j] = k0 + j * 32 + lane;
                    act[j] = ek[j] < e;
                    dk[j] = du;
                }
                relax_edges<false>(qs, q, Q, G, act, ek, dk);
            }
        }
    } else {  // edge-balanced over the tile (tile <= kMaxCtaTile)
        __shared__ uint64_t ws[kNT / 32 + 1];
        for (uint32_t base = 0; base < cnt; base += kNT) {
            const uint32_t i = base + threadIdx.x;
            uint64_t d = 0;
            if (i < cnt) {
                const uint32_t u = __ldcg(cur + t0 + i);
                const uint64_t b = G.off[u];
                s_e0[i] = b;
                s_du[i] = __ldcg(Q.dist + u);
                d = G.off[u + 1] - b;
            }
            uint64_t tot;
            const uint64_t ex = block_excl_scan<kNT>(d, ws, &tot);
            const uint64_t run = base ? s_pref[base] : 0;
            if (i < cnt) s_pref[i] = run + ex;
            if (threadIdx.x == 0) s_pref[min(base + kNT, cnt)] = run + tot;
            __syncthreads();
        }
        const uint64_t total = s_pref[cnt];
        const uint64_t lo = (uint64_t)part * kPartEdges;
        const uint64_t hi = total < lo + kPartEdges ? total : lo + kPartEdges;
        if (part == 0 && total > kPartEdges) {  // spawn parts 1.. of this tile
            __shared__ unsigned long long s_t0;
            __shared__ uint32_t s_n;
            if (threadIdx.x == 0) {
                s_n = (uint32_t)((total - 1) / kPartEdges);
                atomicAdd(&qs[q].tiles_total, s_n);  // before this task counts as done
                s_t0 = atomicAdd(&rc.gl->tail, (unsigned long long)s_n);
                atomicAdd(&rc.gl->tasks, (unsigned long long)s_n);
            }
            __syncthreads();
            if (!publish(rc.ring, rc.mask, s_t0, s_n, q, rc.spin_limit, true, tile))
                atomicOr(&rc.gl->err, 4u);
            __syncthreads();
        }
        edges = threadIdx.x == 0 ? hi - lo : 0;
        for (uint64_t k0 = lo; k0 < hi; k0 += (uint64_t)kNT * kEdgeIlp) {
            bool act[kEdgeIlp];
            uint64_t ek[kEdgeIlp];
            uint32_t dk[kEdgeIlp];
#pragma unroll
            for (int j = 0; j < kEdgeIlp; ++j) {
                const uint64_t k = k0 + (uint64_t)j * kNT + threadIdx.x;
                act[j] = k < hi;
                ek[j] = 0;
                dk[j] = 0;
                if (act[j]) {
                    uint32_t lo = 0, hi = cnt - 1;  // largest i with s_pref[i] <= k
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_pref[mid] <= k) lo = mid; else hi = mid - 1;
                    }
                    ek[j] = s_e0[lo] + (k - s_pref[lo]);
                    dk[j] = s_du[lo];
                }
            }
            relax_edges<true>(qs, q, Q, G, act, ek, dk);
        }
        __syncthreads();
    }
    return edges;
}

constexpr uint32_t kMaxCtaTile = 1024;

// Publish tasks [t0, t0 + count) = (q, tile 0..count-1); the whole block helps.
// Four resident CTAs per SM (<= 64 registers): the grid is 4 x SMs and the
// kernel keeps no CTA waiting for a slot.
__global__ void __launch_bounds__(kNT, 4) batch_kernel(const BGraphDev* graphs, BQuery* qs,
                                                    BGlobal* gl, TaskSlot* ring,
                                                    unsigned long long mask,
                                                    unsigned long long spin_limit) {
    __shared__ uint64_t s_pref[kMaxCtaTile + 1];
    __shared__ uint64_t s_e0[kMaxCtaTile];
    __shared__ uint32_t s_du[kMaxCtaTile];
    __shared__ uint32_t s_gdu[kMaxGroupTile * kMaxGroup];
    __shared__ uint32_t s_gm[kMaxGroupTile];
    __shared__ uint32_t s_q, s_tile, s_part, s_last, s_count;
    const RingCtx rc{ring, mask, spin_limit, gl};
    __shared__ int s_exit;
    __shared__ unsigned long long s_t0;
    __shared__ unsigned long long s_edges;
    if (threadIdx.x == 0) s_edges = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(&gl->head, 1ull);
            TaskSlot* sl = &ring[t & mask];
            unsigned long long spins = 0;
            s_exit = 0;
            for (;;) {
                const unsigned long long s = *(volatile unsigned long long*)&sl->seq;
                if (s == t + 1) {
                    __threadfence();
                    s_q = sl->q;
                    s_tile = sl->tile;
                    s_part = sl->part;
                    *(volatile unsigned long long*)&sl->seq = kConsumed;
                    break;
                }
                if (*(volatile unsigned*)&gl->active == 0) { s_exit = 1; break; }
                if (*(volatile unsigned*)&gl->err) { s_exit = 1; break; }
                if (++spins > spin_limit) { atomicOr(&gl->err, 1u); s_exit = 1; break; }
                __nanosleep(64);
            }
        }
        __syncthreads();
        if (s_exit) break;
        const uint32_t q = s_q;
        const unsigned long long e = process_tile(graphs, qs, q, s_tile, s_part, rc, s_pref, s_e0, s_du,
                                                  s_gdu, s_gm);
        atomicAdd(&s_edges, e);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // this tile's frontier pushes before its completion count
            const uint32_t done = atomicAdd(&qs[q].tiles_done, 1u) + 1;
            s_last = done == *(volatile uint32_t*)&qs[q].tiles_total;
            if (s_last) {  // advance query q to its next round
                __threadfence();
                volatile BQuery* Q = &qs[q];
                bool exact_min = false;  // far_min is the current far pile's minimum
                if (Q->phase == kPhaseFilter) {  // the filter wrote the other far pile
                    Q->fsel = Q->fsel ^ 1u;
                    Q->phase = kPhaseNear;
                    exact_min = true;
                }
                if (Q->phase == kPhasePull) Q->phase = kPhaseNear;
                uint32_t nn = Q->next_n;
                if (nn == 0 && Q->far_n[Q->fsel] > 0) {  // near frontier dry: filter the far pile
                    const uint32_t fs = Q->fsel;
                    nn = Q->far_n[fs];
                    const uint32_t base = exact_min ? Q->far_min : Q->split;
                    const uint32_t lim = SERAPH_INF - 1u - Q->delta;
                    Q->split = base < lim ? base + Q->delta : SERAPH_INF - 1u;
                    Q->far_min = SERAPH_INF;
                    Q->far_n[fs ^ 1u] = 0;
                    Q->far_n[fs] = 0;  // read again through cur_n by the filter tasks
                    Q->epoch = Q->epoch + 1;
                    Q->phase = kPhaseFilter;
                }
                uint32_t tiles = (nn + Q->tile - 1) / Q->tile;
                if (Q->algo == SERAPH_BFS && Q->phase == kPhaseNear && nn > Q->pull_min) {
                    // a large frontier: the next round pulls over all vertices
                    const uint32_t n = graphs[Q->graph].n;
                    Q->phase = kPhasePull;
                    tiles = (n + kPullTile - 1) / kPullTile;
                }
                Q->round = Q->round + 1;
                atomicMax(&gl->max_round, Q->round);
                Q->cur_n = nn;
                Q->next_n = 0;
                Q->tiles_done = 0;
                Q->tiles_total = tiles;
                s_count = Q->tiles_total;
                if (nn == 0) {
                    Q->done = 1;
                    __threadfence();
                    atomicSub(&gl->active, 1u);
                } else {
                    __threadfence();
                    s_t0 = atomicAdd(&gl->tail, (unsigned long long)s_count);
                    atomicAdd(&gl->tasks, (unsigned long long)s_count);
                }
            }
        }
        __syncthreads();
        if (s_last && s_count && !publish(ring, mask, s_t0, s_count, q, spin_limit))
            atomicOr(&gl->err, 2u);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&gl->edges, s_edges);
}

__global__ void init_dist_kernel(BQuery* qs, const BGroupIO* io, const BGraphDev* graphs, uint32_t nq) {
    for (uint32_t q = blockIdx.y; q < nq; q += gridDim.y) {
        const BQuery Q = qs[q];
        const uint32_t n = graphs[Q.graph].n;
        if (Q.gsz > 1) {  // interleaved distances; the tag words start empty
            for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
                for (uint32_t j = 0; j < Q.gsz; ++j)
                    Q.dist[(uint64_t)v * Q.gsz + j] = v == io[q].src[j] ? 0u : SERAPH_INF;
                Q.mword[0][v] = 0;
                Q.mword[1][v] = 0;
                if (Q.fword[0]) { Q.fword[0][v] = 0; Q.fword[1][v] = 0; }
            }
            continue;
        }
        for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
            Q.dist[v] = v == Q.source ? 0u : SERAPH_INF;
            Q.stamp[v] = 0;
            if (Q.fstamp) Q.fstamp[v] = 0;
        }
    }
}

// Round 0 of every query (frontier = its source) and the first nq tasks.
// Round 0 of every record and its first tasks: init_task[i] = (record, tile)
// of task i < ntask0 (a group's distinct sources may take several tiles).
__global__ void init_queries_kernel(BQuery* qs, const BGroupIO* io, uint32_t nq, BGlobal* gl,
                                    TaskSlot* ring, unsigned long long cap, const uint2* init_task,
                                    uint32_t ntask0) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const bool first = i < ntask0;
        ring[i].seq = first ? i + 1 : 0;
        ring[i].q = first ? init_task[i].x : 0u;
        ring[i].tile = first ? init_task[i].y : 0u;
        ring[i].part = 0;
    }
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        BQuery& Q = qs[q];
        Q.round = 0;
        Q.cur_n = 1;
        Q.next_n = 0;
        Q.tiles_total = io[q].tiles0;
        Q.tiles_done = 0;
        Q.done = 0;
        Q.split = Q.algo == SERAPH_SSSP ? Q.delta : SERAPH_INF;
        Q.phase = kPhaseNear;
        Q.fsel = 0;
        Q.epoch = 0;
        Q.far_min = SERAPH_INF;
        Q.far_n[0] = Q.far_n[1] = 0;
        if (Q.gsz > 1) {  // round 0: the distinct sources, each with its sub-queries
            uint32_t c = 0;
            for (uint32_t j = 0; j < Q.gsz; ++j) {
                const uint32_t s = io[q].src[j], w = Q.mword[0][s];
                if (!(w & 0xFFu)) Q.front[0][c++] = s;
                Q.mword[0][s] = w | (1u << j);
            }
            Q.cur_n = c;
        } else {
            Q.front[0][0] = Q.source;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        gl->head = 0;
        gl->tail = ntask0;
        gl->edges = 0;
        gl->tasks = ntask0;
        gl->active = nq;
        gl->err = 0;
        gl->max_round = 0;
    }
}

// Group results out of the interleaved distances into one array per sub-query.
__global__ void group_scatter_kernel(const BQuery* qs, const BGroupIO* io, const BGraphDev* graphs,
                                     uint32_t nq) {
    for (uint32_t q = blockIdx.y; q < nq; q += gridDim.y) {
        const BQuery& Q = qs[q];
        if (Q.gsz <= 1) continue;
        const uint32_t n = graphs[Q.graph].n;
        for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
            for (uint32_t j = 0; j < Q.gsz; ++j) io[q].gout[j][v] = Q.dist[(uint64_t)v * Q.gsz + j];
    }
}

struct QSpec {
    uint32_t graph, algo, source, mapping, tile;
    uint32_t* out;  // device buffer for the distances, or null
    uint32_t delta; // near-far bucket width (SSSP)
    uint32_t pull_div;  // BFS: pull when the frontier exceeds n / pull_div
};

struct Outcome {
    float ms = 0.f;
    unsigned long long edges = 0, tasks = 0;
    unsigned max_round = 0;
    bool captured = false;
};

void wait_stream(cudaStream_t s, uint32_t timeout_ms) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t r = cudaStreamQuery(s);
        if (r == cudaSuccess) return;
        if (r != cudaErrorNotReady) SR_CUDA(r);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        SR_CHECK(ms < timeout_ms, SERAPH_ETIMEOUT, "timed out waiting for the batched kernel");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Everything one batched launch needs on the device, built once and run any
// number of times (a plan keeps it between calls): the record tables, the
// per-query arrays carved from one pool, the task ring, the captured launch.
struct Prepared {
    std::vector<BGraphDev> gd;
    std::vector<std::vector<uint32_t>> recs;  // the queries of each record
    std::vector<BQuery> qh;
    std::vector<BGroupIO> ioh;
    std::vector<DevBuf<uint32_t>> hold;       // the per-query array pool
    DevBuf<BGraphDev> d_g;
    DevBuf<BQuery> d_q;
    DevBuf<BGroupIO> d_io;
    DevBuf<uint2> d_t0;
    DevBuf<BGlobal> d_gl;
    DevBuf<TaskSlot> d_ring;
    PinnedBuf gl_h;                           // the counters read back after a run
    PinnedBuf tab_h;                          // record tables staged for upload
    unsigned long long cap = 0, spin_limit = 0;
    unsigned blocks = 0;
    uint32_t nr = 0, ntask0 = 0, max_n = 1, timeout_ms = 0;
    bool any_group = false, captured = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Prepared() = default;
    Prepared(const Prepared&) = delete;
    Prepared& operator=(const Prepared&) = delete;
    ~Prepared() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    void enqueue(cudaStream_t st) const {
        const dim3 ig((max_n + 255) / 256 < 64 ? (max_n + 255) / 256 : 64, std::min<uint32_t>(nr, 65535));
        init_dist_kernel<<<ig, 256, 0, st>>>(d_q.p, d_io.p, d_g.p, nr);
        init_queries_kernel<<<(unsigned)std::min<unsigned long long>((cap + 255) / 256, 4096), 256, 0, st>>>(
            d_q.p, d_io.p, nr, d_gl.p, d_ring.p, cap, d_t0.p, ntask0);
        batch_kernel<<<blocks, kNT, 0, st>>>(d_g.p, d_q.p, d_gl.p, d_ring.p, cap - 1, spin_limit);
        if (any_group) group_scatter_kernel<<<ig, 256, 0, st>>>(d_q.p, d_io.p, d_g.p, nr);
    }
    // The record tables (as built, or with new sources) to the device on `st`.
    void upload(cudaStream_t st) {
        const size_t qb = nr * sizeof(BQuery), ib = nr * sizeof(BGroupIO);
        std::memcpy(tab_h.p, qh.data(), qb);
        std::memcpy(tab_h.p + qb, ioh.data(), ib);
        SR_CUDA(cudaMemcpyAsync(d_q.p, tab_h.p, qb, cudaMemcpyHostToDevice, st));
        SR_CUDA(cudaMemcpyAsync(d_io.p, tab_h.p + qb, ib, cudaMemcpyHostToDevice, st));
    }
};

// Builds `pb` for the queries `qs` (distances stay in q.out when given, else
// in the pool; `dist_out[q]` says where) and captures its launch in a CUDA
// graph if `use_graph`.
void prepare_batch(Prepared& pb, const std::vector<seraph_bgraph*>& graphs,
                   const std::vector<QSpec>& qs, bool use_graph, uint32_t timeout_ms, cudaStream_t s,
                   std::vector<uint32_t*>* dist_out, bool group) {
    const uint32_t nq = (uint32_t)qs.size();
    std::vector<BGraphDev>& gd = pb.gd;
    gd.assign(graphs.size(), BGraphDev{});
    for (size_t i = 0; i < graphs.size(); ++i) {
        const seraph_bgraph* g = graphs[i];
        gd[i] = BGraphDev{g->adj.off.p, g->adj.col.p, g->weighted ? g->adj.wptr() : nullptr,
                          (uint32_t)g->n, g->adj.wbytes, g->in_adj.off.p, g->in_adj.col.p};
    }
    // Records: with `group`, the queries of one graph, algorithm and tuning
    // (tile, near-far width, pull threshold) run in lockstep groups of up to
    // kMaxGroup; otherwise (and for a query left alone) one record each.
    std::vector<std::vector<uint32_t>>& recs = pb.recs;
    recs.clear();
    {
        std::vector<uint8_t> taken(nq, 0);
        for (uint32_t q = 0; q < nq; ++q) {
            if (taken[q]) continue;
            std::vector<uint32_t> r{q};
            taken[q] = 1;
            for (uint32_t p = q + 1; group && p < nq && r.size() < kMaxGroup; ++p) {
                const QSpec &a = qs[q], &b = qs[p];
                if (!taken[p] && a.graph == b.graph && a.algo == b.algo && a.tile == b.tile &&
                    a.delta == b.delta && a.pull_div == b.pull_div) {
                    r.push_back(p);
                    taken[p] = 1;
                }
            }
            recs.push_back(r);
        }
    }
    const uint32_t nr = (uint32_t)recs.size();
    pb.qh.assign(nr, BQuery{});
    pb.ioh.assign(nr, BGroupIO{});
    std::vector<BQuery>& qh = pb.qh;
    std::vector<BGroupIO>& ioh = pb.ioh;
    std::vector<uint2> init_tasks;  // (record, tile) of every round-0 task
    // every per-query array comes out of one allocation (one cudaMalloc per
    // call instead of several per query), each array 128-byte aligned
    auto words = [](uint64_t n) { return (n + 31) & ~31ull; };
    uint64_t pool_words = 0;
    for (const auto& r : recs) {
        const QSpec& Q = qs[r[0]];
        const uint64_t n = graphs[Q.graph]->n;
        const bool sssp = Q.algo == SERAPH_SSSP;
        if (r.size() == 1) {
            pool_words += words(n) * ((Q.out ? 0 : 1) + 3 + (sssp ? 3 : 0));
        } else {  // distances (n x size), fronts, tag words; outputs per query
            pool_words += words(n * r.size()) + words(n) * (4 + (sssp ? 4 : 0));
            for (uint32_t q : r) pool_words += qs[q].out ? 0 : words(n);
        }
    }
    pb.hold.clear();
    pb.hold.emplace_back(std::max<uint64_t>(pool_words, 1));
    uint32_t* pool = pb.hold.back().p;
    auto carve = [&](uint64_t n) { uint32_t* p = pool; pool += words(n); return p; };
    uint64_t tiles = 0;
    uint32_t max_n = 1;
    bool any_group = false;
    for (uint32_t ri = 0; ri < nr; ++ri) {
        const std::vector<uint32_t>& r = recs[ri];
        const QSpec& Q = qs[r[0]];
        const uint64_t n = graphs[Q.graph]->n;
        max_n = std::max<uint32_t>(max_n, (uint32_t)n);
        BQuery b{};
        b.graph = Q.graph; b.algo = Q.algo; b.source = Q.source; b.mapping = Q.mapping; b.tile = Q.tile;
        b.gsz = (uint32_t)r.size();
        b.delta = Q.delta ? Q.delta : 1u;
        b.pull_min = (uint32_t)(n / (Q.pull_div ? Q.pull_div : 1u));
        if (b.gsz == 1) {
            b.dist = Q.out ? Q.out : carve(n);
            b.stamp = carve(n);
            b.front[0] = carve(n);
            b.front[1] = carve(n);
            if (Q.algo == SERAPH_SSSP) {  // far piles and their per-epoch stamps
                b.far[0] = carve(n);
                b.far[1] = carve(n);
                b.fstamp = carve(n);
            }
            if (dist_out) (*dist_out)[r[0]] = b.dist;
        } else {
            any_group = true;
            b.tile = std::min<uint32_t>(Q.tile, kMaxGroupTile);
            b.dist = carve(n * b.gsz);
            b.front[0] = carve(n);
            b.front[1] = carve(n);
            b.mword[0] = carve(n);
            b.mword[1] = carve(n);
            if (Q.algo == SERAPH_SSSP) {
                b.far[0] = carve(n);
                b.far[1] = carve(n);
                b.fword[0] = carve(n);
                b.fword[1] = carve(n);
            }
            std::vector<uint32_t> distinct;
            for (uint32_t j = 0; j < b.gsz; ++j) {
                const QSpec& S = qs[r[j]];
                ioh[ri].src[j] = S.source;
                ioh[ri].gout[j] = S.out ? S.out : carve(n);
                if (dist_out) (*dist_out)[r[j]] = ioh[ri].gout[j];
                if (std::find(distinct.begin(), distinct.end(), S.source) == distinct.end())
                    distinct.push_back(S.source);
            }
            ioh[ri].tiles0 = ((uint32_t)distinct.size() + b.tile - 1) / b.tile;
        }
        if (b.gsz == 1) ioh[ri].tiles0 = 1;
        for (uint32_t t = 0; t < ioh[ri].tiles0; ++t) init_tasks.push_back(make_uint2(ri, t));
        qh[ri] = b;
        tiles += (n + b.tile - 1) / b.tile + graphs[Q.graph]->adj.E / kPartEdges + 1;
    }
    const int sms = device_sms();
    const unsigned blocks = (unsigned)sms * 4;
    unsigned long long cap = 1024;
    const uint32_t ntask0 = (uint32_t)init_tasks.size();
    while (cap < tiles + ntask0 + 4ull * blocks + 1024) cap <<= 1;
    pb.nr = nr;
    pb.ntask0 = ntask0;
    pb.cap = cap;
    pb.blocks = blocks;
    pb.max_n = max_n;
    pb.any_group = any_group;
    pb.timeout_ms = timeout_ms;
    // ~15 polls per microsecond with the back-off: a limit of timeout_ms
    pb.spin_limit = (unsigned long long)timeout_ms * 15000ull;
    pb.d_g.alloc(gd.size());
    pb.d_q.alloc(nr);
    pb.d_io.alloc(nr);
    pb.d_t0.alloc(ntask0);
    pb.d_gl.alloc(1);
    pb.d_ring.alloc(cap);
    pb.gl_h.alloc(sizeof(BGlobal));
    pb.tab_h.alloc(nr * (sizeof(BQuery) + sizeof(BGroupIO)));
    SR_CUDA(cudaMemcpyAsync(pb.d_g.p, gd.data(), gd.size() * sizeof(BGraphDev), cudaMemcpyHostToDevice, s));
    pb.upload(s);
    SR_CUDA(cudaMemcpyAsync(pb.d_t0.p, init_tasks.data(), ntask0 * sizeof(uint2), cudaMemcpyHostToDevice, s));
    SR_CUDA(cudaStreamSynchronize(s));  // (the staged tables are reused by later uploads)
    if (use_graph) {
        SR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        pb.enqueue(s);
        const cudaError_t ce = cudaStreamEndCapture(s, &pb.graph);
        if (ce == cudaSuccess && cudaGraphInstantiate(&pb.exec, pb.graph, 0) == cudaSuccess) {
            pb.captured = true;
        } else {
            (void)cudaGetLastError();
            if (pb.graph) cudaGraphDestroy(pb.graph);
            pb.graph = nullptr;
        }
    }
}

// `replays` timed runs of a prepared batch (through its captured graph when
// there is one); the distances of the last are left in the queries' arrays.
// Allocates nothing.
Outcome run_batch(Prepared& pb, uint32_t replays, cudaStream_t s) {
    Outcome out;
    out.captured = pb.captured;
    cudaEvent_t e0, e1;
    SR_CUDA(cudaEventCreate(&e0));
    SR_CUDA(cudaEventCreate(&e1));
    const uint32_t reps = std::max<uint32_t>(replays, 1);
    SR_CUDA(cudaEventRecord(e0, s));
    for (uint32_t r = 0; r < reps; ++r) {
        if (pb.captured) SR_CUDA(cudaGraphLaunch(pb.exec, s));
        else pb.enqueue(s);
        SR_LAUNCH();
    }
    SR_CUDA(cudaEventRecord(e1, s));
    SR_CUDA(cudaMemcpyAsync(pb.gl_h.p, pb.d_gl.p, sizeof(BGlobal), cudaMemcpyDeviceToHost, s));
    try {
        wait_stream(s, pb.timeout_ms * reps + 1000);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    float ms = 0.f;
    SR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BGlobal gl;
    std::memcpy(&gl, pb.gl_h.p, sizeof(gl));
    SR_CHECK(gl.err == 0, SERAPH_ETIMEOUT, "batched kernel: a bounded wait ran out (status " +
                                               std::to_string(gl.err) + ")");
    out.ms = ms / reps;
    out.edges = gl.edges;
    out.tasks = gl.tasks;
    out.max_round = gl.max_round;
    return out;
}

// One batched launch: prepare, then run `replays` times.
Outcome launch_batch(Prepared& pb, const std::vector<seraph_bgraph*>& graphs, const std::vector<QSpec>& qs,
                     bool use_graph, uint32_t replays, uint32_t timeout_ms, cudaStream_t s,
                     std::vector<uint32_t*>* dist_out, bool group = false) {
    prepare_batch(pb, graphs, qs, use_graph, timeout_ms, s, dist_out, group);
    return run_batch(pb, replays, s);
}

}  // namespace

void bgraph_build(seraph_bgraph* g, uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                  const uint32_t* w, int mem, cudaStream_t s) {
    SR_CHECK(n >= 1 && n <= 0xFFFFFFFEull, SERAPH_EINVAL, "n must be in [1, 2^32-2]");
    SR_CHECK(mem == SERAPH_MEM_HOST || mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad mem kind");
    SR_CHECK(m == 0 || (src && dst), SERAPH_EINVAL, "src/dst must not be NULL");
    SR_CUDA(cudaGetDevice(&g->device));
    g->n = n;
    g->m_raw = m;
    g->weighted = w != nullptr;
    // rows = sources: the sorted adjacency of the swapped edge list
    sorted_adjacency(n, m, dst, src, w, mem, false, s, g->adj);
    // rows = destinations, for BFS rounds that pull from the frontier
    sorted_adjacency(n, m, src, dst, nullptr, mem, false, s, g->in_adj);
}

namespace {

// The launch specs of a batch call: each graph's mapping, tile and near-far
// width -- fixed, cached in the graph, or autotuned on the graph's own
// queries -- then one spec per query (checked).  S.tune_ms gets the tuning
// time; gmap / gtile the choices.
std::vector<QSpec> batch_specs(const std::vector<seraph_bgraph*>& graphs, const seraph_query* qin,
                               uint32_t nq, int out_mem, const seraph_batch_params* P, cudaStream_t s,
                               seraph_batch_stats& S, std::vector<uint32_t>& gmap,
                               std::vector<uint32_t>& gtile) {
    const uint32_t ng = (uint32_t)graphs.size();
    // 0 = a width per graph (tuned below with the mapping), else the caller's
    const uint32_t delta = P->delta ? P->delta : kDefaultDelta;
    const bool tune_delta = P->delta == 0 && P->mapping == SERAPH_MAP_AUTO;
    const uint32_t pull_div = P->bfs_pull_div ? P->bfs_pull_div : kDefaultPullDiv;
    const bool group = P->group != 0;
    auto t_tune = std::chrono::steady_clock::now();
    // per-graph mapping and tile: fixed, cached, or autotuned on the graph's own queries
    gmap.assign(ng, 0);
    gtile.assign(ng, 0);
    std::vector<uint32_t> gdelta(ng, delta);
    for (uint32_t gi = 0; gi < ng; ++gi) {
        if (P->mapping != SERAPH_MAP_AUTO) {
            gmap[gi] = (uint32_t)P->mapping;
            gtile[gi] = P->tile ? P->tile : 256;
            continue;
        }
        if (graphs[gi]->tuned_mapping) {
            gmap[gi] = graphs[gi]->tuned_mapping;
            gtile[gi] = graphs[gi]->tuned_tile;
            if (tune_delta && graphs[gi]->tuned_delta) gdelta[gi] = graphs[gi]->tuned_delta;
            continue;
        }
        std::vector<QSpec> sub;
        std::vector<seraph_bgraph*> one{graphs[gi]};
        for (uint32_t q = 0; q < nq; ++q)
            if (qin[q].graph == gi)
                sub.push_back(QSpec{0, (uint32_t)qin[q].algo, qin[q].source, 0, 0, nullptr, delta, pull_div});
        float best = 1e30f;
        uint32_t bm = SERAPH_MAP_CTA, bt = 256;
        if (!sub.empty()) {
            // grouped queries take the edge-balanced CTA tiles (of at most 512)
            const std::vector<uint32_t> maps = group ? std::vector<uint32_t>{SERAPH_MAP_CTA}
                                                     : std::vector<uint32_t>{SERAPH_MAP_THREAD,
                                                                             SERAPH_MAP_WARP,
                                                                             SERAPH_MAP_CTA};
            const std::vector<uint32_t> tls = group ? std::vector<uint32_t>{64u, 256u, 512u}
                                                    : std::vector<uint32_t>{64u, 256u, 1024u};
            for (uint32_t mp : maps)
                for (uint32_t tl : tls) {
                    for (auto& x : sub) { x.mapping = mp; x.tile = tl; }
                    Prepared pb;
                    const Outcome o = launch_batch(pb, one, sub, false, 2, P->timeout_ms, s, nullptr,
                                                   group);
                    if (o.ms < best) { best = o.ms; bm = mp; bt = tl; }
                }
        }
        // the near-far width for this graph's SSSP queries, with the chosen mapping
        uint32_t bd = delta;
        std::vector<QSpec> ss;
        for (const QSpec& x : sub)
            if (x.algo == SERAPH_SSSP && graphs[gi]->weighted) ss.push_back(x);
        if (tune_delta && !ss.empty()) {
            float bestd = 1e30f;
            for (uint32_t d : {64u, 128u, 256u, 512u}) {
                for (auto& x : ss) { x.mapping = bm; x.tile = bt; x.delta = d; }
                Prepared pb;
                const Outcome o = launch_batch(pb, one, ss, false, 2, P->timeout_ms, s, nullptr, group);
                if (o.ms < bestd) { bestd = o.ms; bd = d; }
            }
        }
        graphs[gi]->tuned_mapping = (int)bm;
        graphs[gi]->tuned_tile = bt;
        graphs[gi]->tuned_delta = tune_delta && !ss.empty() ? bd : 0;
        gmap[gi] = bm;
        gtile[gi] = bt;
        gdelta[gi] = bd;
    }
    S.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_tune).count();

    std::vector<QSpec> qs(nq);
    for (uint32_t q = 0; q < nq; ++q) {
        const seraph_query& Q = qin[q];
        SR_CHECK(Q.graph < ng, SERAPH_EINVAL, "query graph index out of range");
        SR_CHECK(Q.algo == SERAPH_SSSP || Q.algo == SERAPH_BFS, SERAPH_EINVAL, "batched queries are SSSP or BFS");
        SR_CHECK(Q.source < graphs[Q.graph]->n, SERAPH_EINVAL, "query source >= n");
        SR_CHECK(Q.out != nullptr, SERAPH_EINVAL, "query output must not be NULL");
        const uint32_t algo = (Q.algo == SERAPH_SSSP && !graphs[Q.graph]->weighted) ? SERAPH_BFS : Q.algo;
        uint32_t tile = gtile[Q.graph];
        if (gmap[Q.graph] == SERAPH_MAP_CTA) tile = std::min<uint32_t>(tile, kMaxCtaTile);
        qs[q] = QSpec{Q.graph, algo, Q.source, gmap[Q.graph], tile,
                      out_mem == SERAPH_MEM_DEVICE ? Q.out : nullptr, gdelta[Q.graph], pull_div};
    }
    return qs;
}

}  // namespace

int batch_run(seraph_bgraph* const* graphs_in, uint32_t ng, const seraph_query* qin, uint32_t nq,
              int out_mem, const seraph_batch_params* P, seraph_batch_stats* st) {
    SR_CHECK(graphs_in && qin && P && ng >= 1 && nq >= 1, SERAPH_EINVAL, "bad batch arguments");
    SR_CHECK(out_mem == SERAPH_MEM_HOST || out_mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad out_mem");
    SR_CHECK(P->mapping >= SERAPH_MAP_AUTO && P->mapping <= SERAPH_MAP_CTA, SERAPH_EINVAL, "bad mapping");
    SR_CHECK(P->tile == 0 || (P->tile <= (1u << 20)), SERAPH_EINVAL, "bad tile");
    SR_CHECK(P->group <= 1, SERAPH_EINVAL, "group must be 0 or 1");
    const bool group = P->group != 0;
    std::vector<seraph_bgraph*> graphs(graphs_in, graphs_in + ng);
    for (auto* g : graphs) SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
    SR_CUDA(cudaSetDevice(graphs[0]->device));
    Stream s;
    s.use(P->stream);
    seraph_batch_stats S{};
    std::vector<uint32_t> gmap, gtile;
    const std::vector<QSpec> qs = batch_specs(graphs, qin, nq, out_mem, P, s.s, S, gmap, gtile);
    std::vector<uint32_t*> dist(nq);
    Prepared pb;
    const Outcome o = launch_batch(pb, graphs, qs, P->use_graph != 0, P->replays, P->timeout_ms, s.s, &dist,
                                   group);
    if (out_mem == SERAPH_MEM_HOST)
        for (uint32_t q = 0; q < nq; ++q)
            SR_CUDA(cudaMemcpyAsync(qin[q].out, dist[q], graphs[qin[q].graph]->n * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, s.s));
    SR_CUDA(cudaStreamSynchronize(s.s));
    S.time_ms = o.ms;
    S.edges = o.edges;
    S.tasks = o.tasks;
    S.rounds_max = o.max_round;
    S.graph_captured = o.captured;
    for (uint32_t gi = 0; gi < ng && gi < 16; ++gi) { S.mapping[gi] = gmap[gi]; S.tile[gi] = gtile[gi]; }
    if (st) *st = S;
    return SERAPH_OK;
}

}  // namespace seraph

// A prepared batch (seraph_batch_plan_*): the queries' launch specs, their
// device tables and array pool, and the captured launch, kept between runs
// so that a run allocates nothing.
struct seraph_batch_plan {
    int device = 0;
    std::vector<seraph_bgraph*> graphs;
    std::vector<seraph::QSpec> qs;
    std::vector<uint32_t> rec, pos;  // each query's record and place in it
    seraph::Stream s;
    seraph::Prepared pb;
    seraph_batch_params P{};
    std::vector<uint32_t> gmap, gtile;
};

namespace seraph {
namespace {

// Round-0 tiles of a group record: its distinct sources over its tile.
uint32_t group_tiles0(const BGroupIO& io, const BQuery& b) {
    uint32_t distinct = 0;
    for (uint32_t j = 0; j < b.gsz; ++j) {
        bool seen = false;
        for (uint32_t i = 0; i < j && !seen; ++i) seen = io.src[i] == io.src[j];
        distinct += !seen;
    }
    return (distinct + b.tile - 1) / b.tile;
}

}  // namespace

int batch_plan_create(seraph_bgraph* const* graphs_in, uint32_t ng, const seraph_query* qin, uint32_t nq,
                      const seraph_batch_params* P, seraph_batch_plan** out) {
    SR_CHECK(out, SERAPH_EINVAL, "plan output must not be NULL");
    *out = nullptr;
    SR_CHECK(graphs_in && qin && P && ng >= 1 && nq >= 1, SERAPH_EINVAL, "bad batch arguments");
    SR_CHECK(P->mapping >= SERAPH_MAP_AUTO && P->mapping <= SERAPH_MAP_CTA, SERAPH_EINVAL, "bad mapping");
    SR_CHECK(P->tile == 0 || (P->tile <= (1u << 20)), SERAPH_EINVAL, "bad tile");
    SR_CHECK(P->group <= 1, SERAPH_EINVAL, "group must be 0 or 1");
    auto plan = std::make_unique<seraph_batch_plan>();
    plan->graphs.assign(graphs_in, graphs_in + ng);
    for (auto* g : plan->graphs) SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
    plan->device = plan->graphs[0]->device;
    SR_CUDA(cudaSetDevice(plan->device));
    plan->P = *P;
    plan->s.use(P->stream);
    seraph_batch_stats S{};
    plan->qs = batch_specs(plan->graphs, qin, nq, SERAPH_MEM_DEVICE, P, plan->s.s, S, plan->gmap, plan->gtile);
    prepare_batch(plan->pb, plan->graphs, plan->qs, P->use_graph != 0, P->timeout_ms, plan->s.s, nullptr,
                  P->group != 0);
    plan->rec.assign(nq, 0);
    plan->pos.assign(nq, 0);
    for (uint32_t ri = 0; ri < plan->pb.recs.size(); ++ri)
        for (uint32_t j = 0; j < plan->pb.recs[ri].size(); ++j) {
            plan->rec[plan->pb.recs[ri][j]] = ri;
            plan->pos[plan->pb.recs[ri][j]] = j;
        }
    *out = plan.release();
    return SERAPH_OK;
}

int batch_plan_run(seraph_batch_plan* plan, const uint32_t* sources, seraph_batch_stats* st) {
    SR_CHECK(plan, SERAPH_EINVAL, "null plan");
    SR_CUDA(cudaSetDevice(plan->device));
    Prepared& pb = plan->pb;
    const uint32_t nq = (uint32_t)plan->qs.size();
    if (sources) {
        for (uint32_t q = 0; q < nq; ++q)
            SR_CHECK(sources[q] < plan->graphs[plan->qs[q].graph]->n, SERAPH_EINVAL, "query source >= n");
        bool same_tiles = true;
        for (uint32_t q = 0; q < nq; ++q) {
            plan->qs[q].source = sources[q];
            BQuery& b = pb.qh[plan->rec[q]];
            BGroupIO& io = pb.ioh[plan->rec[q]];
            if (b.gsz == 1) {
                b.source = sources[q];
            } else {
                io.src[plan->pos[q]] = sources[q];
                if (plan->pos[q] == 0) b.source = sources[q];
            }
        }
        for (uint32_t ri = 0; ri < pb.nr; ++ri)
            if (pb.qh[ri].gsz > 1) same_tiles &= group_tiles0(pb.ioh[ri], pb.qh[ri]) == pb.ioh[ri].tiles0;
        if (same_tiles) {
            pb.upload(plan->s.s);
        } else {  // a group's round-0 task count changed (repeated sources, small tiles): rebuild
            prepare_batch(pb, plan->graphs, plan->qs, plan->P.use_graph != 0, plan->P.timeout_ms, plan->s.s,
                          nullptr, plan->P.group != 0);
        }
    }
    const Outcome o = run_batch(pb, 1, plan->s.s);
    if (st) {
        seraph_batch_stats S{};
        S.time_ms = o.ms;
        S.edges = o.edges;
        S.tasks = o.tasks;
        S.rounds_max = o.max_round;
        S.graph_captured = o.captured;
        for (uint32_t gi = 0; gi < plan->graphs.size() && gi < 16; ++gi) {
            S.mapping[gi] = plan->gmap[gi];
            S.tile[gi] = plan->gtile[gi];
        }
        *st = S;
    }
    return SERAPH_OK;
}

void batch_plan_free(seraph_batch_plan* plan) {
    if (!plan) return;
    cudaSetDevice(plan->device);
    delete plan;
}

}  // namespace seraph
