// Kernels of one local pass over the resident window (Sec. 3.2) with
// predictive vertex updating (Sec. 4), plus sweep-boundary kernels.
//
// A pass is
//   compact  -- every destination vertex of the window with in-degree > 0 is
//               tested against the prediction (strong thresholds of Table 1,
//               or the weak state machine of Fig. 6) and, if it must be
//               attempted, appended to one of three lists by in-degree class
//               (warp ballot + block scan + one atomic per block and class);
//   relax    -- a persistent grid pulls from the lists: one CTA per hub, one
//               warp per medium vertex, one thread per small vertex.  Pull
//               means only the owner writes a vertex, so min-updates need no
//               atomics and PageRank sums are deterministic.  Column indices
//               and weights are read with 128-bit loads;
//   apply    -- PageRank only: publish the pass's new values (Jacobi within a
//               pass, Gauss-Seidel across passes and steps).
// Every kernel first does its counter bookkeeping, then returns at once when
// the previous pass of the same step changed nothing (device-side flag: no
// host round trip per pass).
#include <algorithm>

#include "engine.cuh"
#include "leb128.cuh"

namespace seraph {
namespace {

constexpr int kNT = 256;
constexpr int kCompactRounds = 4;
constexpr uint32_t kCompactTile = kNT * kCompactRounds;

// Gathered source value (weak load: values may change during a pass).
__device__ __forceinline__ uint32_t ld_gather(const void* p, uint64_t pol) {
    uint32_t r;
    asm("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

// Four weights of edges idx..idx+3 (idx a multiple of 4) stored WB bytes wide.
template <int WB>
__device__ __forceinline__ void ld_weights4(const uint8_t* w, uint32_t idx, uint32_t out[4],
                                            uint64_t pol) {
    if (WB == 1) {
        const uint32_t v = ld_stream(w + idx, pol);
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = (v >> (8 * k)) & 0xFFu;
    } else if (WB == 2) {
        const uint2 v = ld_stream2(w + 2 * (uint64_t)idx, pol);
        out[0] = v.x & 0xFFFFu; out[1] = v.x >> 16; out[2] = v.y & 0xFFFFu; out[3] = v.y >> 16;
    } else {
        const uint4 v = ld_stream4(w + 4 * (uint64_t)idx, pol);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    }
}

__device__ __forceinline__ uint32_t find_page(const uint32_t* vb, uint32_t first, uint32_t end,
                                              uint32_t v) {
    uint32_t lo = first, hi = end - 1;
    while (lo < hi) {  // largest p in [first, end) with vb[p] <= v
        uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(vb + mid) <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ----------------------------------------------------------- accumulators

struct MinAcc {
    uint32_t best;
    bool ovf;
};

struct SumAcc {
    float s, c;  // compensated sum: value = s - c
};

template <int ALGO>
__device__ __forceinline__ void min_edge(MinAcc& acc, uint32_t u, uint32_t w,
                                         const uint32_t* __restrict__ val) {
    uint32_t du = val[u];
    if (ALGO == ALG_CC) {
        acc.best = min(acc.best, du);
    } else if (du != SERAPH_INF) {
        uint32_t s = du + (ALGO == ALG_SSSP ? w : 1u);
        if (s < du || s == SERAPH_INF) acc.ovf = true;
        else acc.best = min(acc.best, s);
    }
}

template <bool KAHAN>
__device__ __forceinline__ void sum_add(SumAcc& acc, float x) {
    if (KAHAN) {
        float y = x - acc.c;
        float t = acc.s + y;
        acc.c = (t - acc.s) - y;
        acc.s = t;
    } else {
        acc.s += x;
    }
}

template <bool KAHAN>
__device__ __forceinline__ SumAcc sum_merge(SumAcc a, SumAcc b) {
    if (!KAHAN) return SumAcc{a.s + b.s, 0.f};
    float y = (b.s - b.c) - a.c;
    float t = a.s + y;
    SumAcc r;
    r.c = (t - a.s) - y;
    r.s = t;
    return r;
}

// Per-thread counters, flushed once per kernel.
struct Locals {
    unsigned changed;
    unsigned minv;
    unsigned ovf;
    unsigned long long edges;
};

__device__ __forceinline__ uint8_t fsm_next(const AlgoArgs& a, uint32_t st, uint32_t c) {
    return (uint8_t)((a.fsm_bits >> (3 * (2 * st + c))) & 7u);
}

__device__ __forceinline__ uint8_t fsm_step(const AlgoArgs& a, uint8_t st, bool ch) {
    // A dormant state reached here only because prediction is off for the
    // pass: a valid update follows its "changed" edge, otherwise it keeps its
    // state (its ticks belong to predicted passes).
    if ((a.skip_mask >> st) & 1) return ch ? fsm_next(a, st, 1) : st;
    return fsm_next(a, st, ch ? 1 : 0);
}

// The vertex's own value and prediction state, loaded when its processing
// starts so that their latency overlaps the gathers (only the thread
// processing v in this pass writes them).
struct Own {
    uint32_t old;  // SSSP/BFS/CC value
    float xo;      // PageRank value
    uint8_t st;    // weak-prediction state
};

template <int ALGO>
__device__ __forceinline__ Own load_own(const AlgoArgs& a, uint32_t v) {
    Own o{0u, 0.f, 0};
    if (ALGO == ALG_PR) o.xo = a.x[v];
    else o.old = a.val[v];
    if (a.pvu == SERAPH_PVU_WEAK) o.st = a.state[v];
    return o;
}

template <int ALGO>
__device__ __forceinline__ void finish_min(const AlgoArgs& a, uint32_t v, const MinAcc& acc,
                                           uint32_t deg, Locals& L, const Own& o) {
    bool ch = acc.best < o.old;
    if (ch) {
        a.val[v] = acc.best;
        if (a.chg_stamp) a.chg_stamp[v] = a.chg_tag;
    }
    if (ALGO == ALG_SSSP && acc.ovf && acc.best == SERAPH_INF && o.old == SERAPH_INF) L.ovf = 1;
    if (a.pvu == SERAPH_PVU_WEAK) {
        const uint8_t ns = fsm_step(a, o.st, ch);
        if (ns != o.st) a.state[v] = ns;
    }
    L.changed += ch;
    L.edges += deg;
    if (ch) L.minv = min(L.minv, acc.best);
}

__device__ __forceinline__ void finish_pr(const AlgoArgs& a, uint32_t v, float sum, float base,
                                          uint32_t deg, Locals& L, const Own& o) {
    float xn = base + a.damping * sum;
    a.x_next[v] = xn;
    bool ch = fabsf(xn - o.xo) > a.fail_eps * o.xo;
    if (a.pvu == SERAPH_PVU_WEAK) {
        const uint8_t ns = fsm_step(a, o.st, ch);
        if (ns != o.st) a.state[v] = ns;
    }
    L.changed += ch;
    L.edges += deg;
}

// ------------------------------------------------------------- one vertex

// Gather-and-reduce over edges idx0..idx0+3 and idx1..idx1+3 (both multiples
// of 4) restricted to [b, e).  All eight column and gathered-value loads are
// issued before any is used; lanes outside the range gather a valid address
// (zero padding or a neighbour's column) and drop the value.
template <int ALGO, bool KAHAN, int WB>
__device__ __forceinline__ void gather8(const AlgoArgs& a, const PageLoc& loc, uint32_t b,
                                        uint32_t e, uint32_t idx0, uint32_t idx1, MinAcc& macc,
                                        SumAcc& sacc) {
    const bool two = idx1 < e;
    const uint64_t pn = policy_evict_normal();
    const uint64_t ps = a.hints ? policy_evict_first() : pn;
    const uint64_t ph = a.hints ? policy_evict_last() : pn;
    const uint4 c0 = ld_stream4(loc.col + idx0, ps);
    const uint4 c1 = two ? ld_stream4(loc.col + idx1, ps) : make_uint4(0, 0, 0, 0);
    uint32_t w[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    if (ALGO == ALG_SSSP) {
        ld_weights4<WB>(loc.w, idx0, w, ps);
        if (two) ld_weights4<WB>(loc.w, idx1, w + 4, ps);
    }
    const uint32_t cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    if (ALGO == ALG_PR) {
        float g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            g[j] = __uint_as_float(ld_gather(a.contrib + cc[j], cc[j] < a.hot ? ph : pn));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t i = (j < 4 ? idx0 : idx1) + (j & 3);
            if (i >= b && i < e && (j < 4 || two)) sum_add<KAHAN>(sacc, g[j]);
        }
    } else {
        uint32_t g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = ld_gather(a.val + cc[j], cc[j] < a.hot ? ph : pn);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t i = (j < 4 ? idx0 : idx1) + (j & 3);
            if (i >= b && i < e && (j < 4 || two)) {
                const uint32_t du = g[j];
                if (ALGO == ALG_CC) {
                    macc.best = min(macc.best, du);
                } else if (du != SERAPH_INF) {
                    const uint32_t s = du + (ALGO == ALG_SSSP ? w[j] : 1u);
                    if (s < du || s == SERAPH_INF) macc.ovf = true;
                    else macc.best = min(macc.best, s);
                }
            }
        }
    }
}

template <int WB>
__device__ __forceinline__ uint32_t ld_weight1(const uint8_t* w, uint32_t idx, uint64_t pol) {
    uint32_t r;
    if (WB == 1)
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(r) : "l"(w + idx), "l"(pol));
    else if (WB == 2)
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=r"(r) : "l"(w + 2 * (uint64_t)idx), "l"(pol));
    else
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(w + 4 * (uint64_t)idx), "l"(pol));
    return r;
}

// Gathers and reduction of a decoded piece, eight codes in flight at a time,
// in code order: the code at byte j has id run + lid[j] (run = the id before
// the piece; 0xFFFFFFFF before a destination's first) and edge index
// e0 + ord + (codes before j in the piece).
template <int ALGO, bool KAHAN, int WB>
__device__ __forceinline__ void piece_gather(const AlgoArgs& a, const PageLoc& loc, uint32_t e0,
                                             uint32_t st, const uint32_t lid[16], uint32_t run,
                                             uint32_t ord, MinAcc& macc, SumAcc& sacc) {
    const uint64_t pn = policy_evict_normal();
    const uint64_t ps = a.hints ? policy_evict_first() : pn;
    const uint64_t ph = a.hints ? policy_evict_last() : pn;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!((st >> (8 * h)) & 0xFFu)) continue;
        uint32_t id[8], wt[8];
        bool ok[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = 8 * h + k;
            id[k] = run + lid[j];
            ok[k] = ((st >> j) & 1u) && id[k] < a.n;  // a corrupt stream reads nothing
            if (ALGO == ALG_SSSP)
                wt[k] = ok[k] ? ld_weight1<WB>(loc.w, e0 + ord + __popc(st & ((1u << j) - 1u)), ps) : 0u;
        }
        if (ALGO == ALG_PR) {
            float g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                g[k] = ok[k] ? __uint_as_float(ld_gather(a.contrib + id[k], id[k] < a.hot ? ph : pn))
                             : 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (ok[k]) sum_add<KAHAN>(sacc, g[k]);
        } else {
            uint32_t g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                g[k] = ok[k] ? ld_gather(a.val + id[k], id[k] < a.hot ? ph : pn) : SERAPH_INF;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (!ok[k]) continue;
                const uint32_t du = g[k];
                if (ALGO == ALG_CC) {
                    macc.best = min(macc.best, du);
                } else if (du != SERAPH_INF) {
                    const uint32_t s = du + (ALGO == ALG_SSSP ? wt[k] : 1u);
                    if (s < du || s == SERAPH_INF) macc.ovf = true;
                    else macc.best = min(macc.best, s);
                }
            }
        }
    }
}

// Thread per vertex: the pieces one after another, the running id carried.
template <int ALGO, bool KAHAN, int WB>
__device__ __forceinline__ void edges_packed_serial(const AlgoArgs& a, const PageLoc& loc,
                                                    uint32_t li, uint32_t e0, MinAcc& macc,
                                                    SumAcc& sacc) {
    const uint8_t* d = (const uint8_t*)loc.col;
    const uint32_t B = loc.boff[li], Eb = loc.boff[li + 1];
    const uint64_t ps = a.hints ? policy_evict_first() : policy_evict_normal();
    const uint32_t A = B & ~15u;
    uint32_t run = 0xFFFFFFFFu, ord = 0;
    for (uint32_t c = A; c < Eb; c += 16) {
        const Piece P = load_piece(d, c, A, Eb, ps);
        const uint32_t st = leb_starts(P.w0, P.w1, P.w2, P.w3, P.pt, c, B, Eb);
        uint32_t lid[16];
        const uint32_t sum = piece_decode(P, st, lid);
        piece_gather<ALGO, KAHAN, WB>(a, loc, e0, st, lid, run, ord, macc, sacc);
        run += sum;
        ord += __popc(st);
    }
}

// G lanes per vertex (G = 4, 8, 32; every lane of the warp calls this with a
// warp-uniform trip count): lane t takes pieces t, t+G, ... and a width-G
// scan of (count, sum) places its ids.
template <int ALGO, bool KAHAN, int WB, int G>
__device__ __forceinline__ void edges_packed_group(const AlgoArgs& a, const PageLoc& loc,
                                                   bool valid, uint32_t li, uint32_t e0,
                                                   uint32_t t, MinAcc& macc, SumAcc& sacc) {
    const uint8_t* d = (const uint8_t*)loc.col;
    uint32_t B = 0, Eb = 0;
    if (valid) { B = loc.boff[li]; Eb = loc.boff[li + 1]; }
    const uint64_t ps = a.hints ? policy_evict_first() : policy_evict_normal();
    const uint32_t A = B & ~15u;
    const uint32_t pieces = Eb > A ? (Eb - A + 15u) >> 4 : 0u;
    const uint32_t iters = __reduce_max_sync(kFull, (pieces + G - 1) / G);
    uint32_t run = 0xFFFFFFFFu, ord = 0;
    for (uint32_t it = 0; it < iters; ++it) {
        const uint32_t c = A + 16u * (it * G + t);
        const bool act = valid && c < Eb;
        Piece P{0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t st = 0;
        if (act) {
            P = load_piece(d, c, A, Eb, ps);
            st = leb_starts(P.w0, P.w1, P.w2, P.w3, P.pt, c, B, Eb);
        }
        uint32_t lid[16];
        const uint64_t x = ((uint64_t)__popc(st) << 32) | piece_decode(P, st, lid);
        uint64_t inc = x;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const uint64_t y = __shfl_up_sync(kFull, inc, o, G);
            if (t >= (uint32_t)o) inc += y;
        }
        const uint64_t ex = inc - x;
        const uint64_t tot = __shfl_sync(kFull, inc, G - 1, G);
        if (st)
            piece_gather<ALGO, KAHAN, WB>(a, loc, e0, st, lid, run + (uint32_t)ex,
                                          ord + (uint32_t)(ex >> 32), macc, sacc);
        run += (uint32_t)tot;
        ord += (uint32_t)(tot >> 32);
    }
}

// The whole CTA on one vertex: as above with a block-wide scan.
template <int ALGO, bool KAHAN, int WB>
__device__ __forceinline__ void edges_packed_cta(const AlgoArgs& a, const PageLoc& loc, uint32_t li,
                                                 uint32_t e0, MinAcc& macc, SumAcc& sacc,
                                                 unsigned long long* ws) {
    const uint8_t* d = (const uint8_t*)loc.col;
    const uint32_t B = loc.boff[li], Eb = loc.boff[li + 1];
    const uint64_t ps = a.hints ? policy_evict_first() : policy_evict_normal();
    const uint32_t A = B & ~15u;
    const uint32_t pieces = Eb > A ? (Eb - A + 15u) >> 4 : 0u;
    const uint32_t iters = (pieces + kNT - 1) / kNT;
    uint32_t run = 0xFFFFFFFFu, ord = 0;
    for (uint32_t it = 0; it < iters; ++it) {
        const uint32_t c = A + 16u * (it * kNT + threadIdx.x);
        const bool act = c < Eb;
        Piece P{0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t st = 0;
        if (act) {
            P = load_piece(d, c, A, Eb, ps);
            st = leb_starts(P.w0, P.w1, P.w2, P.w3, P.pt, c, B, Eb);
        }
        uint32_t lid[16];
        const unsigned long long x =
            ((unsigned long long)__popc(st) << 32) | piece_decode(P, st, lid);
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>(x, ws, &tot);
        if (st)
            piece_gather<ALGO, KAHAN, WB>(a, loc, e0, st, lid, run + (uint32_t)ex,
                                          ord + (uint32_t)(ex >> 32), macc, sacc);
        run += (uint32_t)tot;
        ord += (uint32_t)(tot >> 32);
    }
}

template <int ALGO, bool KAHAN, int WB, bool PK>
__device__ __forceinline__ void vertex_thread(const AlgoArgs& a, unsigned long long ent, float base,
                                              Locals& L) {
    const uint32_t v = (uint32_t)ent, p = (uint32_t)(ent >> 32);
    const PageLoc loc = a.loc[p];
    const uint32_t li = v - loc.vb;
    const Own own = load_own<ALGO>(a, v);
    const uint32_t b = loc.off[li], e = loc.off[li + 1];
    MinAcc macc{SERAPH_INF, false};
    SumAcc sacc{0.f, 0.f};
    if constexpr (PK) {
        edges_packed_serial<ALGO, KAHAN, WB>(a, loc, li, b, macc, sacc);
    } else {
        for (uint32_t idx = b & ~3u; idx < e; idx += 8) {
            gather8<ALGO, KAHAN, WB>(a, loc, b, e, idx, idx + 4, macc, sacc);
            if (ALGO == ALG_BFS && macc.best <= a.bfs_lb) break;  // no smaller level exists
        }
    }
    if (ALGO == ALG_PR) finish_pr(a, v, sacc.s - sacc.c, base, e - b, L, own);
    else finish_min<ALGO>(a, v, macc, e - b, L, own);
}

// Group of G lanes (G = 32: a warp; G = CTA size for hubs).  Lane t reads the
// aligned 16-byte column vectors t and t+G of every 8G-edge stretch of the
// vertex's range [b, e).
template <int ALGO, bool KAHAN, int WB>
__device__ __forceinline__ void edges_strided(const AlgoArgs& a, const PageLoc& loc, uint32_t b,
                                              uint32_t e, uint32_t t, uint32_t G, MinAcc& macc,
                                              SumAcc& sacc) {
    for (uint32_t idx = (b & ~3u) + 4 * t; idx < e; idx += 8 * G) {
        gather8<ALGO, KAHAN, WB>(a, loc, b, e, idx, idx + 4 * G, macc, sacc);
        if (ALGO == ALG_BFS && macc.best <= a.bfs_lb) break;  // this lane can find nothing smaller
    }
}

// One vertex per group of G lanes (G = 4, 8 or 32), 32/G vertices per warp
// at once so that their dependent load chains (list entry, page location,
// offsets, columns, gathered values) overlap.  Every lane of the warp calls
// this (inactive groups pass valid = false) because the group reduction
// shuffles across the whole warp; xor offsets below G stay inside a group.
template <int ALGO, bool KAHAN, int WB, int G, bool PK>
__device__ __forceinline__ void vertex_group(const AlgoArgs& a, unsigned long long ent, bool valid,
                                             float base, Locals& L) {
    const uint32_t t = lane_id() & (G - 1);
    MinAcc macc{SERAPH_INF, false};
    SumAcc sacc{0.f, 0.f};
    uint32_t v = 0, b = 0, e = 0;
    Own own{0u, 0.f, 0};
    if constexpr (PK) {
        PageLoc loc{};
        uint32_t li = 0;
        if (valid) {
            v = (uint32_t)ent;
            if (t == 0) own = load_own<ALGO>(a, v);
            loc = a.loc[(uint32_t)(ent >> 32)];
            li = v - loc.vb;
            b = loc.off[li];
            e = loc.off[li + 1];
        }
        edges_packed_group<ALGO, KAHAN, WB, G>(a, loc, valid, li, b, t, macc, sacc);
    } else if (valid) {
        v = (uint32_t)ent;
        if (t == 0) own = load_own<ALGO>(a, v);
        const PageLoc loc = a.loc[(uint32_t)(ent >> 32)];
        const uint32_t li = v - loc.vb;
        b = loc.off[li];
        e = loc.off[li + 1];
        edges_strided<ALGO, KAHAN, WB>(a, loc, b, e, t, G, macc, sacc);
    }
    if (ALGO == ALG_PR) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            SumAcc other{__shfl_xor_sync(kFull, sacc.s, o), __shfl_xor_sync(kFull, sacc.c, o)};
            sacc = (t & o) ? sum_merge<KAHAN>(other, sacc) : sum_merge<KAHAN>(sacc, other);
        }
        if (valid && t == 0) finish_pr(a, v, sacc.s - sacc.c, base, e - b, L, own);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            macc.best = min(macc.best, __shfl_xor_sync(kFull, macc.best, o));
            macc.ovf |= __shfl_xor_sync(kFull, (int)macc.ovf, o) != 0;
        }
        if (valid && t == 0) finish_min<ALGO>(a, v, macc, e - b, L, own);
    }
}

template <int ALGO, bool KAHAN, int WB, bool PK>
__device__ __forceinline__ void vertex_cta(const AlgoArgs& a, unsigned long long ent, float base,
                                           Locals& L, float* s_sum, float* s_comp,
                                           unsigned* s_min, unsigned* s_ovf,
                                           unsigned long long* s_scan) {
    const uint32_t v = (uint32_t)ent, p = (uint32_t)(ent >> 32);
    const PageLoc loc = a.loc[p];
    const uint32_t li = v - loc.vb;
    const uint32_t b = loc.off[li], e = loc.off[li + 1];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    Own own{0u, 0.f, 0};
    if (threadIdx.x == 0) own = load_own<ALGO>(a, v);
    MinAcc macc{SERAPH_INF, false};
    SumAcc sacc{0.f, 0.f};
    if constexpr (PK) edges_packed_cta<ALGO, KAHAN, WB>(a, loc, li, b, macc, sacc, s_scan);
    else edges_strided<ALGO, KAHAN, WB>(a, loc, b, e, threadIdx.x, kNT, macc, sacc);
    if (ALGO == ALG_PR) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            SumAcc other{__shfl_xor_sync(kFull, sacc.s, o), __shfl_xor_sync(kFull, sacc.c, o)};
            sacc = (lane & o) ? sum_merge<KAHAN>(other, sacc) : sum_merge<KAHAN>(sacc, other);
        }
        if (lane == 0) { s_sum[warp] = sacc.s; s_comp[warp] = sacc.c; }
        __syncthreads();
        if (threadIdx.x == 0) {
            SumAcc t{s_sum[0], s_comp[0]};
            for (int w = 1; w < kNT / 32; ++w) t = sum_merge<KAHAN>(t, SumAcc{s_sum[w], s_comp[w]});
            finish_pr(a, v, t.s - t.c, base, e - b, L, own);
        }
    } else {
        macc.best = __reduce_min_sync(kFull, macc.best);
        macc.ovf = __any_sync(kFull, macc.ovf);
        if (lane == 0) { s_min[warp] = macc.best; s_ovf[warp] = macc.ovf; }
        __syncthreads();
        if (threadIdx.x == 0) {
            MinAcc t{s_min[0], s_ovf[0] != 0};
            for (int w = 1; w < kNT / 32; ++w) { t.best = min(t.best, s_min[w]); t.ovf |= s_ovf[w] != 0; }
            finish_min<ALGO>(a, v, t, e - b, L, own);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void flush_locals(const AlgoArgs& a, int par, uint32_t step, Locals L) {
    unsigned ch = __reduce_add_sync(kFull, L.changed);
    unsigned mn = __reduce_min_sync(kFull, L.minv);
    unsigned ov = __reduce_or_sync(kFull, L.ovf);
    unsigned long long ed = L.edges;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ed += __shfl_xor_sync(kFull, ed, o);
    if (lane_id() == 0) {
        RunState* rs = a.rs;
        if (ch) {
            atomicAdd(&rs->pass_changed[par], ch);
            atomicAdd(&rs->cur.changed, (unsigned long long)ch);
            atomicAdd(&a.step_changed[step & a.step_mask], ch);
        }
        if (mn != SERAPH_INF) atomicMin(&rs->thr_cur, mn);
        if (ov) atomicOr(&rs->cur.overflow, 1u);
        if (ed) atomicAdd(&rs->cur.edges, ed);
    }
}

// ---------------------------------------------------------------- kernels

__global__ void gate_kernel(RunState* rs, uint32_t pass, int check_prev, int idle,
                            uint32_t want_loaded, uint32_t j, int learned, unsigned* rec_gains) {
    const int par = pass & 1;
    if (rec_gains && j > 0) rec_gains[j - 1] = rs->pass_changed[par ^ 1];
    bool go = true;
    if (check_prev && rs->pass_changed[par ^ 1] == 0) go = false;
    if (idle && (int)(*(volatile unsigned*)&rs->loaded - want_loaded) >= 0) go = false;
    if (learned && j >= rs->k_limit) go = false;
    if (go) rs->step_passes += 1;
    rs->pass_go[par] = go;
    for (int k = 0; k < 8; ++k) rs->work[par][k] = 0;
    rs->pass_changed[par] = 0;
    if (go) rs->cur.passes_run += 1;
    else rs->cur.passes_skipped += 1;
}

// Vertices of the window to attempt, by in-degree class, in vertex order
// within each block: warp w of a block takes vertices [v0 + 128w, +128) in
// four rounds of 32; per class, ballots give each lane its place, one shared
// exchange gives each warp its offset, one atomic per class and block
// reserves the block's run of the list.
template <int ALGO>
__global__ void __launch_bounds__(kNT) compact_kernel(WindowDesc wd, AlgoArgs a, uint32_t pass,
                                                      int predict) {
    constexpr int kWarps = kNT / 32;
    __shared__ unsigned s_cnt[kWarps][kClasses + 2];
    __shared__ unsigned s_off[kWarps][kClasses];
    __shared__ unsigned long long s_pk[kWarps][2];
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (!rs->pass_go[par]) return;

    int c = 0;
    while (c + 1 < (int)wd.nchunks && blockIdx.x >= wd.c[c + 1].block_begin) ++c;
    const ChunkDesc cd = wd.c[c];
    const bool strong = predict && a.pvu == SERAPH_PVU_STRONG;
    const bool weak = predict && a.pvu == SERAPH_PVU_WEAK;
    uint32_t thr = 0;
    if (strong) thr = ALGO == ALG_BFS ? rs->sweeps_done : min(rs->thr_prev, rs->thr_cur);

    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t vw = cd.v_begin + (blockIdx.x - cd.block_begin) * kCompactTile + warp * 32 * kCompactRounds;
    int my_cls[kCompactRounds];
    uint32_t my_p[kCompactRounds];
    unsigned n_att = 0, n_skip = 0;
    unsigned pk_edges = 0, pk_bytes = 0;  // attempted in-edges / code bytes on packed pages
#pragma unroll
    for (int r = 0; r < kCompactRounds; ++r) {
        my_cls[r] = -1;
        my_p[r] = 0;
        const uint32_t v = vw + r * 32 + lane;
        if (v >= vw && v < cd.v_end) {
            const uint32_t p = find_page(a.vb, cd.first_page, cd.end_page, v);
            const PageLoc loc = a.loc[p];
            const uint32_t li = v - loc.vb;
            const uint32_t deg = loc.off[li + 1] - loc.off[li];
            if (deg > 0 || ALGO == ALG_PR) {
                bool skip = false;
                if (strong) {
                    skip = a.val[v] <= thr;
                } else if (weak) {
                    const uint8_t st = a.state[v];
                    if ((a.skip_mask >> st) & 1) {
                        skip = true;
                        a.state[v] = fsm_next(a, st, 0);  // dormant tick
                    }
                }
                if (skip) {
                    ++n_skip;
                } else {
                    ++n_att;
                    if (loc.boff) {
                        pk_edges += deg;
                        pk_bytes += loc.boff[li + 1] - loc.boff[li];
                    }
                    my_cls[r] = deg <= a.cls_max[0] ? 0
                              : deg <= a.cls_max[1] ? 1
                              : deg <= a.cls_max[2] ? 2
                              : deg <= a.cls_max[3] ? 3 : 4;
                    my_p[r] = p;
                }
            }
        }
    }
    unsigned m[kCompactRounds][kClasses];
    unsigned cnt[kClasses];
#pragma unroll
    for (int k = 0; k < kClasses; ++k) {
        cnt[k] = 0;
#pragma unroll
        for (int r = 0; r < kCompactRounds; ++r) {
            m[r][k] = __ballot_sync(kFull, my_cls[r] == k);
            cnt[k] += __popc(m[r][k]);
        }
    }
    n_att = __reduce_add_sync(kFull, n_att);
    n_skip = __reduce_add_sync(kFull, n_skip);
    unsigned long long pe = pk_edges, pb = pk_bytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pe += __shfl_xor_sync(kFull, pe, o);
        pb += __shfl_xor_sync(kFull, pb, o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kClasses; ++k) s_cnt[warp][k] = cnt[k];
        s_cnt[warp][kClasses] = n_att;
        s_cnt[warp][kClasses + 1] = n_skip;
        s_pk[warp][0] = pe;
        s_pk[warp][1] = pb;
    }
    __syncthreads();
    if (threadIdx.x < kClasses) {  // thread k: class k's run of the list for this block
        const unsigned k = threadIdx.x;
        unsigned tot = 0;
        for (int w = 0; w < kWarps; ++w) tot += s_cnt[w][k];
        unsigned base = tot ? atomicAdd(&rs->list_cnt[par][k], tot) : 0u;
        for (int w = 0; w < kWarps; ++w) {
            s_off[w][k] = base;
            base += s_cnt[w][k];
        }
    } else if (threadIdx.x == 32) {
        unsigned att = 0, sk = 0;
        for (int w = 0; w < kWarps; ++w) { att += s_cnt[w][kClasses]; sk += s_cnt[w][kClasses + 1]; }
        if (att) atomicAdd(&rs->cur.attempted, (unsigned long long)att);
        if (sk) atomicAdd(&rs->cur.skipped, (unsigned long long)sk);
        unsigned long long pe = 0, pb = 0;
        for (int w = 0; w < kWarps; ++w) { pe += s_pk[w][0]; pb += s_pk[w][1]; }
        if (pe) {
            atomicAdd(&rs->cur.packed_edges, pe);
            atomicAdd(&rs->cur.code_bytes, pb);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kClasses; ++k) {
        unsigned pos = s_off[warp][k];
#pragma unroll
        for (int r = 0; r < kCompactRounds; ++r) {
            if (my_cls[r] == k)
                a.list[k][pos + __popc(m[r][k] & lanemask_lt())] =
                    ((unsigned long long)my_p[r] << 32) | (vw + r * 32 + lane);
            pos += __popc(m[r][k]);
        }
    }
}

// Class-k list (k = 1, 2, 3) with G lanes per vertex: each warp grabs
// 4 * 32/G entries at a time.
template <int ALGO, bool KAHAN, int WB, int G, bool PK>
__device__ __forceinline__ void group_phase(const AlgoArgs& a, int par, int k, float base,
                                            Locals& L) {
    constexpr unsigned per = 32 / G;
    const unsigned n = a.rs->list_cnt[par][k];
    const unsigned lane = lane_id(), grp = lane / G;
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(&a.rs->work[par][k], 4 * per);
        i0 = __shfl_sync(kFull, i0, 0);
        if (i0 >= n) break;
#pragma unroll 1
        for (unsigned r = 0; r < 4; ++r) {
            const unsigned i = i0 + r * per + grp;
            const bool valid = i < n;
            vertex_group<ALGO, KAHAN, WB, G, PK>(a, valid ? a.list[k][i] : 0ull, valid, base, L);
        }
    }
}

// Six CTAs per SM (<= 42 registers) keep enough warps in flight for the
// gathers (PageRank's compensated sums would otherwise take 48); SSSP's
// weights need more registers, five CTAs (<= 51).
template <int ALGO, bool KAHAN, int WB, bool PK>
__global__ void __launch_bounds__(kNT, PK ? 4 : (ALGO == ALG_SSSP ? 5 : 6))
    relax_kernel(AlgoArgs a, uint32_t pass, uint32_t step) {
    __shared__ unsigned s_item;
    __shared__ unsigned long long s_scan[kNT / 32 + 1];
    __shared__ float s_sum[kNT / 32], s_comp[kNT / 32];
    __shared__ unsigned s_min[kNT / 32], s_ovf[kNT / 32];
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (blockIdx.x == 0 && threadIdx.x < 8) rs->list_cnt[par ^ 1][threadIdx.x] = 0;
    if (!rs->pass_go[par]) return;
    const float base = ALGO == ALG_PR ? rs->base : 0.f;
    Locals L{0u, SERAPH_INF, 0u, 0ull};

    const unsigned n_cta = rs->list_cnt[par][4];
    for (;;) {  // one CTA per hub vertex
        if (threadIdx.x == 0) s_item = atomicAdd(&rs->work[par][4], 1u);
        __syncthreads();
        const unsigned i = s_item;
        __syncthreads();
        if (i >= n_cta) break;
        vertex_cta<ALGO, KAHAN, WB, PK>(a, a.list[4][i], base, L, s_sum, s_comp, s_min, s_ovf,
                                        s_scan);
    }
    group_phase<ALGO, KAHAN, WB, 32, PK>(a, par, 3, base, L);
    group_phase<ALGO, KAHAN, WB, 8, PK>(a, par, 2, base, L);
    group_phase<ALGO, KAHAN, WB, 4, PK>(a, par, 1, base, L);
    const unsigned lane = lane_id();
    const unsigned n0 = rs->list_cnt[par][0];
    for (;;) {  // one thread per small vertex, 128 per warp grab
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(&rs->work[par][0], 128u);
        i0 = __shfl_sync(kFull, i0, 0);
        if (i0 >= n0) break;
#pragma unroll
        for (unsigned j = 0; j < 4; ++j) {
            const unsigned i = i0 + j * 32 + lane;
            if (i < n0) vertex_thread<ALGO, KAHAN, WB, PK>(a, a.list[0][i], base, L);
        }
    }
    flush_locals(a, par, step, L);
}

// Publishes a pass's new PageRank values (Jacobi within the pass): x and
// contrib = x / outdeg of every attempted vertex, optionally over-relaxed.
__global__ void __launch_bounds__(kNT) pr_apply_kernel(AlgoArgs a, uint32_t pass) {
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (!rs->pass_go[par]) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < kClasses; ++k) {
        const unsigned nk = rs->list_cnt[par][k];
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nk; i += stride) {
            const uint32_t v = (uint32_t)a.list[k][i];
            float xn = a.x_next[v];
            if (a.omega != 1.0f) {  // over-relaxed: x + omega (x_next - x), kept >= 0
                const float xo = a.x[v];
                xn = fmaxf(fmaf(a.omega, xn - xo, xo), 0.0f);
            }
            a.x[v] = xn;
            a.contrib[v] = xn * a.inv_out[v];
        }
    }
}

__global__ void set_locs_kernel(PageLoc* loc, const uint32_t* vb, uint32_t first, uint32_t end,
                                const uint64_t* rel_soff, const uint64_t* rel_woff,
                                const uint64_t* off_bytes, uint8_t* sbase, uint8_t* wbase,
                                bool packed, RunState* rs, uint32_t seq) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *(volatile unsigned*)&rs->loaded = seq;
    for (uint32_t p = first + blockIdx.x * blockDim.x + threadIdx.x; p < end;
         p += gridDim.x * blockDim.x) {
        PageLoc L;
        const uint8_t* s = sbase + rel_soff[p];
        L.off = (const uint32_t*)s;
        L.boff = packed ? (const uint32_t*)(s + off_bytes[p]) : nullptr;
        L.col = (const uint32_t*)(s + (packed ? 2 : 1) * off_bytes[p]);
        L.w = wbase ? wbase + rel_woff[p] : nullptr;
        L.vb = vb[p];
        L.nv = vb[p + 1] - vb[p];
        loc[p] = L;
    }
}

// CC labels start at the caller's vertex id (label0 = internal -> caller id
// map of a reordered graph, or null for the identity), so the fixpoint label
// is the smallest caller id in the component whatever the internal order.
__global__ void init_min_kernel(uint32_t* val, uint8_t* state, uint64_t n, int algo,
                                uint32_t source, const uint32_t* __restrict__ label0) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        val[v] = algo == ALG_CC ? (label0 ? label0[v] : (uint32_t)v)
                                : (v == source ? 0u : SERAPH_INF);
        if (state) state[v] = 0;
    }
}

__global__ void init_pr_kernel(const uint32_t* outdeg, float* x, float* contrib, float* x_prev,
                               float* inv_out, uint8_t* state, uint64_t n) {
    const float x0 = (float)(1.0 / (double)n);
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t od = outdeg[v];
        const float io = od ? 1.0f / (float)od : 0.0f;
        inv_out[v] = io;
        x[v] = x0;
        x_prev[v] = x0;
        contrib[v] = x0 * io;
        if (state) state[v] = 0;
    }
}

__global__ void step_epilogue_kernel(RunState* rs, ChunkDyn* cd, uint32_t chunk,
                                     uint32_t last_pass, uint32_t npass, unsigned* rec_gains) {
    const unsigned last = rs->pass_changed[last_pass & 1];
    if (rec_gains && npass > 0) rec_gains[npass - 1] = last;
    if (cd) {
        ChunkDyn d = cd[chunk];
        d.visits += 1;
        d.last_passes = rs->step_passes;
        for (int k = 0; k < 4; ++k) d.gains[k] = 0;
        if (rec_gains)
            for (uint32_t k = 0; k < 4 && k < npass; ++k) d.gains[k] = rec_gains[k];
        cd[chunk] = d;
    }
}

__global__ void close_min_kernel(RunState* rs, SweepReport* out) {
    SweepReport r = rs->cur;
    r.thr_min = rs->thr_cur;
    rs->prev_changed = r.changed;
    *out = r;
    rs->thr_prev = rs->thr_cur;
    rs->thr_cur = SERAPH_INF;
    rs->sweeps_done += 1;
    rs->cur = SweepReport{};
}

// Fixed-order FP64 reduction of `nparts` partials by one block.
__device__ double reduce_partials(const double* partial, int nparts, double* ws) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kNT) s += partial[i];
    double tot;
    block_excl_scan<kNT>(s, ws, &tot);
    return tot;
}

// The sweep-close kernels stream whole vertex arrays: 16-byte vector accesses
// when every array is 16-byte aligned (the tail, or everything otherwise, one
// element at a time), all loads of an element before its stores.  The
// element -> thread mapping depends only on n and the grid, so the partial
// sums are deterministic.
__device__ __forceinline__ bool aligned16(const void* a, const void* b = nullptr,
                                          const void* c = nullptr, const void* d = nullptr) {
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
             reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
}

// Total PageRank mass sum(x): per-thread partials in compensated FP32, FP64
// across threads and blocks in a fixed order.
__global__ void __launch_bounds__(kNT) pr_mass_partial_kernel(const float* __restrict__ x,
                                                              uint64_t n, double* part_s) {
    __shared__ double ws[kNT / 32 + 1];
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = aligned16(x) ? n / 4 : 0;
    SumAcc ss{0.f, 0.f};
    for (uint64_t i = tid; i < n4; i += stride) {
        const float4 v = reinterpret_cast<const float4*>(x)[i];
        sum_add<true>(ss, v.x);
        sum_add<true>(ss, v.y);
        sum_add<true>(ss, v.z);
        sum_add<true>(ss, v.w);
    }
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) sum_add<true>(ss, x[v]);
    double tot;
    block_excl_scan<kNT>((double)ss.s - (double)ss.c, ws, &tot);
    if (threadIdx.x == 0) part_s[blockIdx.x] = tot;
}

// The fixpoint sums to 1, so a sweep end whose sum is further than 2^-22 from
// it is scaled back onto the unit sum; closer than that (a few FP32 ulps of
// 1) the values are left alone, so converged values can freeze.
__global__ void __launch_bounds__(kNT) pr_mass_final_kernel(RunState* rs, const double* part_s,
                                                            int nparts) {
    __shared__ double ws[kNT / 32 + 1];
    const double m = reduce_partials(part_s, nparts, ws);
    if (threadIdx.x == 0)
        rs->scale = (m > 0.0 && fabs(m - 1.0) > 0x1p-22) ? (float)(1.0 / m) : 1.0f;
}

// One vertex of the sweep close: scaled value (when sc != 1), its L1 change
// against the last sweep end and, for a dangling vertex, its mass.
__device__ __forceinline__ float close_vertex(float xv, float xp, float io, float sc, SumAcc& rr,
                                              SumAcc& dd) {
    if (sc != 1.0f) xv *= sc;
    sum_add<true>(rr, fabsf(xv - xp));
    if (io == 0.0f) sum_add<true>(dd, xv);
    return xv;
}

// PageRank sweep close, one pass over the vertices: the optional mass
// scaling (x and contrib = x / outdeg rewritten when rs->scale != 1), FP64
// partial sums of the dangling mass D = sum of x over out-degree-0 vertices
// and of the L1 change |x - x_prev| against the last sweep end, then the
// snapshot x_prev = x.  |x - x_prev| in FP32 is exact whenever the two are
// within a factor of two (Sterbenz), else correctly rounded; the sums are FP64.
__global__ void __launch_bounds__(kNT) pr_close_partial_kernel(
    float* __restrict__ x, float* __restrict__ contrib, float* __restrict__ x_prev,
    const float* __restrict__ inv_out, uint64_t n, const RunState* rs, double* part_r,
    double* part_d) {
    __shared__ double ws[kNT / 32 + 1];
    const float sc = rs ? rs->scale : 1.0f;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = aligned16(x, contrib, x_prev, inv_out) ? n / 4 : 0;
    // per-thread partials (a few hundred terms) in compensated FP32 -- FP64
    // arithmetic is scarce on this GPU -- then FP64 across threads and blocks
    SumAcc rr{0.f, 0.f}, dd{0.f, 0.f};
    for (uint64_t i = tid; i < n4; i += stride) {
        float4 xv = reinterpret_cast<const float4*>(x)[i];
        const float4 xp = reinterpret_cast<const float4*>(x_prev)[i];
        const float4 io = reinterpret_cast<const float4*>(inv_out)[i];
        xv.x = close_vertex(xv.x, xp.x, io.x, sc, rr, dd);
        xv.y = close_vertex(xv.y, xp.y, io.y, sc, rr, dd);
        xv.z = close_vertex(xv.z, xp.z, io.z, sc, rr, dd);
        xv.w = close_vertex(xv.w, xp.w, io.w, sc, rr, dd);
        if (sc != 1.0f) {
            reinterpret_cast<float4*>(x)[i] = xv;
            reinterpret_cast<float4*>(contrib)[i] =
                make_float4(xv.x * io.x, xv.y * io.y, xv.z * io.z, xv.w * io.w);
        }
        reinterpret_cast<float4*>(x_prev)[i] = xv;
    }
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) {
        const float io = inv_out[v];
        const float xv = close_vertex(x[v], x_prev[v], io, sc, rr, dd);
        if (sc != 1.0f) {
            x[v] = xv;
            contrib[v] = xv * io;
        }
        x_prev[v] = xv;
    }
    const double r = (double)rr.s - (double)rr.c, d = (double)dd.s - (double)dd.c;
    double tot;
    block_excl_scan<kNT>(r, ws, &tot);
    if (threadIdx.x == 0) part_r[blockIdx.x] = tot;
    block_excl_scan<kNT>(d, ws, &tot);
    if (threadIdx.x == 0) part_d[blockIdx.x] = tot;
}

// Residual and dangling mass of the sweep; base term (1-d)/n + d D/n for the
// next sweep (the dangling mass lags one sweep, which leaves the fixpoint
// unchanged).  `out` may be null (initialisation).
__global__ void __launch_bounds__(kNT) pr_close_final_kernel(RunState* rs, const double* part_r,
                                                             const double* part_d, int nparts,
                                                             uint64_t n, double damping,
                                                             SweepReport* out) {
    __shared__ double ws[kNT / 32 + 1];
    const double r = reduce_partials(part_r, nparts, ws);
    const double D = reduce_partials(part_d, nparts, ws);
    if (threadIdx.x == 0) {
        rs->rsum = r;
        rs->dsum = D;
        rs->base = (float)((1.0 - damping) / (double)n + damping * D / (double)n);
        if (out) {
            SweepReport rep = rs->cur;
            rs->prev_changed = rep.changed;
            rep.resid = r;
            rep.dangling = D;
            rep.thr_min = rs->thr_cur;
            *out = rep;
            rs->sweeps_done += 1;
            rs->cur = SweepReport{};
        }
    }
}

__global__ void __launch_bounds__(kNT) dirty_blocks_kernel(const uint32_t* __restrict__ stamp,
                                                           uint64_t n, uint32_t tag, uint32_t bsz,
                                                           uint32_t* __restrict__ dirty) {
    __shared__ uint32_t bits[32];
    if (threadIdx.x < 32) bits[threadIdx.x] = 0;
    __syncthreads();
    // bsz is a multiple of 32, so the 32 vertices of a warp share one block
    for (uint64_t v0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; v0 < n;
         v0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = v0 + lane_id();
        if (__any_sync(kFull, v < n && stamp[v] == tag) && lane_id() == 0) {
            const uint32_t blk = (uint32_t)(v0 / bsz);
            atomicOr(&bits[blk >> 5], 1u << (blk & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x < 32 && bits[threadIdx.x]) atomicOr(&dirty[threadIdx.x], bits[threadIdx.x]);
}

__global__ void clean_pages_kernel(const uint32_t* __restrict__ page_blocks, uint32_t P,
                                   const uint32_t* __restrict__ dirty, RunState* rs) {
    unsigned clean = 0;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        uint32_t hit = 0;
        for (int w = 0; w < 32; ++w) hit |= page_blocks[(uint64_t)p * 32 + w] & dirty[w];
        clean += hit == 0;
    }
    clean = __reduce_add_sync(kFull, clean);
    if (lane_id() == 0 && clean) atomicAdd(&rs->cur.clean_pages, (unsigned long long)clean);
}

unsigned grid_1d(uint64_t n) {
    uint64_t b = (n + kNT - 1) / kNT, cap = (uint64_t)device_sms() * 16;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

void launch_gate(RunState* rs, uint32_t pass, int check_prev, int idle, uint32_t want_loaded,
                 uint32_t j, int learned, unsigned* rec_gains, cudaStream_t s) {
    gate_kernel<<<1, 1, 0, s>>>(rs, pass, check_prev, idle, want_loaded, j, learned, rec_gains);
    SR_LAUNCH();
}

void launch_step_epilogue(RunState* rs, ChunkDyn* cd, uint32_t chunk, uint32_t last_pass,
                          uint32_t npass, unsigned* rec_gains, cudaStream_t s) {
    step_epilogue_kernel<<<1, 1, 0, s>>>(rs, cd, chunk, last_pass, npass, rec_gains);
    SR_LAUNCH();
}

void launch_compact(int algo, const WindowDesc& wd, const AlgoArgs& a, uint32_t pass,
                    int predict, cudaStream_t s) {
    const unsigned g = wd.nblocks ? wd.nblocks : 1;
    switch (algo) {
        case ALG_SSSP: compact_kernel<ALG_SSSP><<<g, kNT, 0, s>>>(wd, a, pass, predict); break;
        case ALG_BFS: compact_kernel<ALG_BFS><<<g, kNT, 0, s>>>(wd, a, pass, predict); break;
        case ALG_CC: compact_kernel<ALG_CC><<<g, kNT, 0, s>>>(wd, a, pass, predict); break;
        default: compact_kernel<ALG_PR><<<g, kNT, 0, s>>>(wd, a, pass, predict); break;
    }
    SR_LAUNCH();
}

template <bool PK>
void launch_relax_form(int algo, int kahan, const AlgoArgs& a, uint32_t pass, uint32_t step,
                       int grid, cudaStream_t s) {
    switch (algo) {
        case ALG_SSSP:
            if (a.wbytes == 1) relax_kernel<ALG_SSSP, false, 1, PK><<<grid, kNT, 0, s>>>(a, pass, step);
            else if (a.wbytes == 2) relax_kernel<ALG_SSSP, false, 2, PK><<<grid, kNT, 0, s>>>(a, pass, step);
            else relax_kernel<ALG_SSSP, false, 4, PK><<<grid, kNT, 0, s>>>(a, pass, step);
            break;
        case ALG_BFS: relax_kernel<ALG_BFS, false, 4, PK><<<grid, kNT, 0, s>>>(a, pass, step); break;
        case ALG_CC: relax_kernel<ALG_CC, false, 4, PK><<<grid, kNT, 0, s>>>(a, pass, step); break;
        default:
            if (kahan) relax_kernel<ALG_PR, true, 4, PK><<<grid, kNT, 0, s>>>(a, pass, step);
            else relax_kernel<ALG_PR, false, 4, PK><<<grid, kNT, 0, s>>>(a, pass, step);
            break;
    }
}

void launch_relax(int algo, int kahan, const AlgoArgs& a, uint32_t pass, uint32_t step, int grid,
                  cudaStream_t s) {
    if (a.packed) launch_relax_form<true>(algo, kahan, a, pass, step, grid, s);
    else launch_relax_form<false>(algo, kahan, a, pass, step, grid, s);
    SR_LAUNCH();
}

void launch_pr_apply(const AlgoArgs& a, uint32_t pass, int grid, cudaStream_t s) {
    pr_apply_kernel<<<grid, kNT, 0, s>>>(a, pass);
    SR_LAUNCH();
}

void launch_set_locs(PageLoc* loc, const uint32_t* vb, uint32_t first, uint32_t end,
                     const uint64_t* rel_soff, const uint64_t* rel_woff, const uint64_t* off_bytes,
                     uint8_t* sbase, uint8_t* wbase, bool packed, RunState* rs, uint32_t seq,
                     cudaStream_t s) {
    unsigned g = end > first ? (end - first + kNT - 1) / kNT : 1;
    set_locs_kernel<<<g, kNT, 0, s>>>(loc, vb, first, end, rel_soff, rel_woff, off_bytes, sbase,
                                       wbase, packed, rs, seq);
    SR_LAUNCH();
}

void launch_init_values(int algo, const AlgoArgs& a, uint64_t n, uint32_t source,
                        const uint32_t* label0, cudaStream_t s) {
    if (algo == ALG_PR) return;  // PageRank init is done by launch_init_pr
    init_min_kernel<<<grid_1d(n), kNT, 0, s>>>(a.val, a.state, n, algo, source, label0);
    SR_LAUNCH();
}

__global__ void unpermute_kernel(const uint32_t* __restrict__ in, const uint32_t* __restrict__ inv,
                                 uint64_t n, uint32_t* __restrict__ out) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        out[v] = in[inv[v]];
}

void launch_unpermute(const uint32_t* in, const uint32_t* inv, uint64_t n, uint32_t* out,
                      cudaStream_t s) {
    unpermute_kernel<<<grid_1d(n), kNT, 0, s>>>(in, inv, n, out);
    SR_LAUNCH();
}

void launch_init_pr(const uint32_t* outdeg, const AlgoArgs& a, float* x_prev, uint64_t n,
                    cudaStream_t s) {
    init_pr_kernel<<<grid_1d(n), kNT, 0, s>>>(outdeg, a.x, a.contrib, x_prev,
                                               const_cast<float*>(a.inv_out), a.state, n);
    SR_LAUNCH();
}

void launch_count_clean(const uint32_t* stamp, uint64_t n, uint32_t tag, uint32_t bsz,
                        const uint32_t* page_blocks, uint32_t P, uint32_t* dirty, RunState* rs,
                        cudaStream_t s) {
    SR_CUDA(cudaMemsetAsync(dirty, 0, 32 * sizeof(uint32_t), s));
    dirty_blocks_kernel<<<grid_1d(n), kNT, 0, s>>>(stamp, n, tag, bsz, dirty);
    clean_pages_kernel<<<(P + kNT - 1) / kNT, kNT, 0, s>>>(page_blocks, P, dirty, rs);
    SR_LAUNCH();
}

void launch_close_min(RunState* rs, SweepReport* out, cudaStream_t s) {
    close_min_kernel<<<1, 1, 0, s>>>(rs, out);
    SR_LAUNCH();
}

void launch_close_pr(const AlgoArgs& a, uint64_t n, float* x_prev, double damping,
                     double* partial, int nparts, SweepReport* out, bool normalize,
                     cudaStream_t s) {
    if (normalize) {
        pr_mass_partial_kernel<<<nparts, kNT, 0, s>>>(a.x, n, partial + 2 * nparts);
        pr_mass_final_kernel<<<1, kNT, 0, s>>>(a.rs, partial + 2 * nparts, nparts);
    }
    pr_close_partial_kernel<<<nparts, kNT, 0, s>>>(a.x, a.contrib, x_prev, a.inv_out, n,
                                                    normalize ? a.rs : nullptr, partial,
                                                    partial + nparts);
    pr_close_final_kernel<<<1, kNT, 0, s>>>(a.rs, partial, partial + nparts, nparts, n, damping,
                                             out);
    SR_LAUNCH();
}

}  // namespace seraph
