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
#include "engine.cuh"

namespace seraph {
namespace {

constexpr int kNT = 256;
constexpr int kCompactRounds = 4;
constexpr uint32_t kCompactTile = kNT * kCompactRounds;

__device__ __forceinline__ uint4 ld_stream4(const uint32_t* p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) {
    uint32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
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

__device__ __forceinline__ uint8_t fsm_step(const AlgoArgs& a, uint8_t st, bool ch) {
    // A dormant state reached here only because prediction is off for the
    // pass: a valid update follows its "changed" edge, otherwise it keeps its
    // state (its ticks belong to predicted passes).
    if ((a.skip_mask >> st) & 1) return ch ? a.fsm_next[2 * st + 1] : st;
    return a.fsm_next[2 * st + (ch ? 1 : 0)];
}

template <int ALGO>
__device__ __forceinline__ void finish_min(const AlgoArgs& a, uint32_t v, const MinAcc& acc,
                                           uint32_t deg, Locals& L) {
    uint32_t old = a.val[v];
    bool ch = acc.best < old;
    if (ch) a.val[v] = acc.best;
    if (ALGO == ALG_SSSP && acc.ovf && acc.best == SERAPH_INF && old == SERAPH_INF) L.ovf = 1;
    if (a.pvu == SERAPH_PVU_WEAK) a.state[v] = fsm_step(a, a.state[v], ch);
    L.changed += ch;
    L.edges += deg;
    if (ch) L.minv = min(L.minv, acc.best);
}

__device__ __forceinline__ void finish_pr(const AlgoArgs& a, uint32_t v, float sum, float base,
                                          uint32_t deg, Locals& L) {
    float xo = a.x[v];
    float xn = base + a.damping * sum;
    a.x_next[v] = xn;
    bool ch = fabsf(xn - xo) > a.fail_eps * xo;
    if (a.pvu == SERAPH_PVU_WEAK) a.state[v] = fsm_step(a, a.state[v], ch);
    L.changed += ch;
    L.edges += deg;
}

// ------------------------------------------------------------- one vertex

template <int ALGO, bool KAHAN>
__device__ __forceinline__ void vertex_thread(const AlgoArgs& a, unsigned long long ent, float base,
                                              Locals& L) {
    const uint32_t v = (uint32_t)ent, p = (uint32_t)(ent >> 32);
    const PageLoc loc = a.loc[p];
    const uint32_t li = v - loc.vb;
    const uint32_t b = loc.off[li], e = loc.off[li + 1];
    if (ALGO == ALG_PR) {
        SumAcc acc{0.f, 0.f};
        for (uint32_t i = b; i < e; ++i) sum_add<KAHAN>(acc, a.contrib[ld_stream(loc.col + i)]);
        finish_pr(a, v, acc.s - acc.c, base, e - b, L);
    } else {
        MinAcc acc{SERAPH_INF, false};
        for (uint32_t i = b; i < e; ++i)
            min_edge<ALGO>(acc, ld_stream(loc.col + i), ALGO == ALG_SSSP ? ld_stream(loc.w + i) : 1u,
                           a.val);
        finish_min<ALGO>(a, v, acc, e - b, L);
    }
}

// Group of G lanes (G = 32: a warp; the CTA variant reduces across warps).
// Lane t of the group reads the aligned 16-byte vectors t, t+G, ... of the
// vertex's column range [b, e), masking elements outside it.
template <int ALGO, bool KAHAN>
__device__ __forceinline__ void edges_strided(const AlgoArgs& a, const PageLoc& loc, uint32_t b,
                                              uint32_t e, uint32_t t, uint32_t G, MinAcc& macc,
                                              SumAcc& sacc) {
    for (uint32_t idx = (b & ~3u) + 4 * t; idx < e; idx += 4 * G) {
        const uint4 c4 = ld_stream4(loc.col + idx);
        uint4 w4 = make_uint4(1, 1, 1, 1);
        if (ALGO == ALG_SSSP) w4 = ld_stream4(loc.w + idx);
        const uint32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
        const uint32_t ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = idx + j;
            if (i >= b && i < e) {
                if (ALGO == ALG_PR) sum_add<KAHAN>(sacc, a.contrib[cc[j]]);
                else min_edge<ALGO>(macc, cc[j], ww[j], a.val);
            }
        }
    }
}

template <int ALGO, bool KAHAN>
__device__ __forceinline__ void vertex_warp(const AlgoArgs& a, unsigned long long ent, float base,
                                            Locals& L) {
    const uint32_t v = (uint32_t)ent, p = (uint32_t)(ent >> 32);
    const PageLoc loc = a.loc[p];
    const uint32_t li = v - loc.vb;
    const uint32_t b = loc.off[li], e = loc.off[li + 1];
    const uint32_t lane = lane_id();
    MinAcc macc{SERAPH_INF, false};
    SumAcc sacc{0.f, 0.f};
    edges_strided<ALGO, KAHAN>(a, loc, b, e, lane, 32, macc, sacc);
    if (ALGO == ALG_PR) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            SumAcc other{__shfl_xor_sync(kFull, sacc.s, o), __shfl_xor_sync(kFull, sacc.c, o)};
            sacc = (lane & o) ? sum_merge<KAHAN>(other, sacc) : sum_merge<KAHAN>(sacc, other);
        }
        if (lane == 0) finish_pr(a, v, sacc.s - sacc.c, base, e - b, L);
    } else {
        macc.best = __reduce_min_sync(kFull, macc.best);
        macc.ovf = __any_sync(kFull, macc.ovf);
        if (lane == 0) finish_min<ALGO>(a, v, macc, e - b, L);
    }
}

template <int ALGO, bool KAHAN>
__device__ __forceinline__ void vertex_cta(const AlgoArgs& a, unsigned long long ent, float base,
                                           Locals& L, float* s_sum, float* s_comp,
                                           unsigned* s_min, unsigned* s_ovf) {
    const uint32_t v = (uint32_t)ent, p = (uint32_t)(ent >> 32);
    const PageLoc loc = a.loc[p];
    const uint32_t li = v - loc.vb;
    const uint32_t b = loc.off[li], e = loc.off[li + 1];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    MinAcc macc{SERAPH_INF, false};
    SumAcc sacc{0.f, 0.f};
    edges_strided<ALGO, KAHAN>(a, loc, b, e, threadIdx.x, kNT, macc, sacc);
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
            finish_pr(a, v, t.s - t.c, base, e - b, L);
        }
    } else {
        macc.best = __reduce_min_sync(kFull, macc.best);
        macc.ovf = __any_sync(kFull, macc.ovf);
        if (lane == 0) { s_min[warp] = macc.best; s_ovf[warp] = macc.ovf; }
        __syncthreads();
        if (threadIdx.x == 0) {
            MinAcc t{s_min[0], s_ovf[0] != 0};
            for (int w = 1; w < kNT / 32; ++w) { t.best = min(t.best, s_min[w]); t.ovf |= s_ovf[w] != 0; }
            finish_min<ALGO>(a, v, t, e - b, L);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void flush_locals(const AlgoArgs& a, int par, Locals L) {
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
        }
        if (mn != SERAPH_INF) atomicMin(&rs->thr_cur, mn);
        if (ov) atomicOr(&rs->cur.overflow, 1u);
        if (ed) atomicAdd(&rs->cur.edges, ed);
    }
}

// ---------------------------------------------------------------- kernels

template <int ALGO>
__global__ void __launch_bounds__(kNT) compact_kernel(WindowDesc wd, AlgoArgs a, uint32_t pass,
                                                      int check_prev, int predict) {
    __shared__ unsigned ws[kNT / 32 + 1];
    __shared__ unsigned s_base[3];
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (blockIdx.x == 0) {
        if (threadIdx.x < 4) rs->work[par][threadIdx.x] = 0;
        if (threadIdx.x == 4) rs->pass_changed[par] = 0;
    }
    const bool skip_pass = check_prev && rs->pass_changed[par ^ 1] == 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (skip_pass) atomicAdd(&rs->cur.passes_skipped, 1u);
        else atomicAdd(&rs->cur.passes_run, 1u);
    }
    if (skip_pass) return;

    int c = 0;
    while (c + 1 < (int)wd.nchunks && blockIdx.x >= wd.c[c + 1].block_begin) ++c;
    const ChunkDesc cd = wd.c[c];
    const bool strong = predict && a.pvu == SERAPH_PVU_STRONG;
    const bool weak = predict && a.pvu == SERAPH_PVU_WEAK;
    uint32_t thr = 0;
    if (strong) thr = ALGO == ALG_BFS ? rs->sweeps_done : min(rs->thr_prev, rs->thr_cur);

    unsigned long long my_ent[kCompactRounds];
    int my_cls[kCompactRounds];
    unsigned n_att = 0, n_skip = 0;
    const uint32_t v0 = cd.v_begin + (blockIdx.x - cd.block_begin) * kCompactTile;
#pragma unroll
    for (int r = 0; r < kCompactRounds; ++r) {
        my_cls[r] = -1;
        my_ent[r] = 0;
        const uint32_t v = v0 + r * kNT + threadIdx.x;
        if (v >= v0 && v < cd.v_end) {
            const uint32_t p = find_page(a.vb, cd.first_page, cd.end_page, v);
            const PageLoc loc = a.loc[p];
            const uint32_t li = v - loc.vb;
            const uint32_t deg = loc.off[li + 1] - loc.off[li];
            if (deg > 0) {
                bool skip = false;
                if (strong) {
                    skip = a.val[v] <= thr;
                } else if (weak) {
                    const uint8_t st = a.state[v];
                    if ((a.skip_mask >> st) & 1) {
                        skip = true;
                        a.state[v] = a.fsm_next[2 * st];  // dormant tick
                    }
                }
                if (skip) {
                    ++n_skip;
                } else {
                    ++n_att;
                    my_cls[r] = deg <= a.thread_max ? 0 : (deg <= a.warp_max ? 1 : 2);
                    my_ent[r] = ((unsigned long long)p << 32) | v;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned mine = 0;
#pragma unroll
        for (int r = 0; r < kCompactRounds; ++r) mine += my_cls[r] == k;
        unsigned tot, ex = block_excl_scan<kNT>(mine, ws, &tot);
        if (tot == 0) continue;  // uniform: every thread sees the same total
        if (threadIdx.x == 0) s_base[k] = atomicAdd(&rs->list_cnt[par][k], tot);
        __syncthreads();
        unsigned pos = s_base[k] + ex;
#pragma unroll
        for (int r = 0; r < kCompactRounds; ++r)
            if (my_cls[r] == k) a.list[k][pos++] = my_ent[r];
    }
    unsigned tot_att, tot_skip;
    block_excl_scan<kNT>(n_att, ws, &tot_att);
    block_excl_scan<kNT>(n_skip, ws, &tot_skip);
    if (threadIdx.x == 0) {
        if (tot_att) atomicAdd(&rs->cur.attempted, (unsigned long long)tot_att);
        if (tot_skip) atomicAdd(&rs->cur.skipped, (unsigned long long)tot_skip);
    }
}

template <int ALGO, bool KAHAN>
__global__ void __launch_bounds__(kNT) relax_kernel(AlgoArgs a, uint32_t pass, int check_prev) {
    __shared__ unsigned s_item;
    __shared__ float s_sum[kNT / 32], s_comp[kNT / 32];
    __shared__ unsigned s_min[kNT / 32], s_ovf[kNT / 32];
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (blockIdx.x == 0 && threadIdx.x < 4) rs->list_cnt[par ^ 1][threadIdx.x] = 0;
    if (check_prev && rs->pass_changed[par ^ 1] == 0) return;
    const unsigned n0 = rs->list_cnt[par][0], n1 = rs->list_cnt[par][1], n2 = rs->list_cnt[par][2];
    const float base = ALGO == ALG_PR ? rs->base : 0.f;
    Locals L{0u, SERAPH_INF, 0u, 0ull};

    for (;;) {  // one CTA per hub vertex
        if (threadIdx.x == 0) s_item = atomicAdd(&rs->work[par][2], 1u);
        __syncthreads();
        const unsigned i = s_item;
        __syncthreads();
        if (i >= n2) break;
        vertex_cta<ALGO, KAHAN>(a, a.list[2][i], base, L, s_sum, s_comp, s_min, s_ovf);
    }
    const unsigned lane = lane_id();
    for (;;) {  // one warp per medium vertex, four at a time
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(&rs->work[par][1], 4u);
        i0 = __shfl_sync(kFull, i0, 0);
        if (i0 >= n1) break;
        for (unsigned j = 0; j < 4 && i0 + j < n1; ++j)
            vertex_warp<ALGO, KAHAN>(a, a.list[1][i0 + j], base, L);
    }
    for (;;) {  // one thread per small vertex, 128 per warp grab
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(&rs->work[par][0], 128u);
        i0 = __shfl_sync(kFull, i0, 0);
        if (i0 >= n0) break;
#pragma unroll
        for (unsigned j = 0; j < 4; ++j) {
            const unsigned i = i0 + j * 32 + lane;
            if (i < n0) vertex_thread<ALGO, KAHAN>(a, a.list[0][i], base, L);
        }
    }
    flush_locals(a, par, L);
}

__global__ void __launch_bounds__(kNT) pr_apply_kernel(AlgoArgs a, uint32_t pass, int check_prev) {
    const int par = pass & 1;
    RunState* rs = a.rs;
    if (check_prev && rs->pass_changed[par ^ 1] == 0) return;
    const unsigned n[3] = {rs->list_cnt[par][0], rs->list_cnt[par][1], rs->list_cnt[par][2]};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < 3; ++k) {
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n[k]; i += stride) {
            const uint32_t v = (uint32_t)a.list[k][i];
            const float xn = a.x_next[v];
            a.x[v] = xn;
            a.contrib[v] = xn * a.inv_out[v];
        }
    }
}

__global__ void set_locs_kernel(PageLoc* loc, const uint32_t* vb, uint32_t first, uint32_t end,
                                const uint64_t* rel_soff, const uint64_t* rel_woff,
                                const uint64_t* off_bytes, uint8_t* sbase, uint8_t* wbase) {
    for (uint32_t p = first + blockIdx.x * blockDim.x + threadIdx.x; p < end;
         p += gridDim.x * blockDim.x) {
        PageLoc L;
        const uint8_t* s = sbase + rel_soff[p];
        L.off = (const uint32_t*)s;
        L.col = (const uint32_t*)(s + off_bytes[p]);
        L.w = wbase ? (const uint32_t*)(wbase + rel_woff[p]) : nullptr;
        L.vb = vb[p];
        L.nv = vb[p + 1] - vb[p];
        loc[p] = L;
    }
}

__global__ void init_min_kernel(uint32_t* val, uint8_t* state, uint64_t n, int algo,
                                uint32_t source) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        val[v] = algo == ALG_CC ? (uint32_t)v : (v == source ? 0u : SERAPH_INF);
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

__global__ void close_min_kernel(RunState* rs, SweepReport* out) {
    SweepReport r = rs->cur;
    r.thr_min = rs->thr_cur;
    *out = r;
    rs->thr_prev = rs->thr_cur;
    rs->thr_cur = SERAPH_INF;
    rs->sweeps_done += 1;
    rs->cur = SweepReport{};
}

// PageRank sweep close, step 1: per-block FP64 sums of dangling mass.
__global__ void __launch_bounds__(kNT) pr_dangling_kernel(const float* x, const float* inv_out,
                                                          uint64_t n, double* partial) {
    __shared__ double ws[kNT / 32 + 1];
    double s = 0.0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (inv_out[v] == 0.0f) s += (double)x[v];
    double tot;
    block_excl_scan<kNT>(s, ws, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Fixed-order FP64 reduction of `nparts` partials by one block.
__device__ double reduce_partials(const double* partial, int nparts, double* ws) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kNT) s += partial[i];
    double tot;
    block_excl_scan<kNT>(s, ws, &tot);
    return tot;
}

__global__ void __launch_bounds__(kNT) pr_base_kernel(RunState* rs, const double* partial,
                                                      int nparts, uint64_t n, double d) {
    __shared__ double ws[kNT / 32 + 1];
    double D = reduce_partials(partial, nparts, ws);
    if (threadIdx.x == 0) {
        rs->dsum = D;
        rs->base = (float)((1.0 - d) / (double)n + d * D / (double)n);
    }
}

// Step 2: zero-in-degree vertices take the new base value (their whole
// PageRank equation), then the FP64 L1 change against the last sweep end.
__global__ void __launch_bounds__(kNT) pr_resid_kernel(RunState* rs, float* x, float* contrib,
                                                       const float* inv_out, float* x_prev,
                                                       const uint32_t* zero_in, uint64_t n,
                                                       double* partial) {
    __shared__ double ws[kNT / 32 + 1];
    const float base = rs->base;
    double s = 0.0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        float xv = x[v];
        if ((zero_in[v >> 5] >> (v & 31)) & 1u) {
            xv = base;
            x[v] = xv;
            contrib[v] = xv * inv_out[v];
        }
        s += fabs((double)xv - (double)x_prev[v]);
        x_prev[v] = xv;
    }
    double tot;
    block_excl_scan<kNT>(s, ws, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kNT) pr_close_kernel(RunState* rs, const double* partial,
                                                       int nparts, SweepReport* out) {
    __shared__ double ws[kNT / 32 + 1];
    double r = reduce_partials(partial, nparts, ws);
    if (threadIdx.x == 0) {
        rs->rsum = r;
        SweepReport rep = rs->cur;
        rep.resid = r;
        rep.dangling = rs->dsum;
        rep.thr_min = rs->thr_cur;
        *out = rep;
        rs->sweeps_done += 1;
        rs->cur = SweepReport{};
    }
}

unsigned grid_1d(uint64_t n) {
    uint64_t b = (n + kNT - 1) / kNT, cap = (uint64_t)device_sms() * 16;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

void launch_compact(int algo, const WindowDesc& wd, const AlgoArgs& a, uint32_t pass,
                    int check_prev, int predict, cudaStream_t s) {
    const unsigned g = wd.nblocks ? wd.nblocks : 1;
    switch (algo) {
        case ALG_SSSP: compact_kernel<ALG_SSSP><<<g, kNT, 0, s>>>(wd, a, pass, check_prev, predict); break;
        case ALG_BFS: compact_kernel<ALG_BFS><<<g, kNT, 0, s>>>(wd, a, pass, check_prev, predict); break;
        case ALG_CC: compact_kernel<ALG_CC><<<g, kNT, 0, s>>>(wd, a, pass, check_prev, predict); break;
        default: compact_kernel<ALG_PR><<<g, kNT, 0, s>>>(wd, a, pass, check_prev, predict); break;
    }
    SR_LAUNCH();
}

void launch_relax(int algo, int kahan, const AlgoArgs& a, uint32_t pass, int check_prev, int grid,
                  cudaStream_t s) {
    switch (algo) {
        case ALG_SSSP: relax_kernel<ALG_SSSP, false><<<grid, kNT, 0, s>>>(a, pass, check_prev); break;
        case ALG_BFS: relax_kernel<ALG_BFS, false><<<grid, kNT, 0, s>>>(a, pass, check_prev); break;
        case ALG_CC: relax_kernel<ALG_CC, false><<<grid, kNT, 0, s>>>(a, pass, check_prev); break;
        default:
            if (kahan) relax_kernel<ALG_PR, true><<<grid, kNT, 0, s>>>(a, pass, check_prev);
            else relax_kernel<ALG_PR, false><<<grid, kNT, 0, s>>>(a, pass, check_prev);
            break;
    }
    SR_LAUNCH();
}

void launch_pr_apply(const AlgoArgs& a, uint32_t pass, int check_prev, int grid, cudaStream_t s) {
    pr_apply_kernel<<<grid, kNT, 0, s>>>(a, pass, check_prev);
    SR_LAUNCH();
}

void launch_set_locs(PageLoc* loc, const uint32_t* vb, uint32_t first, uint32_t end,
                     const uint64_t* rel_soff, const uint64_t* rel_woff, const uint64_t* off_bytes,
                     uint8_t* sbase, uint8_t* wbase, cudaStream_t s) {
    if (end <= first) return;
    unsigned g = (end - first + kNT - 1) / kNT;
    set_locs_kernel<<<g, kNT, 0, s>>>(loc, vb, first, end, rel_soff, rel_woff, off_bytes, sbase, wbase);
    SR_LAUNCH();
}

void launch_init_values(int algo, const AlgoArgs& a, uint64_t n, uint32_t source, cudaStream_t s) {
    if (algo == ALG_PR) return;  // PageRank init is done by launch_init_pr
    init_min_kernel<<<grid_1d(n), kNT, 0, s>>>(a.val, a.state, n, algo, source);
    SR_LAUNCH();
}

void launch_init_pr(const uint32_t* outdeg, const AlgoArgs& a, float* x_prev, uint64_t n,
                    cudaStream_t s) {
    init_pr_kernel<<<grid_1d(n), kNT, 0, s>>>(outdeg, a.x, a.contrib, x_prev,
                                               const_cast<float*>(a.inv_out), a.state, n);
    SR_LAUNCH();
}

void launch_close_min(RunState* rs, SweepReport* out, cudaStream_t s) {
    close_min_kernel<<<1, 1, 0, s>>>(rs, out);
    SR_LAUNCH();
}

void launch_close_pr(const AlgoArgs& a, uint64_t n, float* x_prev, const uint32_t* zero_in,
                     double damping, double* partial, int nparts, SweepReport* out,
                     cudaStream_t s) {
    pr_dangling_kernel<<<nparts, kNT, 0, s>>>(a.x, a.inv_out, n, partial);
    pr_base_kernel<<<1, kNT, 0, s>>>(a.rs, partial, nparts, n, damping);
    pr_resid_kernel<<<nparts, kNT, 0, s>>>(a.rs, a.x, a.contrib, a.inv_out, x_prev, zero_in, n,
                                            partial);
    if (out) pr_close_kernel<<<1, kNT, 0, s>>>(a.rs, partial, nparts, out);
    SR_LAUNCH();
}

}  // namespace seraph
