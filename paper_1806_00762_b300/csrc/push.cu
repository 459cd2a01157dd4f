// Push rounds of the sparse stage (see push.cuh for the argument that makes
// them exact).  A round: one warp per frontier vertex walks its out-edges
// (read straight from pinned host memory over the host link: consecutive
// lanes read consecutive destinations), relaxes each destination with an
// atomic minimum, and appends every destination it improved -- once per
// round, by swapping the round's tag into the vertex's stamp -- to the next
// frontier (one atomic per warp).  Vertices with more than kPushWarpMax
// out-edges are set aside and walked by the whole grid afterwards.
#include "push.cuh"

namespace seraph {
namespace {

constexpr int kNT = 256;

__device__ __forceinline__ void append_warp(uint32_t* list, unsigned* cnt, bool add, uint32_t v,
                                            unsigned& appended) {
    const unsigned m = __ballot_sync(kFull, add);
    if (!m) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (add) list[base + __popc(m & lanemask_lt())] = v;
    appended += __popc(m);
}

template <int WB>
__device__ __forceinline__ uint32_t load_w(const uint8_t* w, uint64_t k) {
    if (WB == 1) return w[k];
    if (WB == 2) return ((const uint16_t*)w)[k];
    return ((const uint32_t*)w)[k];
}

// Relax out-edge k = (u, v) from u's value du; true if v improved and was not
// yet in the next frontier.
template <int ALGO, int WB>
__device__ __forceinline__ bool push_edge(const PushArgs& a, uint32_t du, uint64_t k, uint32_t tag,
                                          uint32_t& v, unsigned& ovf) {
    v = a.out_col[k];
    uint32_t cand = du;
    if (ALGO != ALG_CC) {
        if (du == SERAPH_INF) return false;
        cand = du + (ALGO == ALG_SSSP ? load_w<WB>(a.out_w, k) : 1u);
        if (cand < du || cand == SERAPH_INF) { ovf = 1; return false; }
    }
    // values only decrease, so a stale read can only skip a useless atomic
    if (cand >= a.val[v]) return false;
    if (cand >= atomicMin(&a.val[v], cand)) return false;
    return atomicExch(&a.stamp[v], tag) != tag;
}

// Called by whole warps: `edges` and `appended` are the same in every lane of
// a warp (counted per warp), `ovf` is per lane.
__device__ __forceinline__ void flush(PushState* ps, unsigned long long edges, unsigned appended,
                                      unsigned ovf) {
    ovf = __reduce_or_sync(kFull, ovf);
    if (lane_id() == 0) {
        if (edges) atomicAdd(&ps->edges, edges);
        if (appended) atomicAdd(&ps->changes, (unsigned long long)appended);
        if (ovf) atomicOr(&ps->ovf, 1u);
    }
}

__global__ void push_begin_kernel(PushState* ps, uint32_t r) {
    const int cur = r & 1;
    ps->cnt[cur ^ 1] = 0;
    ps->nbig = 0;
    if (ps->cnt[cur]) ps->rounds += 1;
}

__global__ void __launch_bounds__(kNT) push_frontier_kernel(const uint32_t* __restrict__ stamp,
                                                            uint32_t n, uint32_t tag,
                                                            uint32_t* __restrict__ front,
                                                            unsigned* cnt) {
    const uint32_t lane = lane_id();
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned appended = 0;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const uint64_t v = base + lane;
        append_warp(front, cnt, v < n && stamp[v] >= tag, (uint32_t)v, appended);
    }
}

template <int ALGO, int WB>
__global__ void __launch_bounds__(kNT) push_small_kernel(PushArgs a, uint32_t r, uint32_t tag) {
    const int cur = r & 1;
    PushState* ps = a.ps;
    const unsigned count = cur ? ps->cnt[1] : ps->cnt[0];
    if (count == 0) return;
    const uint32_t* F = cur ? a.front[1] : a.front[0];  // (no dynamic index into the parameters)
    uint32_t* Fn = cur ? a.front[0] : a.front[1];
    unsigned* cnt_n = cur ? &ps->cnt[0] : &ps->cnt[1];
    const unsigned lane = lane_id();
    const unsigned w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long edges = 0;
    unsigned appended = 0, ovf = 0;
    for (unsigned i = w0; i < count; i += nw) {
        const uint32_t u = F[i];
        uint64_t b = 0, e = 0;
        if (lane == 0) { b = a.out_off[u]; e = a.out_off[u + 1]; }
        b = __shfl_sync(kFull, b, 0);
        e = __shfl_sync(kFull, e, 0);
        if (e - b > kPushWarpMax) {  // walked by the whole grid afterwards
            if (lane == 0) {
                const unsigned k = atomicAdd(&ps->nbig, 1u);
                if (k < a.big_cap) a.big[k] = u;
            }
            continue;
        }
        const uint32_t du = a.val[u];
        for (uint64_t base = b; base < e; base += 32) {
            const uint64_t k = base + lane;
            uint32_t v = 0;
            const bool add = k < e && push_edge<ALGO, WB>(a, du, k, tag, v, ovf);
            append_warp(Fn, cnt_n, add, v, appended);
        }
        edges += e - b;
    }
    flush(ps, edges, appended, ovf);
}

template <int ALGO, int WB>
__global__ void __launch_bounds__(kNT) push_big_kernel(PushArgs a, uint32_t r, uint32_t tag) {
    const int nxt = (r & 1) ^ 1;
    PushState* ps = a.ps;
    const unsigned nbig = min(ps->nbig, a.big_cap);
    if (nbig == 0) return;
    uint32_t* Fn = nxt ? a.front[1] : a.front[0];
    unsigned* cnt_n = nxt ? &ps->cnt[1] : &ps->cnt[0];
    const unsigned lane = lane_id();
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long edges = 0;
    unsigned appended = 0, ovf = 0;
    for (unsigned i = 0; i < nbig; ++i) {
        const uint32_t u = a.big[i];
        const uint64_t b = a.out_off[u], e = a.out_off[u + 1];
        const uint32_t du = a.val[u];
        for (uint64_t base = b + w0 * 32; base < e; base += nw * 32) {
            const uint64_t k = base + lane;
            uint32_t v = 0;
            const bool add = k < e && push_edge<ALGO, WB>(a, du, k, tag, v, ovf);
            append_warp(Fn, cnt_n, add, v, appended);
        }
        if (w0 == 0) edges += e - b;
    }
    flush(ps, edges, appended, ovf);
}

template <int ALGO, int WB>
void round_for(const PushArgs& a, uint32_t r, uint32_t tag, unsigned grid, cudaStream_t s) {
    push_small_kernel<ALGO, WB><<<grid, kNT, 0, s>>>(a, r, tag);
    push_big_kernel<ALGO, WB><<<grid, kNT, 0, s>>>(a, r, tag);
}

template <int ALGO>
void round_w(const PushArgs& a, uint32_t r, uint32_t tag, unsigned grid, cudaStream_t s) {
    if (ALGO != ALG_SSSP || a.wbytes == 1) round_for<ALGO, 1>(a, r, tag, grid, s);
    else if (a.wbytes == 2) round_for<ALGO, 2>(a, r, tag, grid, s);
    else round_for<ALGO, 4>(a, r, tag, grid, s);
}

}  // namespace

void launch_push_frontier(const PushArgs& a, uint32_t tag, cudaStream_t s) {
    SR_CUDA(cudaMemsetAsync(a.ps, 0, sizeof(PushState), s));
    push_frontier_kernel<<<(unsigned)device_sms() * 8, kNT, 0, s>>>(a.stamp, a.n, tag, a.front[0],
                                                                     &a.ps->cnt[0]);
    SR_LAUNCH();
}

void launch_push_round(int algo, const PushArgs& a, uint32_t r, uint32_t tag, cudaStream_t s) {
    push_begin_kernel<<<1, 1, 0, s>>>(a.ps, r);
    const unsigned grid = (unsigned)device_sms() * 8;
    if (algo == ALG_SSSP) round_w<ALG_SSSP>(a, r, tag, grid, s);
    else if (algo == ALG_BFS) round_w<ALG_BFS>(a, r, tag, grid, s);
    else round_w<ALG_CC>(a, r, tag, grid, s);
    SR_LAUNCH();
}

}  // namespace seraph
