// seraph_pull_fixpoint_noalloc: the pull relaxation (min over in-edges, one
// warp per vertex) run to its fixpoint over a CSC that already sits in
// device memory, without allocating anything.
//
// Who needs it: callers whose device memory is owned by someone else -- a
// framework's memory planner or a latency-critical serving loop that may not
// call cudaMalloc/cudaFree (they synchronise the device and can fail under
// memory pressure).  Such callers pass their own input and output buffers;
// the only scratch this entry point uses is the file-scope device array
// below (counters plus the list of vertices that have in-edges), so graphs
// are limited to SERAPH_NOALLOC_MAX_VERTICES vertices.
//
// The array lives in every GPU that loads the library until the process
// exits.  All calls share it and it keeps the last call's contents, so the
// counters and the list length are cleared at the start of every call, and
// two calls that overlap on the GPU (different streams or threads) race.
// The first call on each device resolves the array's device address with
// cudaGetSymbolAddress.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace seraph {
void set_last_error(const char* msg);
}

namespace {

using seraph::kFull;

constexpr uint32_t kCounters = 64;  // [0] changes in the pass, [1] list length, [2] overflow,
                                    // [3] input check: 1 bad offsets, 2 a source id >= n
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint32_t g_noalloc_scratch[kCounters + SERAPH_NOALLOC_MAX_VERTICES];

std::mutex g_mu;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once
// per device; the host-side symbol is not a device address).
uint32_t* scratch_on_current_device() {
    int dev = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CHECK(dev >= 0 && dev < kMaxDevices, SERAPH_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        SR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = (uint32_t*)p;
    }
    return g_scratch_addr[dev];
}

// Input check before anything is read through the CSC: offsets that do not
// start at 0 or that decrease, and source ids >= n (which would index
// outside `values`), are flagged in scratch[3].
__global__ void na_check(const uint64_t* __restrict__ col_off, const uint32_t* __restrict__ row,
                         uint32_t n, uint32_t* scratch) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned bad = 0;
    for (uint64_t v = tid; v < n; v += stride)
        if ((v == 0 && col_off[0] != 0) || col_off[v] > col_off[v + 1]) bad |= 1u;
    const uint64_t m = col_off[n];
    for (uint64_t k = tid; k < m; k += stride)
        if (row[k] >= n) bad |= 2u;
    bad = __reduce_or_sync(kFull, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicOr(&scratch[3], bad);
}

__global__ void na_init(int algo, uint32_t n, uint32_t source, uint32_t* values) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        values[v] = algo == SERAPH_CC ? v : (v == source ? 0u : SERAPH_INF);
}

__global__ void na_list(const uint64_t* __restrict__ col_off, uint32_t n, uint32_t* scratch) {
    uint32_t* list = scratch + kCounters;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t v = base + threadIdx.x;
        const bool has_in = v < n && col_off[v + 1] > col_off[v];
        const unsigned m = __ballot_sync(kFull, has_in);
        unsigned pos = 0;
        if ((threadIdx.x & 31) == 0 && m) pos = atomicAdd(&scratch[1], __popc(m));
        pos = __shfl_sync(kFull, pos, 0);
        if (has_in) list[pos + __popc(m & seraph::lanemask_lt())] = v;
    }
}

template <int ALGO>
__global__ void na_pass(const uint64_t* __restrict__ col_off, const uint32_t* __restrict__ row,
                        const uint32_t* __restrict__ w, uint32_t* values, uint32_t* scratch) {
    const uint32_t* list = scratch + kCounters;
    const uint32_t count = scratch[1];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    unsigned changed = 0, ovf = 0;
    for (uint32_t i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < count; i += warps) {
        const uint32_t v = list[i];
        const uint64_t b = col_off[v], e = col_off[v + 1];
        uint32_t best = SERAPH_INF;
        bool o = false;
        for (uint64_t k = b + lane; k < e; k += 32) {
            const uint32_t du = values[row[k]];
            if (ALGO == SERAPH_CC) {
                best = min(best, du);
            } else if (du != SERAPH_INF) {
                const uint32_t s = du + (ALGO == SERAPH_SSSP && w ? w[k] : 1u);
                if (s < du || s == SERAPH_INF) o = true; else best = min(best, s);
            }
        }
        best = __reduce_min_sync(kFull, best);
        o = __any_sync(kFull, o);
        if (lane == 0) {
            const uint32_t old = values[v];
            if (best < old) { values[v] = best; ++changed; }
            if (o && best == SERAPH_INF && old == SERAPH_INF) ovf = 1;
        }
    }
    changed = __reduce_add_sync(kFull, changed);
    ovf = __reduce_or_sync(kFull, ovf);
    if (lane == 0) {
        if (changed) atomicAdd(&scratch[0], changed);
        if (ovf) atomicOr(&scratch[2], 1u);
    }
}

int run_noalloc(int algo, uint64_t n, const uint64_t* col_off, const uint32_t* row,
                const uint32_t* w, uint32_t source, uint32_t* values, uint32_t* passes_out,
                cudaStream_t s) {
    SR_CHECK(algo == SERAPH_SSSP || algo == SERAPH_BFS || algo == SERAPH_CC, SERAPH_EINVAL,
             "algo must be SERAPH_SSSP, SERAPH_BFS or SERAPH_CC");
    SR_CHECK(n >= 1, SERAPH_EINVAL, "n must be >= 1");
    SR_CHECK(n <= SERAPH_NOALLOC_MAX_VERTICES, SERAPH_EINVAL,
             "n exceeds SERAPH_NOALLOC_MAX_VERTICES (2^20) of the static scratch");
    SR_CHECK(col_off && values, SERAPH_EINVAL, "col_off and values must not be NULL");
    SR_CHECK(row != nullptr, SERAPH_EINVAL, "row must not be NULL");
    if (algo != SERAPH_CC) SR_CHECK(source < n, SERAPH_EINVAL, "source >= n");
    uint32_t* scratch = scratch_on_current_device();
    const uint32_t nn = (uint32_t)n;
    const int sms = seraph::device_sms();
    const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
    SR_CUDA(cudaMemsetAsync(scratch, 0, kCounters * sizeof(uint32_t), s));
    na_check<<<(unsigned)sms * 8, 256, 0, s>>>(col_off, row, nn, scratch);
    SR_LAUNCH();
    uint32_t check = 0;
    SR_CUDA(cudaMemcpyAsync(&check, scratch + 3, sizeof(check), cudaMemcpyDeviceToHost, s));
    SR_CUDA(cudaStreamSynchronize(s));
    SR_CHECK(!(check & 1u), SERAPH_EINVAL, "col_off must start at 0 and be non-decreasing");
    SR_CHECK(!(check & 2u), SERAPH_EINVAL, "a source id in row is >= n");
    na_init<<<grid, 256, 0, s>>>(algo, nn, source, values);
    na_list<<<grid, 256, 0, s>>>(col_off, nn, scratch);
    SR_LAUNCH();
    const unsigned pass_grid = (unsigned)sms * 8;
    for (uint64_t pass = 1; pass <= n + 1; ++pass) {
        SR_CUDA(cudaMemsetAsync(scratch, 0, sizeof(uint32_t), s));
        SR_CUDA(cudaMemsetAsync(scratch + 2, 0, sizeof(uint32_t), s));
        if (algo == SERAPH_SSSP)
            na_pass<SERAPH_SSSP><<<pass_grid, 256, 0, s>>>(col_off, row, w, values, scratch);
        else if (algo == SERAPH_BFS)
            na_pass<SERAPH_BFS><<<pass_grid, 256, 0, s>>>(col_off, row, w, values, scratch);
        else
            na_pass<SERAPH_CC><<<pass_grid, 256, 0, s>>>(col_off, row, w, values, scratch);
        SR_LAUNCH();
        uint32_t host_counters[3] = {0, 0, 0};
        SR_CUDA(cudaMemcpyAsync(host_counters, scratch, sizeof(host_counters),
                                cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        if (host_counters[0] == 0) {
            if (passes_out) *passes_out = (uint32_t)pass;
            SR_CHECK(host_counters[2] == 0, SERAPH_EOVERFLOW,
                     "an SSSP distance does not fit below 2^32-1");
            return SERAPH_OK;
        }
    }
    throw seraph::Error(SERAPH_ENOTCONV, "no fixpoint after n+1 passes");
}

}  // namespace

extern "C" int seraph_pull_fixpoint_noalloc(int algo, uint64_t n, const uint64_t* col_off,
                                            const uint32_t* row, const uint32_t* w,
                                            uint32_t source, uint32_t* values,
                                            uint32_t* passes_out, void* stream) {
    try {
        seraph::set_last_error("");
        return run_noalloc(algo, n, col_off, row, w, source, values, passes_out,
                           (cudaStream_t)stream);
    } catch (const seraph::Error& e) {
        seraph::set_last_error(e.what());
        return e.code;
    } catch (...) {
        seraph::set_last_error("unknown error");
        return SERAPH_EINVAL;
    }
}
