// seraph_gather_probe: the relax kernels' inner operation -- 4-byte reads of
// a vertex array at indexes taken from a sequential column stream -- timed in
// isolation, with the same L2 hints seraph_run uses (column stream
// evict-first, the hot index range evict-last under a persisting-L2
// set-aside).  With every index in a small hot range it measures the rate at
// which an SM turns random gathers into L2 hits, the ceiling of a pull pass
// whose gathers all hit L2; with cold indexes it shows what a DRAM miss
// costs.  A measurement aid: nothing in the method depends on it.
#include "common.cuh"

namespace seraph {
void set_last_error(const char* msg);
}

namespace {

using seraph::DevBuf;
using seraph::PersistingL2;
using seraph::device_sms;

constexpr int kProbeThreads = 256;

__device__ __forceinline__ uint64_t probe_policy_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t probe_policy_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t probe_policy_normal() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 probe_ld_stream(const uint4* p, uint64_t pol) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t probe_ld_gather(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

// splitmix64's output function (Steele, Lea and Flood, 2014) as an index hash.
__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Index i: hot with probability hot_p20 / 2^20, uniform over [0, hot)
// then, else uniform over [hot, n).  Both ranges are non-empty whenever they
// can be drawn (the host folds an empty range into the other).
__global__ void probe_index_kernel(uint32_t* idx, uint64_t m, uint32_t hot, uint32_t n,
                                   uint32_t hot_p20) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = probe_mix(i);
        const uint32_t lo = (uint32_t)r, sel = (uint32_t)(r >> 44);  // 20 bits
        idx[i] = sel < hot_p20 ? (uint32_t)(((uint64_t)lo * hot) >> 32)
                               : hot + (uint32_t)(((uint64_t)lo * (n - hot)) >> 32);
    }
}

// Eight gathers per thread and group, the relax kernels' batch size; their
// sum is written so that none of the loads can be dropped.
__global__ void __launch_bounds__(kProbeThreads) probe_gather_kernel(
    const uint4* __restrict__ idx, const uint32_t* __restrict__ val, float* __restrict__ out,
    uint64_t groups, uint32_t hot) {
    const uint64_t ps = probe_policy_first(), ph = probe_policy_last(), pn = probe_policy_normal();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < groups;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a = probe_ld_stream(idx + 2 * i, ps), b = probe_ld_stream(idx + 2 * i + 1, ps);
        const uint32_t c[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = probe_ld_gather(val + c[j], c[j] < hot ? ph : pn);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s += __uint_as_float(g[j]);
        out[i] = s;
    }
}

struct ProbeEvent {
    cudaEvent_t e = nullptr;
    ProbeEvent() { SR_CUDA(cudaEventCreate(&e)); }
    ~ProbeEvent() { if (e) cudaEventDestroy(e); }
};

int run_probe(uint64_t n_values, uint64_t n_gathers, uint64_t hot_values, double hot_frac,
              uint32_t reps, cudaStream_t s, double* best_seconds) {
    SR_CHECK(best_seconds != nullptr, SERAPH_EINVAL, "best_seconds is NULL");
    SR_CHECK(n_values > 0 && n_values < (1ull << 32), SERAPH_EINVAL,
             "n_values must be in [1, 2^32)");
    SR_CHECK(n_gathers > 0 && n_gathers % 8 == 0, SERAPH_EINVAL,
             "n_gathers must be a positive multiple of 8");
    SR_CHECK(hot_values <= n_values, SERAPH_EINVAL, "hot_values > n_values");
    SR_CHECK(hot_frac >= 0.0 && hot_frac <= 1.0, SERAPH_EINVAL, "hot_frac outside [0, 1]");
    SR_CHECK(reps > 0, SERAPH_EINVAL, "reps must be positive");
    // an empty range is never drawn
    const uint32_t hot_p20 = hot_values == 0 ? 0u
                             : hot_values == n_values ? (1u << 20)
                             : (uint32_t)(hot_frac * (double)(1u << 20) + 0.5);
    int dev = 0;
    SR_CUDA(cudaGetDevice(&dev));
    DevBuf<uint32_t> val(n_values), idx(n_gathers);
    DevBuf<float> out(n_gathers / 8);
    SR_CUDA(cudaMemsetAsync(val.p, 0, n_values * 4, s));
    const unsigned grid = (unsigned)device_sms() * 8;
    probe_index_kernel<<<grid, kProbeThreads, 0, s>>>(idx.p, n_gathers, (uint32_t)hot_values,
                                                      (uint32_t)n_values, hot_p20);
    SR_LAUNCH();
    PersistingL2 guard;
    if (hot_values) guard.reserve(dev, hot_values * 4);
    ProbeEvent t0, t1;
    double best = 1e30;
    for (uint32_t r = 0; r <= reps; ++r) {  // launch 0 warms up
        SR_CUDA(cudaEventRecord(t0.e, s));
        probe_gather_kernel<<<grid, kProbeThreads, 0, s>>>(
            reinterpret_cast<const uint4*>(idx.p), val.p, out.p, n_gathers / 8,
            (uint32_t)hot_values);
        SR_LAUNCH();
        SR_CUDA(cudaEventRecord(t1.e, s));
        SR_CUDA(cudaEventSynchronize(t1.e));
        float ms = 0.f;
        SR_CUDA(cudaEventElapsedTime(&ms, t0.e, t1.e));
        if (r > 0 && ms * 1e-3 < best) best = ms * 1e-3;
    }
    *best_seconds = best;
    return SERAPH_OK;
}

}  // namespace

extern "C" int seraph_gather_probe(uint64_t n_values, uint64_t n_gathers, uint64_t hot_values,
                                   double hot_frac, uint32_t reps, void* stream,
                                   double* best_seconds) {
    try {
        seraph::set_last_error("");
        return run_probe(n_values, n_gathers, hot_values, hot_frac, reps, (cudaStream_t)stream,
                         best_seconds);
    } catch (const seraph::Error& e) {
        seraph::set_last_error(e.what());
        return e.code;
    } catch (...) {
        seraph::set_last_error("unknown error");
        return SERAPH_EINVAL;
    }
}
