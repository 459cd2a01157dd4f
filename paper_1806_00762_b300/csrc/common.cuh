// Shared host/device helpers of the seraph library: error handling, RAII
// buffers, warp/block primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "seraph.h"

namespace seraph {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SR_CUDA(x)                                                                     \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            if (e_ == cudaErrorMemoryAllocation) (void)cudaGetLastError();             \
            throw ::seraph::Error(e_ == cudaErrorMemoryAllocation ? SERAPH_ENOMEM      \
                                                                  : SERAPH_ECUDA,      \
                                  std::string(#x) + ": " + cudaGetErrorString(e_));    \
        }                                                                              \
    } while (0)

#define SR_CHECK(cond, code, msg)                                                      \
    do {                                                                               \
        if (!(cond)) throw ::seraph::Error((code), (msg));                             \
    } while (0)

#define SR_LAUNCH() SR_CUDA(cudaGetLastError())

int device_sms();

// Evict-last lines live in the L2 set-aside for persisting accesses, which is
// empty unless the context limit is raised.  Held for one run, then the
// persisting lines are reset to normal and the previous limit comes back (a
// context limit: nothing outlasts the process).
struct PersistingL2 {
    bool set = false;
    size_t prev = 0;
    void reserve(int device, uint64_t bytes) {
        int maxp = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, device) != cudaSuccess ||
            maxp <= 0) {
            (void)cudaGetLastError();
            return;
        }
        if (cudaDeviceGetLimit(&prev, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        const size_t want = bytes < (uint64_t)maxp ? (size_t)bytes : (size_t)maxp;
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) set = true;
        else (void)cudaGetLastError();
    }
    ~PersistingL2() {
        if (!set) return;
        (void)cudaCtxResetPersistingL2Cache();
        (void)cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, prev);
        (void)cudaGetLastError();
    }
};

// The context's persisting-L2 set-aside for the evict-last hot range, held
// by the graphs whose runs use it: raised (only ever grown) on a run's
// first need, and put back to the context's earlier value -- persisting
// lines demoted first -- when the last holder lets go (graph freed or its
// buffers released).  A run that finds it raised calls nothing, so it never
// waits on work in flight elsewhere in the context.
void l2_setaside_hold(const void* holder, int device, uint64_t bytes);
void l2_setaside_drop(const void* holder);

// Device allocation owned by the library.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) SR_CUDA(cudaMalloc((void**)&p, count * sizeof(T)));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
};

// Host-side fault injection and accounting of pinned allocations (capi.cu;
// seraph_debug_fail_pinned_alloc / seraph_debug_pinned_bytes).
bool take_injected_pinned_failure();
void note_pinned_bytes(int64_t delta);

// Pinned host allocation owned by the library.
struct PinnedBuf {
    uint8_t* p = nullptr;
    size_t bytes = 0;
    // mapped: also map the pages into the device address space (kernels read
    // them directly over the host link; see device_ptr)
    void alloc(size_t b, bool mapped = false) {
        release();
        if (!b) return;
        SR_CHECK(!take_injected_pinned_failure(), SERAPH_ENOMEM,
                 "pinned host allocation failed (injected by seraph_debug_fail_pinned_alloc)");
        SR_CUDA(cudaHostAlloc((void**)&p, b,
                              cudaHostAllocPortable | (mapped ? cudaHostAllocMapped : 0u)));
        bytes = b;
        note_pinned_bytes((int64_t)b);
    }
    void release() {
        if (p) {
            cudaFreeHost(p);
            note_pinned_bytes(-(int64_t)bytes);
        }
        p = nullptr;
        bytes = 0;
    }
    PinnedBuf() = default;
    ~PinnedBuf() { release(); }
    PinnedBuf(const PinnedBuf&) = delete;
    PinnedBuf& operator=(const PinnedBuf&) = delete;
    PinnedBuf(PinnedBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    PinnedBuf& operator=(PinnedBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    // The device address of a mapped allocation (an error, not a device
    // fault, if it is not mapped); null for an empty buffer.
    template <class T>
    const T* device_ptr() const {
        if (!p) return nullptr;
        void* d = nullptr;
        SR_CUDA(cudaHostGetDevicePointer(&d, p, 0));
        return (const T*)d;
    }
};

struct Stream {
    cudaStream_t s = nullptr;
    bool owned = false;
    void create() {
        SR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        owned = true;
    }
    void use(void* ext) {
        if (ext) { s = (cudaStream_t)ext; owned = false; } else create();
    }
    ~Stream() { if (owned && s) cudaStreamDestroy(s); }
};

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------- device side

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan (blockDim.x = NT, multiple of 32).  `ws` must
// hold NT/32 + 1 elements of shared memory.  Returns the exclusive prefix
// and writes the block total to *total.
template <int NT, class T>
__device__ __forceinline__ T block_excl_scan(T x, T* ws, T* total) {
    const int warp = threadIdx.x >> 5, nw = NT / 32;
    T inc = warp_incl_scan(x);
    if (lane_id() == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T v = lane_id() < (unsigned)nw ? ws[lane_id()] : T(0);
        T s = warp_incl_scan(v);
        if (lane_id() < (unsigned)nw) ws[lane_id()] = s - v;
        if (lane_id() == (unsigned)nw - 1) ws[nw] = s;
    }
    __syncthreads();
    T r = ws[warp] + inc - x;
    *total = ws[nw];
    __syncthreads();
    return r;
}

// Vertices per checkpoint of a streamed header (one CTA's tile when the page
// is rebuilt on the device).
constexpr uint32_t kStreamTile = 256;
__host__ __device__ inline uint64_t stream_ckpt_bytes(uint64_t nv) {
    return 16 * ((nv + kStreamTile - 1) / kStreamTile + 1);
}
// one bit per vertex: set when it has an in-edge (32 bytes per tile)
__host__ __device__ inline uint64_t stream_bitmap_bytes(uint64_t nv) {
    return 32 * ((nv + kStreamTile - 1) / kStreamTile);
}
// two bytes per vertex with an in-edge
__host__ __device__ inline uint64_t stream_hdr_bytes(uint64_t nnz) { return (2 * nnz + 15) & ~15ull; }
__host__ __device__ inline uint64_t stream_esc_bytes(uint64_t nesc) { return (8 * nesc + 15) & ~15ull; }

}  // namespace seraph
