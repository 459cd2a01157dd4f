// Partitioner (Sec. 3.1 "Subgraph Organization"): raw edges -> paged CSC in
// pinned host memory, all on the GPU.
//
//   1. keys = (dst << b) | src per edge (self-loops -> the all-ones marker);
//   2. stable LSD radix sort of the keys (8-bit digits), weights as payload;
//   3. drop markers and duplicate keys (keeping the smallest weight);
//   4. in-edge offsets by binary search of each vertex in the sorted
//      destinations; out-degrees by atomic counting of the sources;
//   5. page cut: page j starts at the smallest v with
//      (v + off[v]) * P >= j * (n + E)  (balanced on vertices + in-edges);
//   6. page-relative u32 offsets staged on the device, then every page's
//      offsets / sources / weights copied into the pinned page images.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"
#include "graph.hpp"

namespace seraph {

int device_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

namespace {

constexpr int kNT = 256;
constexpr int kItems = 16;
constexpr uint64_t kTile = kNT * kItems;  // 4096 items per CTA tile
constexpr uint64_t kMarker = ~0ull;

unsigned grid_for(uint64_t n, int per_block = kNT) {
    uint64_t b = (n + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)device_sms() * 32;
    if (b > cap) b = cap;
    return (unsigned)std::max<uint64_t>(b, 1);
}

// ------------------------------------------------------------ device scan

template <class TI>
__global__ void __launch_bounds__(kNT) scan_reduce_kernel(const TI* __restrict__ in, uint64_t n,
                                                          uint64_t* __restrict__ sums) {
    __shared__ uint64_t ws[kNT / 32 + 1];
    uint64_t base = blockIdx.x * kTile, s = 0;
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + threadIdx.x;
        if (i < n) s += (uint64_t)in[i];
    }
    uint64_t tot;
    block_excl_scan<kNT>(s, ws, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class TI>
__global__ void __launch_bounds__(kNT) scan_down_kernel(const TI* in, uint64_t n,
                                                        const uint64_t* __restrict__ offs,
                                                        uint64_t* out) {
    __shared__ uint64_t ws[kNT / 32 + 1];
    uint64_t base = blockIdx.x * kTile, run = offs[blockIdx.x];
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + threadIdx.x;
        uint64_t x = i < n ? (uint64_t)in[i] : 0;
        uint64_t tot, ex = block_excl_scan<kNT>(x, ws, &tot);
        if (i < n) out[i] = run + ex;
        run += tot;
    }
}

// Exclusive scan of n values into uint64 (out may alias in when TI = uint64_t).
template <class TI>
void exclusive_scan(const TI* in, uint64_t n, uint64_t* out, cudaStream_t s) {
    if (n == 0) return;
    uint64_t nb = (n + kTile - 1) / kTile;
    DevBuf<uint64_t> offs(nb);
    if (nb == 1) {
        SR_CUDA(cudaMemsetAsync(offs.p, 0, sizeof(uint64_t), s));
    } else {
        DevBuf<uint64_t> sums(nb);
        scan_reduce_kernel<TI><<<(unsigned)nb, kNT, 0, s>>>(in, n, sums.p);
        SR_LAUNCH();
        exclusive_scan<uint64_t>(sums.p, nb, offs.p, s);
        SR_CUDA(cudaStreamSynchronize(s));  // sums freed at scope exit
    }
    scan_down_kernel<TI><<<(unsigned)nb, kNT, 0, s>>>(in, n, offs.p, out);
    SR_LAUNCH();
    SR_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ radix sort

__global__ void __launch_bounds__(kNT) rs_hist_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                      int shift, uint32_t* __restrict__ hist,
                                                      uint64_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + threadIdx.x;
        unsigned d = i < n ? (unsigned)(keys[i] >> shift) & 255u : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        if (d < 256 && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

constexpr size_t kScatterSmem = kTile * 8 + kTile * 4 + 8 * 256 * 4 + 256 * 4 + 256 * 4 +
                                256 * 8 + (kNT / 32 + 1) * 4;

template <bool HAS_VAL>
__global__ void __launch_bounds__(kNT) rs_scatter_kernel(const uint64_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint64_t n, int shift,
                                                         const uint64_t* __restrict__ offs,
                                                         uint64_t ntiles,
                                                         uint64_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t* s_keys = (uint64_t*)smem;
    uint32_t* s_vals = (uint32_t*)(s_keys + kTile);
    uint32_t* s_wcnt = s_vals + kTile;        // [8 warps][256 digits]
    uint32_t* s_run = s_wcnt + 8 * 256;       // running count per digit
    uint32_t* s_start = s_run + 256;          // tile-local digit start
    uint64_t* s_goff = (uint64_t*)(s_start + 256);
    uint32_t* ws = (uint32_t*)(s_goff + 256);

    const unsigned tid = threadIdx.x, warp = tid >> 5;
    const uint64_t tile = blockIdx.x, base = tile * kTile;
    s_run[tid] = 0;
    s_goff[tid] = offs[(uint64_t)tid * ntiles + tile];

    uint64_t k[kItems];
    uint32_t v[kItems], rank[kItems];
    unsigned dg[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + tid;
        bool valid = i < n;
        k[r] = valid ? kin[i] : kMarker;
        v[r] = (HAS_VAL && valid) ? vin[i] : 0u;
        dg[r] = valid ? (unsigned)(k[r] >> shift) & 255u : 256u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        for (unsigned j = tid; j < 8 * 256; j += kNT) s_wcnt[j] = 0;
        __syncthreads();
        unsigned d = dg[r];
        unsigned peers = __match_any_sync(kFull, d);
        unsigned lr = __popc(peers & lanemask_lt());
        if (d < 256 && lr == 0) s_wcnt[warp * 256 + d] = __popc(peers);
        __syncthreads();
        {
            unsigned run = s_run[tid];
#pragma unroll
            for (int w = 0; w < kNT / 32; ++w) {
                unsigned c = s_wcnt[w * 256 + tid];
                s_wcnt[w * 256 + tid] = run;
                run += c;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        rank[r] = d < 256 ? s_wcnt[warp * 256 + d] + lr : 0u;
        __syncthreads();
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<kNT>(s_run[tid], ws, &tot);
    s_start[tid] = ex;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        if (dg[r] < 256) {
            unsigned pos = s_start[dg[r]] + rank[r];
            s_keys[pos] = k[r];
            if (HAS_VAL) s_vals[pos] = v[r];
        }
    }
    __syncthreads();
    uint64_t count = n - base < kTile ? n - base : kTile;
    for (unsigned j = tid; j < count; j += kNT) {
        uint64_t key = s_keys[j];
        unsigned d = (unsigned)(key >> shift) & 255u;
        uint64_t g = s_goff[d] + (j - s_start[d]);
        kout[g] = key;
        if (HAS_VAL) vout[g] = s_vals[j];
    }
}

// Sorts keys (and vals) ascending on their low `bits` bits; stable.  On
// return keys/vals point at the sorted data (buffers may have swapped).
void radix_sort(DevBuf<uint64_t>& keys, DevBuf<uint64_t>& keys_alt, DevBuf<uint32_t>& vals,
                DevBuf<uint32_t>& vals_alt, uint64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return;
    const bool has_val = vals.p != nullptr;
    uint64_t ntiles = (n + kTile - 1) / kTile;
    DevBuf<uint32_t> hist(256 * ntiles);
    DevBuf<uint64_t> offs(256 * ntiles);
    static bool attr_set = false;
    if (!attr_set) {
        SR_CUDA(cudaFuncSetAttribute(rs_scatter_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kScatterSmem));
        SR_CUDA(cudaFuncSetAttribute(rs_scatter_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kScatterSmem));
        attr_set = true;
    }
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<(unsigned)ntiles, kNT, 0, s>>>(keys.p, n, shift, hist.p, ntiles);
        SR_LAUNCH();
        exclusive_scan<uint32_t>(hist.p, 256 * ntiles, offs.p, s);
        if (has_val)
            rs_scatter_kernel<true><<<(unsigned)ntiles, kNT, kScatterSmem, s>>>(
                keys.p, vals.p, n, shift, offs.p, ntiles, keys_alt.p, vals_alt.p);
        else
            rs_scatter_kernel<false><<<(unsigned)ntiles, kNT, kScatterSmem, s>>>(
                keys.p, nullptr, n, shift, offs.p, ntiles, keys_alt.p, nullptr);
        SR_LAUNCH();
        std::swap(keys, keys_alt);
        if (has_val) std::swap(vals, vals_alt);
    }
    SR_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------- build steps

__global__ void check_ids_kernel(const uint32_t* __restrict__ a, uint64_t m, uint64_t n,
                                 unsigned* bad) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (a[i] >= n) atomicOr(bad, 1u);
}

__global__ void make_keys_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                 const uint32_t* __restrict__ w, uint64_t m, int b, bool sym,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t u = src[i], v = dst[i];
        uint64_t k = u == v ? kMarker : (v << b) | u;
        keys[i] = k;
        if (vals) vals[i] = w[i];
        if (sym) {
            keys[m + i] = u == v ? kMarker : (u << b) | v;
            if (vals) vals[m + i] = w[i];
        }
    }
}

__global__ void __launch_bounds__(kNT) dedupe_count_kernel(const uint64_t* __restrict__ keys,
                                                           uint64_t n, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t ws[kNT / 32 + 1];
    uint64_t base = blockIdx.x * kTile;
    uint32_t c = 0;
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + threadIdx.x;
        if (i < n) {
            uint64_t k = keys[i];
            c += (k != kMarker && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
        }
    }
    uint32_t tot;
    block_excl_scan<kNT>(c, ws, &tot);
    if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kNT) dedupe_write_kernel(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n,
    const uint64_t* __restrict__ tile_off, int b, uint32_t* __restrict__ col,
    uint32_t* __restrict__ dcol, uint32_t* __restrict__ wout) {
    __shared__ uint32_t ws[kNT / 32 + 1];
    const uint64_t base = blockIdx.x * kTile;
    const uint64_t mask = (1ull << b) - 1;
    uint64_t run = tile_off[blockIdx.x];
    for (int r = 0; r < kItems; ++r) {
        uint64_t i = base + (uint64_t)r * kNT + threadIdx.x;
        uint64_t k = i < n ? keys[i] : kMarker;
        uint32_t keep = (i < n && k != kMarker && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
        uint32_t tot, ex = block_excl_scan<kNT>(keep, ws, &tot);
        if (keep) {
            uint64_t pos = run + ex;
            col[pos] = (uint32_t)(k & mask);
            dcol[pos] = (uint32_t)(k >> b);
            if (vals) {
                uint32_t wm = vals[i];
                for (uint64_t j = i + 1; j < n && keys[j] == k; ++j) wm = min(wm, vals[j]);
                wout[pos] = wm;
            }
        }
        run += tot;
    }
}

__global__ void col_off_kernel(const uint32_t* __restrict__ dcol, uint64_t E, uint64_t n,
                               uint64_t* __restrict__ col_off) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v <= n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo = 0, hi = E;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if ((uint64_t)dcol[mid] < v) lo = mid + 1; else hi = mid;
        }
        col_off[v] = lo;
    }
}

__global__ void outdeg_kernel(const uint32_t* __restrict__ col, uint64_t E,
                              uint32_t* __restrict__ outdeg) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E;
         i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&outdeg[col[i]], 1u);
}

__global__ void max_indeg_kernel(const uint64_t* __restrict__ col_off, uint64_t n, unsigned* mx) {
    unsigned local = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t d = col_off[v + 1] - col_off[v];
        local = max(local, d > 0xFFFFFFFFull ? 0xFFFFFFFFu : (unsigned)d);
    }
    local = __reduce_max_sync(kFull, local);
    if (lane_id() == 0) atomicMax(mx, local);
}

__global__ void max_u32_kernel(const uint32_t* __restrict__ a, uint64_t n, unsigned* mx) {
    unsigned local = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        local = max(local, a[i]);
    local = __reduce_max_sync(kFull, local);
    if (lane_id() == 0) atomicMax(mx, local);
}

// Weights narrowed to `wb` bytes (lossless: wb is chosen from the maximum).
__global__ void narrow_kernel(const uint32_t* __restrict__ w, uint64_t n, int wb,
                              uint8_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (wb == 1) out[i] = (uint8_t)w[i];
        else ((uint16_t*)out)[i] = (uint16_t)w[i];
    }
}

__global__ void zero_in_kernel(const uint64_t* __restrict__ col_off, uint64_t n,
                               uint32_t* __restrict__ bits) {
    const uint64_t words = (n + 31) / 32;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (uint32_t j = 0; j < 32; ++j) {
            uint64_t v = 32 * w + j;
            if (v < n && col_off[v + 1] == col_off[v]) m |= 1u << j;
        }
        bits[w] = m;
    }
}

// Page p's source-block bitmap: one CTA per page ORs the block of every
// in-edge source into shared memory, then writes the page's words.
__global__ void __launch_bounds__(kNT) page_blocks_kernel(const uint32_t* __restrict__ col,
                                                          const uint64_t* __restrict__ eb,
                                                          uint32_t bsz, uint32_t* __restrict__ out) {
    __shared__ uint32_t bits[kPageBlockWords];
    if (threadIdx.x < kPageBlockWords) bits[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t b = eb[blockIdx.x], e = eb[blockIdx.x + 1];
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const uint32_t blk = col[i] / bsz;
        atomicOr(&bits[blk >> 5], 1u << (blk & 31));
    }
    __syncthreads();
    if (threadIdx.x < kPageBlockWords) out[(uint64_t)blockIdx.x * kPageBlockWords + threadIdx.x] = bits[threadIdx.x];
}

__global__ void page_cut_kernel(const uint64_t* __restrict__ col_off, uint64_t n, uint32_t P,
                                uint64_t* __restrict__ vb) {
    const uint64_t total = n + col_off[n];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j <= P;
         j += (uint64_t)gridDim.x * blockDim.x) {
        if (j == 0) { vb[0] = 0; continue; }
        if (j == P) { vb[P] = n; continue; }
        uint64_t lo = 0, hi = n, target = j * total;
        while (lo < hi) {  // smallest v in [0, n] with (v + off[v]) * P >= j * total
            uint64_t mid = (lo + hi) >> 1;
            if ((mid + col_off[mid]) * (uint64_t)P >= target) hi = mid; else lo = mid + 1;
        }
        vb[j] = lo;
    }
}

__global__ void gather_off_kernel(const uint64_t* __restrict__ col_off,
                                  const uint64_t* __restrict__ vb, uint32_t P,
                                  uint64_t* __restrict__ eb) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j <= P;
         j += (uint64_t)gridDim.x * blockDim.x)
        eb[j] = col_off[vb[j]];
}

// Page-relative offsets: stage[st[p] + i] = off[vb_p + i] - off[vb_p], i in [0, nv_p].
__global__ void stage_off_kernel(const uint64_t* __restrict__ col_off,
                                 const uint64_t* __restrict__ vb, const uint64_t* __restrict__ st,
                                 uint32_t P, uint64_t n, uint32_t* __restrict__ stage,
                                 unsigned* __restrict__ page_maxdeg) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v <= n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        // page p owning v: largest p with vb[p] <= v, p < P (v = n closes page P-1)
        uint32_t lo = 0, hi = P - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (vb[mid] <= v) lo = mid; else hi = mid - 1;
        }
        uint32_t p = lo;
        stage[st[p] + (v - vb[p])] = (uint32_t)(col_off[v] - col_off[vb[p]]);
        if (v < n) {
            const uint64_t d = col_off[v + 1] - col_off[v];
            if (d) atomicMax(&page_maxdeg[p], d > 0xFFFFFFFFull ? 0xFFFFFFFFu : (unsigned)d);
        }
        // a vertex that closes page p-1 (v == vb[p], p > 0) also writes its end
        if (v == vb[p] && p > 0) {
            uint32_t q = p - 1;
            while (true) {  // pages q with vb[q+1] == v (several if some are empty)
                stage[st[q] + (v - vb[q])] = (uint32_t)(col_off[v] - col_off[vb[q]]);
                if (q == 0 || vb[q] != v) break;
                --q;
            }
        }
    }
}

// Flags CSR offsets that do not start at 0 or decrease somewhere.
__global__ void check_csr_kernel(const uint64_t* __restrict__ row_off, uint64_t n,
                                 unsigned* __restrict__ bad) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        if ((v == 0 && row_off[0] != 0) || row_off[v] > row_off[v + 1]) atomicOr(bad, 1u);
    }
}

__global__ void expand_csr_kernel(const uint64_t* __restrict__ row_off, uint64_t n,
                                  uint32_t* __restrict__ src) {
    uint64_t E = row_off[n];
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo = 0, hi = n - 1;  // largest u with row_off[u] <= e
        while (lo < hi) {
            uint64_t mid = (lo + hi + 1) >> 1;
            if (row_off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        src[e] = (uint32_t)lo;
    }
}

// Vertex keys for the out-degree order: (maxdeg - deg) above the id, so an
// ascending sort gives non-increasing degree with ascending ids among ties.
__global__ void vertex_key_kernel(const uint32_t* __restrict__ deg, uint64_t n, uint32_t maxdeg,
                                  int b, uint64_t* __restrict__ keys) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(maxdeg - deg[v]) << b) | v;
}

__global__ void perm_kernel(const uint64_t* __restrict__ keys, uint64_t n, int b,
                            uint32_t* __restrict__ perm, uint32_t* __restrict__ inv) {
    const uint64_t mask = (1ull << b) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(keys[i] & mask);
        perm[i] = v;
        inv[v] = (uint32_t)i;
    }
}

__global__ void relabel_keys_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ dcol,
                                    const uint32_t* __restrict__ inv, uint64_t E, int b,
                                    uint64_t* __restrict__ keys) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x)
        keys[e] = ((uint64_t)inv[dcol[e]] << b) | inv[col[e]];
}

// Out-edge keys (source << b) | destination of the CSC's edges (dst[e] is
// edge e's destination), with the stored weight widened to 32 bits.
__global__ void out_keys_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                const uint8_t* __restrict__ w, int wb, uint64_t E, int b,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x) {
        keys[e] = ((uint64_t)src[e] << b) | dst[e];
        if (vals) {
            uint32_t x = 0;
            if (wb == 1) x = w[e];
            else if (wb == 2) x = ((const uint16_t*)w)[e];
            else x = ((const uint32_t*)w)[e];
            vals[e] = x;
        }
    }
}

__global__ void split_keys_kernel(const uint64_t* __restrict__ keys, uint64_t E, int b,
                                  uint32_t* __restrict__ col, uint32_t* __restrict__ dcol) {
    const uint64_t mask = (1ull << b) - 1;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x) {
        col[e] = (uint32_t)(keys[e] & mask);
        dcol[e] = (uint32_t)(keys[e] >> b);
    }
}

// ------------------------------------------------------- packed columns

__device__ __forceinline__ uint32_t leb_len(uint32_t v) {
    return v < (1u << 7) ? 1u : v < (1u << 14) ? 2u : v < (1u << 21) ? 3u : v < (1u << 28) ? 4u : 5u;
}

// Bit e set: edge e is the first in-edge of its destination.
__global__ void first_bits_kernel(const uint64_t* __restrict__ col_off, uint64_t n,
                                  uint32_t* __restrict__ bits) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = col_off[v];
        if (e < col_off[v + 1]) atomicOr(&bits[e >> 5], 1u << (e & 31));
    }
}

// The value stored for edge e: its source id if it is its destination's
// first in-edge, else the gap to the previous source minus one (sources are
// strictly ascending within a destination).
__device__ __forceinline__ uint32_t gap_value(const uint32_t* __restrict__ col,
                                              const uint32_t* __restrict__ first, uint64_t e) {
    const bool f = (first[e >> 5] >> (e & 31)) & 1u;
    return f ? col[e] : col[e] - col[e - 1] - 1u;
}

__global__ void leb_len_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ first,
                               uint64_t E, uint8_t* __restrict__ lens) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x)
        lens[e] = (uint8_t)leb_len(gap_value(col, first, e));
}

__global__ void leb_write_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ first,
                                 uint64_t E, const uint64_t* __restrict__ pos,
                                 uint8_t* __restrict__ data) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v = gap_value(col, first, e);
        uint64_t q = pos[e];
        for (;;) {
            const uint8_t b = (uint8_t)(v & 0x7Fu);
            v >>= 7;
            if (!v) { data[q] = b; break; }
            data[q++] = b | 0x80u;
        }
    }
}

// Global byte offset of each destination's bytes (n+1 entries).
__global__ void vertex_boff_kernel(const uint64_t* __restrict__ col_off, uint64_t n,
                                   const uint64_t* __restrict__ pos, uint64_t E, uint64_t total,
                                   uint64_t* __restrict__ gboff) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v <= n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = col_off[v];
        gboff[v] = e < E ? pos[e] : total;
    }
}

int bits_for(uint64_t n) {
    int b = 1;
    while (b < 64 && (1ull << b) < n) ++b;
    return b;
}

template <class T>
const T* to_device(const T* p, uint64_t count, int mem, DevBuf<T>& hold, cudaStream_t s) {
    if (mem == SERAPH_MEM_DEVICE || p == nullptr) return p;
    hold.alloc(count);
    if (count) SR_CUDA(cudaMemcpyAsync(hold.p, p, count * sizeof(T), cudaMemcpyHostToDevice, s));
    return hold.p;
}

// Renumber the vertices of a deduplicated edge list (col = lo endpoint, dcol =
// hi endpoint, sorted by (hi, lo)) in order of non-increasing occurrence count
// in `col` -- the out-degree for the CSC -- ties by ascending id, and re-sort
// the edges by (new hi, new lo).  perm: new -> old, inv: old -> new.
void relabel_by_degree(uint64_t n, uint64_t E, int b, DevBuf<uint32_t>& col, DevBuf<uint32_t>& dcol,
                       DevBuf<uint32_t>& wcol, bool weighted, DevBuf<uint32_t>& perm,
                       DevBuf<uint32_t>& inv, cudaStream_t s) {
    {
        DevBuf<uint32_t> deg(n);
        SR_CUDA(cudaMemsetAsync(deg.p, 0, n * sizeof(uint32_t), s));
        if (E) {
            outdeg_kernel<<<grid_for(E), kNT, 0, s>>>(col.p, E, deg.p);
            SR_LAUNCH();
        }
        DevBuf<unsigned> mx(1);
        SR_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned), s));
        max_u32_kernel<<<grid_for(n), kNT, 0, s>>>(deg.p, n, mx.p);
        SR_LAUNCH();
        unsigned hmx = 0;
        SR_CUDA(cudaMemcpyAsync(&hmx, mx.p, 4, cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        DevBuf<uint64_t> vk(n), vk_alt(n);
        vertex_key_kernel<<<grid_for(n), kNT, 0, s>>>(deg.p, n, hmx, b, vk.p);
        SR_LAUNCH();
        DevBuf<uint32_t> none, none_alt;
        radix_sort(vk, vk_alt, none, none_alt, n, b + bits_for((uint64_t)hmx + 1), s);
        perm.alloc(n);
        inv.alloc(n);
        perm_kernel<<<grid_for(n), kNT, 0, s>>>(vk.p, n, b, perm.p, inv.p);
        SR_LAUNCH();
        SR_CUDA(cudaStreamSynchronize(s));
    }
    if (!E) return;
    DevBuf<uint64_t> keys(E);
    relabel_keys_kernel<<<grid_for(E), kNT, 0, s>>>(col.p, dcol.p, inv.p, E, b, keys.p);
    SR_LAUNCH();
    SR_CUDA(cudaStreamSynchronize(s));
    col.release();
    dcol.release();
    DevBuf<uint64_t> keys_alt(E);
    DevBuf<uint32_t> vals, vals_alt;
    if (weighted) {
        vals = std::move(wcol);
        vals_alt.alloc(E);
    }
    radix_sort(keys, keys_alt, vals, vals_alt, E, 2 * b, s);
    keys_alt.release();
    vals_alt.release();
    col.alloc(E);
    dcol.alloc(E);
    split_keys_kernel<<<grid_for(E), kNT, 0, s>>>(keys.p, E, b, col.p, dcol.p);
    SR_LAUNCH();
    if (weighted) wcol = std::move(vals);
    SR_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

// Sorted, deduplicated adjacency of raw edges (lo -> hi): rows are the `hi`
// endpoints, each row lists its `lo` endpoints ascending.  With lo = source
// and hi = destination this is the CSC of Sec. 3.1; with the two swapped it is
// the out-edge CSR.  Self-loops are dropped, duplicates keep the smallest
// weight, weights are narrowed to the smallest lossless width.
void sorted_adjacency(uint64_t n, uint64_t m, const uint32_t* lo_in, const uint32_t* hi_in,
                      const uint32_t* w_in, int mem, bool sym, cudaStream_t s, Adjacency& A,
                      DevBuf<uint32_t>* perm, DevBuf<uint32_t>* inv) {
    const uint64_t M = sym ? 2 * m : m;
    const bool weighted = w_in != nullptr;
    const int b = bits_for(n);
    DevBuf<uint64_t> keys(M), keys_alt(M);
    DevBuf<uint32_t> vals, vals_alt;
    if (weighted) { vals.alloc(M); vals_alt.alloc(M); }
    {
        DevBuf<uint32_t> hs, hd, hw;
        const uint32_t* src = to_device(lo_in, m, mem, hs, s);
        const uint32_t* dst = to_device(hi_in, m, mem, hd, s);
        const uint32_t* w = to_device(w_in, m, mem, hw, s);
        if (m) {
            DevBuf<unsigned> bad(1);
            SR_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
            check_ids_kernel<<<grid_for(m), kNT, 0, s>>>(src, m, n, bad.p);
            check_ids_kernel<<<grid_for(m), kNT, 0, s>>>(dst, m, n, bad.p);
            SR_LAUNCH();
            unsigned hb = 0;
            SR_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            SR_CUDA(cudaStreamSynchronize(s));
            SR_CHECK(hb == 0, SERAPH_EINVAL, "an edge endpoint is >= n");
            make_keys_kernel<<<grid_for(m), kNT, 0, s>>>(src, dst, w, m, b, sym, keys.p, vals.p);
            SR_LAUNCH();
        }
        SR_CUDA(cudaStreamSynchronize(s));
    }
    radix_sort(keys, keys_alt, vals, vals_alt, M, 2 * b, s);
    keys_alt.release();
    vals_alt.release();

    // dedupe + compaction
    uint64_t ntiles = (M + kTile - 1) / kTile;
    uint64_t E = 0;
    DevBuf<uint32_t> dcol;
    DevBuf<uint32_t>& col = A.col;
    DevBuf<uint32_t>& wcol = A.wcol;
    if (M) {
        DevBuf<uint32_t> cnt(ntiles);
        DevBuf<uint64_t> toff(ntiles + 1);
        dedupe_count_kernel<<<(unsigned)ntiles, kNT, 0, s>>>(keys.p, M, cnt.p);
        SR_LAUNCH();
        exclusive_scan<uint32_t>(cnt.p, ntiles, toff.p, s);
        uint64_t last_off = 0;
        uint32_t last_cnt = 0;
        SR_CUDA(cudaMemcpyAsync(&last_off, toff.p + ntiles - 1, 8, cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaMemcpyAsync(&last_cnt, cnt.p + ntiles - 1, 4, cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        E = last_off + last_cnt;
        col.alloc(std::max<uint64_t>(E, 1));
        dcol.alloc(std::max<uint64_t>(E, 1));
        if (weighted) wcol.alloc(std::max<uint64_t>(E, 1));
        dedupe_write_kernel<<<(unsigned)ntiles, kNT, 0, s>>>(keys.p, vals.p, M, toff.p, b, col.p,
                                                             dcol.p, wcol.p);
        SR_LAUNCH();
        SR_CUDA(cudaStreamSynchronize(s));
    }
    keys.release();
    vals.release();
    if (perm) relabel_by_degree(n, E, b, col, dcol, wcol, weighted, *perm, *inv, s);
    A.E = E;
    // Narrowest lossless weight width (Sec. 3.1: the page format keeps the
    // transferred data as compact as possible).
    DevBuf<uint8_t>& wnar = A.wnar;
    if (weighted && E) {
        DevBuf<unsigned> mx(1);
        SR_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned), s));
        max_u32_kernel<<<grid_for(E), kNT, 0, s>>>(wcol.p, E, mx.p);
        SR_LAUNCH();
        unsigned hmx = 0;
        SR_CUDA(cudaMemcpyAsync(&hmx, mx.p, 4, cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        A.wbytes = hmx <= 0xFFu ? 1 : (hmx <= 0xFFFFu ? 2 : 4);
        if (A.wbytes < 4) {
            wnar.alloc(E * A.wbytes);
            narrow_kernel<<<grid_for(E), kNT, 0, s>>>(wcol.p, E, (int)A.wbytes, wnar.p);
            SR_LAUNCH();
            SR_CUDA(cudaStreamSynchronize(s));
            wcol.release();
        }
    }
    A.off.alloc(n + 1);
    col_off_kernel<<<grid_for(n + 1), kNT, 0, s>>>(dcol.p, E, n, A.off.p);
    SR_LAUNCH();
    dcol.release();
    SR_CUDA(cudaStreamSynchronize(s));
}

// Out-edge CSR (SERAPH_OUT_EDGES) from the CSC: every kept edge as the key
// (source << b) | destination with its weight, sorted, then split into
// offsets per source and destinations ascending; copied into pinned memory.
void build_out_edges(seraph_graph* g, uint64_t n, uint64_t E, DevBuf<uint32_t>& col,
                     const DevBuf<uint64_t>& col_off, const uint8_t* wsrc, bool weighted,
                     cudaStream_t s) {
    const int b = bits_for(n);
    g->h_out_off.alloc(8 * (n + 1), true);
    if (E) g->h_out_col.alloc(4 * E, true);
    if (weighted && E) g->h_out_w.alloc((uint64_t)g->wbytes * E, true);
    DevBuf<uint64_t> out_off(n + 1);
    if (E) {
        DevBuf<uint64_t> keys(E), keys_alt(E);
        DevBuf<uint32_t> vals, vals_alt;
        {
            DevBuf<uint32_t> dst(E);
            expand_csr_kernel<<<grid_for(E), kNT, 0, s>>>(col_off.p, n, dst.p);
            SR_LAUNCH();
            if (weighted) { vals.alloc(E); vals_alt.alloc(E); }
            out_keys_kernel<<<grid_for(E), kNT, 0, s>>>(col.p, dst.p, wsrc, (int)g->wbytes, E, b,
                                                       keys.p, vals.p);
            SR_LAUNCH();
            SR_CUDA(cudaStreamSynchronize(s));
        }
        radix_sort(keys, keys_alt, vals, vals_alt, E, 2 * b, s);
        keys_alt.release();
        vals_alt.release();
        DevBuf<uint32_t> ocol(E), osrc(E);
        split_keys_kernel<<<grid_for(E), kNT, 0, s>>>(keys.p, E, b, ocol.p, osrc.p);
        SR_LAUNCH();
        col_off_kernel<<<grid_for(n + 1), kNT, 0, s>>>(osrc.p, E, n, out_off.p);
        SR_LAUNCH();
        SR_CUDA(cudaStreamSynchronize(s));
        keys.release();
        osrc.release();
        SR_CUDA(cudaMemcpyAsync(g->h_out_col.p, ocol.p, 4 * E, cudaMemcpyDeviceToHost, s));
        if (weighted) {
            if (g->wbytes < 4) {
                DevBuf<uint8_t> wn((uint64_t)g->wbytes * E);
                narrow_kernel<<<grid_for(E), kNT, 0, s>>>(vals.p, E, (int)g->wbytes, wn.p);
                SR_LAUNCH();
                SR_CUDA(cudaMemcpyAsync(g->h_out_w.p, wn.p, (uint64_t)g->wbytes * E,
                                        cudaMemcpyDeviceToHost, s));
                SR_CUDA(cudaStreamSynchronize(s));
            } else {
                SR_CUDA(cudaMemcpyAsync(g->h_out_w.p, vals.p, 4 * E, cudaMemcpyDeviceToHost, s));
            }
        }
    } else {
        SR_CUDA(cudaMemsetAsync(out_off.p, 0, 8 * (n + 1), s));
    }
    SR_CUDA(cudaMemcpyAsync(g->h_out_off.p, out_off.p, 8 * (n + 1), cudaMemcpyDeviceToHost, s));
    SR_CUDA(cudaStreamSynchronize(s));
    g->out_edges = true;
}

// Runs f(p) for every page p on a few host threads (pages taken in turn).
template <class F>
void for_pages(uint32_t P, F f) {
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<uint32_t> next{0};
    auto work = [&] {
        for (uint32_t p; (p = next.fetch_add(1)) < P;) f(p);
    };
    std::vector<std::thread> ts;
    for (unsigned i = 1; i < hw; ++i) ts.emplace_back(work);
    work();
    for (auto& t : ts) t.join();
}

// The header that a packed page streams with when a plain chunk is sent in
// compact form (PageMeta::sh_*): per vertex one bit (has an in-edge) and,
// for the vertices that have one, two bytes (in-degree, code bytes) instead
// of the two u32 offsets, plus the offsets of every kStreamTile-th vertex, so
// the device rebuilds both offset arrays one tile per CTA without a
// page-wide scan.  Read from the packed pages' own off and boff arrays, on
// the host.
static void build_stream_headers(seraph_graph* g) {
    const uint32_t P = g->num_pages;
    auto arrays = [&](const PageMeta& pm, const uint32_t*& off, const uint32_t*& boff) {
        off = (const uint32_t*)(g->h_pack.p + pm.pk_off);
        boff = (const uint32_t*)(g->h_pack.p + pm.pk_off + pm.off_bytes);
    };
    auto escaped = [](uint32_t d, uint32_t l) { return d >= 255u || l >= 255u; };
    for_pages(P, [&](uint32_t p) {
        PageMeta& pm = g->pages[p];
        const uint32_t *off, *boff;
        arrays(pm, off, boff);
        uint32_t nesc = 0, nnz = 0;
        for (uint64_t v = 0; v < pm.nv; ++v) {
            const uint32_t d = off[v + 1] - off[v];
            nnz += d > 0;
            nesc += escaped(d, boff[v + 1] - boff[v]);
        }
        pm.sh_nesc = nesc;
        pm.sh_nnz = nnz;
        pm.sh_bytes = stream_ckpt_bytes(pm.nv) + stream_bitmap_bytes(pm.nv) + stream_hdr_bytes(nnz) +
                      stream_esc_bytes(nesc);
    });
    uint64_t total = 0;
    for (uint32_t p = 0; p < P; ++p) {
        g->pages[p].sh_off = total;
        total += g->pages[p].sh_bytes;
    }
    g->h_shdr.alloc(total);
    for_pages(P, [&](uint32_t p) {
        const PageMeta& pm = g->pages[p];
        const uint32_t *off, *boff;
        arrays(pm, off, boff);
        uint8_t* h = g->h_shdr.p + pm.sh_off;
        std::memset(h, 0, pm.sh_bytes);
        uint32_t* ck = (uint32_t*)h;
        uint32_t* bits = (uint32_t*)(h + stream_ckpt_bytes(pm.nv));
        uint16_t* hd = (uint16_t*)(h + stream_ckpt_bytes(pm.nv) + stream_bitmap_bytes(pm.nv));
        uint32_t* es = (uint32_t*)(h + stream_ckpt_bytes(pm.nv) + stream_bitmap_bytes(pm.nv) +
                                   stream_hdr_bytes(pm.sh_nnz));
        uint32_t ne = 0, nz = 0;
        for (uint64_t v = 0; v <= pm.nv; ++v) {
            if (v % kStreamTile == 0 || v == pm.nv) {
                const uint64_t t = (v + kStreamTile - 1) / kStreamTile;  // v / tile, or T at the end
                ck[4 * t] = off[v];
                ck[4 * t + 1] = boff[v];
                ck[4 * t + 2] = ne;
                ck[4 * t + 3] = nz;
            }
            if (v == pm.nv) break;
            const uint32_t d = off[v + 1] - off[v], l = boff[v + 1] - boff[v];
            if (d == 0) continue;
            bits[v / 32] |= 1u << (v % 32);
            if (escaped(d, l)) {
                hd[nz] = 0xFFFFu;
                es[2 * ne] = d;
                es[2 * ne + 1] = l;
                ++ne;
            } else {
                hd[nz] = (uint16_t)(d | (l << 8));
            }
            ++nz;
        }
    });
}

// The packed page form (SERAPH_COMPRESS): LEB128 gap streams of every
// destination's sources, encoded on the device, then laid out per page in
// pinned memory as off (copied from `stage`), boff and the stream bytes.
void build_packed(seraph_graph* g, uint64_t n, uint64_t E, const uint32_t* col,
                  const uint64_t* col_off, const uint64_t* d_vb, const uint64_t* d_st,
                  const std::vector<uint64_t>& st, const DevBuf<uint32_t>& stage, cudaStream_t s) {
    const uint32_t P = g->num_pages;
    DevBuf<uint64_t> pos(std::max<uint64_t>(E, 1));
    uint64_t total = 0;
    if (E) {
        DevBuf<uint32_t> first((E + 31) / 32);
        SR_CUDA(cudaMemsetAsync(first.p, 0, ((E + 31) / 32) * sizeof(uint32_t), s));
        first_bits_kernel<<<grid_for(n), kNT, 0, s>>>(col_off, n, first.p);
        SR_LAUNCH();
        {
            DevBuf<uint8_t> lens(E);
            leb_len_kernel<<<grid_for(E), kNT, 0, s>>>(col, first.p, E, lens.p);
            SR_LAUNCH();
            exclusive_scan<uint8_t>(lens.p, E, pos.p, s);
            uint64_t last_pos = 0;
            uint8_t last_len = 0;
            SR_CUDA(cudaMemcpyAsync(&last_pos, pos.p + E - 1, 8, cudaMemcpyDeviceToHost, s));
            SR_CUDA(cudaMemcpyAsync(&last_len, lens.p + E - 1, 1, cudaMemcpyDeviceToHost, s));
            SR_CUDA(cudaStreamSynchronize(s));
            total = last_pos + last_len;
        }
        DevBuf<uint8_t> data(total);
        leb_write_kernel<<<grid_for(E), kNT, 0, s>>>(col, first.p, E, pos.p, data.p);
        SR_LAUNCH();
        SR_CUDA(cudaStreamSynchronize(s));
        g->d_pack_tmp = std::move(data);
    }
    DevBuf<uint64_t> gboff(n + 1);
    vertex_boff_kernel<<<grid_for(n + 1), kNT, 0, s>>>(col_off, n, pos.p, E, total, gboff.p);
    SR_LAUNCH();
    SR_CUDA(cudaStreamSynchronize(s));
    pos.release();
    DevBuf<uint64_t> d_gb(P + 1);
    gather_off_kernel<<<grid_for(P + 1), kNT, 0, s>>>(gboff.p, d_vb, P, d_gb.p);
    SR_LAUNCH();
    std::vector<uint64_t> gb(P + 1);
    SR_CUDA(cudaMemcpyAsync(gb.data(), d_gb.p, (P + 1) * 8, cudaMemcpyDeviceToHost, s));
    DevBuf<uint32_t> bstage(st[P]);
    DevBuf<unsigned> pmax(P);
    SR_CUDA(cudaMemsetAsync(pmax.p, 0, P * sizeof(unsigned), s));
    stage_off_kernel<<<grid_for(n + 1), kNT, 0, s>>>(gboff.p, d_vb, d_st, P, n, bstage.p, pmax.p);
    SR_LAUNCH();
    SR_CUDA(cudaStreamSynchronize(s));
    uint64_t pk_off = 0;
    for (uint32_t p = 0; p < P; ++p) {
        PageMeta& pm = g->pages[p];
        pm.pk_data = gb[p + 1] - gb[p];
        SR_CHECK(pm.pk_data < 0xFFFFFFFFull, SERAPH_EOVERFLOW, "a packed page holds 2^32 or more bytes");
        pm.pk_off = pk_off;
        pm.pk_bytes = 2 * pm.off_bytes + align_up(pm.pk_data, 16);
        pk_off += pm.pk_bytes;
    }
    g->h_pack.alloc(pk_off);
    for (uint32_t p = 0; p < P; ++p) {
        const PageMeta& pm = g->pages[p];
        uint8_t* h = g->h_pack.p + pm.pk_off;
        const uint64_t ob = 4 * (pm.nv + 1);
        SR_CUDA(cudaMemcpyAsync(h, stage.p + st[p], ob, cudaMemcpyDeviceToHost, s));
        std::memset(h + ob, 0, pm.off_bytes - ob);
        SR_CUDA(cudaMemcpyAsync(h + pm.off_bytes, bstage.p + st[p], ob, cudaMemcpyDeviceToHost, s));
        std::memset(h + pm.off_bytes + ob, 0, pm.off_bytes - ob);
        uint8_t* hd = h + 2 * pm.off_bytes;
        if (pm.pk_data)
            SR_CUDA(cudaMemcpyAsync(hd, g->d_pack_tmp.p + gb[p], pm.pk_data, cudaMemcpyDeviceToHost, s));
        std::memset(hd + pm.pk_data, 0, align_up(pm.pk_data, 16) - pm.pk_data);
    }
    SR_CUDA(cudaStreamSynchronize(s));
    g->d_pack_tmp.release();
    build_stream_headers(g);
    g->packed = true;
}

void build_graph(seraph_graph* g, uint64_t n, uint64_t m, const uint32_t* src_in,
                 const uint32_t* dst_in, const uint32_t* w_in, int mem, uint32_t flags,
                 uint32_t P, cudaStream_t s) {
    SR_CHECK(n >= 1 && n <= 0xFFFFFFFEull, SERAPH_EINVAL, "n must be in [1, 2^32-2]");
    SR_CHECK(P >= 1 && P <= (1u << 20), SERAPH_EINVAL, "num_pages must be in [1, 2^20]");
    SR_CHECK(mem == SERAPH_MEM_HOST || mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad mem kind");
    SR_CHECK(m == 0 || (src_in && dst_in), SERAPH_EINVAL, "src/dst must not be NULL");
    SR_CHECK(m < (1ull << 36), SERAPH_EINVAL, "too many edges");
    SR_CHECK((flags & ~(SERAPH_SYMMETRIZE | SERAPH_REORDER | SERAPH_COMPRESS | SERAPH_OUT_EDGES)) == 0,
             SERAPH_EINVAL,
             "unknown flag");
    const bool sym = flags & SERAPH_SYMMETRIZE;
    const bool reorder = flags & SERAPH_REORDER;
    const bool weighted = w_in != nullptr;
    SR_CUDA(cudaGetDevice(&g->device));
    g->reordered = reorder;
    g->n = n;
    g->m_raw = sym ? 2 * m : m;
    g->num_pages = P;
    g->weighted = weighted;
    g->symmetrized = sym;

    Adjacency A;
    sorted_adjacency(n, m, src_in, dst_in, w_in, mem, sym, s, A, reorder ? &g->d_perm : nullptr,
                     reorder ? &g->d_inv : nullptr);
    const uint64_t E = A.E;
    g->m = E;
    g->wbytes = A.wbytes;
    DevBuf<uint32_t>& col = A.col;
    const uint8_t* wsrc = A.wptr();
    DevBuf<uint64_t>& col_off = A.off;
    g->d_zero_in.alloc((n + 31) / 32);
    zero_in_kernel<<<grid_for((n + 31) / 32), kNT, 0, s>>>(col_off.p, n, g->d_zero_in.p);
    SR_LAUNCH();
    g->d_outdeg.alloc(n);
    SR_CUDA(cudaMemsetAsync(g->d_outdeg.p, 0, n * sizeof(uint32_t), s));
    if (E) {
        outdeg_kernel<<<grid_for(E), kNT, 0, s>>>(col.p, E, g->d_outdeg.p);
        SR_LAUNCH();
    }
    {
        DevBuf<unsigned> mx(1);
        SR_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned), s));
        max_indeg_kernel<<<grid_for(n), kNT, 0, s>>>(col_off.p, n, mx.p);
        SR_LAUNCH();
        SR_CUDA(cudaMemcpyAsync(&g->max_in_degree, mx.p, 4, cudaMemcpyDeviceToHost, s));
    }

    // page cut
    DevBuf<uint64_t> d_vb(P + 1), d_eb(P + 1);
    page_cut_kernel<<<grid_for(P + 1), kNT, 0, s>>>(col_off.p, n, P, d_vb.p);
    gather_off_kernel<<<grid_for(P + 1), kNT, 0, s>>>(col_off.p, d_vb.p, P, d_eb.p);
    SR_LAUNCH();
    // source blocks of 32-multiple sizes: 32 consecutive ids share a block
    g->src_block = (uint32_t)align_up((n + 32 * kPageBlockWords - 1) / (32 * kPageBlockWords), 32);
    g->d_page_blocks.alloc((uint64_t)P * kPageBlockWords);
    page_blocks_kernel<<<P, kNT, 0, s>>>(col.p, d_eb.p, g->src_block, g->d_page_blocks.p);
    SR_LAUNCH();
    g->vb.resize(P + 1);
    std::vector<uint64_t> eb(P + 1);
    SR_CUDA(cudaMemcpyAsync(g->vb.data(), d_vb.p, (P + 1) * 8, cudaMemcpyDeviceToHost, s));
    SR_CUDA(cudaMemcpyAsync(eb.data(), d_eb.p, (P + 1) * 8, cudaMemcpyDeviceToHost, s));
    SR_CUDA(cudaStreamSynchronize(s));

    g->pages.resize(P);
    std::vector<uint64_t> st(P + 1);
    uint64_t s_off = 0, w_off = 0, stage_n = 0;
    for (uint32_t p = 0; p < P; ++p) {
        PageMeta& pm = g->pages[p];
        pm.vb = g->vb[p];
        pm.nv = g->vb[p + 1] - g->vb[p];
        pm.e0 = eb[p];
        pm.ne = eb[p + 1] - eb[p];
        SR_CHECK(pm.ne < 0xFFFFFFFFull, SERAPH_EOVERFLOW, "a page holds 2^32 or more edges");
        pm.off_bytes = align_up(4 * (pm.nv + 1), 16);
        pm.s_bytes = pm.off_bytes + align_up(4 * pm.ne, 16);
        pm.w_bytes = weighted ? align_up((uint64_t)g->wbytes * pm.ne, 16) : 0;
        pm.s_off = s_off;
        pm.w_off = w_off;
        s_off += pm.s_bytes;
        w_off += pm.w_bytes;
        st[p] = stage_n;
        stage_n += pm.nv + 1;
    }
    st[P] = stage_n;
    g->d_vb.alloc(P + 1);
    {
        std::vector<uint32_t> vb32(P + 1);
        for (uint32_t p = 0; p <= P; ++p) vb32[p] = (uint32_t)g->vb[p];
        SR_CUDA(cudaMemcpyAsync(g->d_vb.p, vb32.data(), (P + 1) * 4, cudaMemcpyHostToDevice, s));
        SR_CUDA(cudaStreamSynchronize(s));
    }

    DevBuf<uint64_t> d_st(P + 1);
    DevBuf<uint32_t> stage(stage_n);
    DevBuf<unsigned> pmax(P);
    SR_CUDA(cudaMemcpyAsync(d_st.p, st.data(), (P + 1) * 8, cudaMemcpyHostToDevice, s));
    SR_CUDA(cudaMemsetAsync(pmax.p, 0, P * sizeof(unsigned), s));
    stage_off_kernel<<<grid_for(n + 1), kNT, 0, s>>>(col_off.p, d_vb.p, d_st.p, P, n, stage.p, pmax.p);
    SR_LAUNCH();
    {
        std::vector<unsigned> hmax(P);
        SR_CUDA(cudaMemcpyAsync(hmax.data(), pmax.p, P * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        for (uint32_t p = 0; p < P; ++p) g->pages[p].maxdeg = hmax[p];
    }

    g->h_struct.alloc(s_off);
    if (weighted) g->h_weight.alloc(w_off);
    for (uint32_t p = 0; p < P; ++p) {
        const PageMeta& pm = g->pages[p];
        uint8_t* hs = g->h_struct.p + pm.s_off;
        SR_CUDA(cudaMemcpyAsync(hs, stage.p + st[p], 4 * (pm.nv + 1), cudaMemcpyDeviceToHost, s));
        std::memset(hs + 4 * (pm.nv + 1), 0, pm.off_bytes - 4 * (pm.nv + 1));
        if (pm.ne)
            SR_CUDA(cudaMemcpyAsync(hs + pm.off_bytes, col.p + pm.e0, 4 * pm.ne,
                                    cudaMemcpyDeviceToHost, s));
        std::memset(hs + pm.off_bytes + 4 * pm.ne, 0, pm.s_bytes - pm.off_bytes - 4 * pm.ne);
        if (weighted) {
            uint8_t* hw = g->h_weight.p + pm.w_off;
            const uint64_t nb = (uint64_t)g->wbytes * pm.ne;
            if (pm.ne)
                SR_CUDA(cudaMemcpyAsync(hw, wsrc + (uint64_t)g->wbytes * pm.e0, nb,
                                        cudaMemcpyDeviceToHost, s));
            std::memset(hw + nb, 0, pm.w_bytes - nb);
        }
    }
    SR_CUDA(cudaStreamSynchronize(s));
    if (flags & SERAPH_COMPRESS) build_packed(g, n, E, col.p, col_off.p, d_vb.p, d_st.p, st, stage, s);
    if (flags & SERAPH_OUT_EDGES) {
        stage.release();
        build_out_edges(g, n, E, col, col_off, wsrc, weighted, s);
    }
}

void check_csr_offsets_host(uint64_t n, const uint64_t* row_off) {
    SR_CHECK(n >= 1 && n <= 0xFFFFFFFEull, SERAPH_EINVAL, "n must be in [1, 2^32-2]");
    SR_CHECK(row_off != nullptr, SERAPH_EINVAL, "row_off must not be NULL");
    SR_CHECK(row_off[0] == 0, SERAPH_EINVAL, "row_off[0] must be 0");
    for (uint64_t v = 0; v < n; ++v)
        SR_CHECK(row_off[v] <= row_off[v + 1], SERAPH_EINVAL,
                 "row_off must be non-decreasing (row_off[" + std::to_string(v) + "] > row_off[" +
                     std::to_string(v + 1) + "])");
}

void build_graph_csr(seraph_graph* g, uint64_t n, const uint64_t* row_off_in, const uint32_t* col_in,
                     const uint32_t* w_in, int mem, uint32_t flags, uint32_t P, cudaStream_t s) {
    SR_CHECK(n >= 1 && n <= 0xFFFFFFFEull, SERAPH_EINVAL, "n must be in [1, 2^32-2]");
    SR_CHECK(row_off_in != nullptr, SERAPH_EINVAL, "row_off must not be NULL");
    SR_CHECK(mem == SERAPH_MEM_HOST || mem == SERAPH_MEM_DEVICE, SERAPH_EINVAL, "bad mem kind");
    uint64_t m = 0;
    if (mem == SERAPH_MEM_DEVICE) {
        DevBuf<unsigned> bad(1);
        SR_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
        check_csr_kernel<<<grid_for(n), kNT, 0, s>>>(row_off_in, n, bad.p);
        SR_LAUNCH();
        unsigned nbad = 0;
        SR_CUDA(cudaMemcpyAsync(&nbad, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaMemcpyAsync(&m, row_off_in + n, 8, cudaMemcpyDeviceToHost, s));
        SR_CUDA(cudaStreamSynchronize(s));
        SR_CHECK(nbad == 0, SERAPH_EINVAL, "row_off must start at 0 and be non-decreasing");
    } else {
        check_csr_offsets_host(n, row_off_in);
        m = row_off_in[n];
    }
    DevBuf<uint64_t> hro;
    DevBuf<uint32_t> hc, hw;
    const uint64_t* row_off = to_device(row_off_in, n + 1, mem, hro, s);
    const uint32_t* col = to_device(col_in, m, mem, hc, s);
    const uint32_t* w = to_device(w_in, m, mem, hw, s);
    DevBuf<uint32_t> src(std::max<uint64_t>(m, 1));
    if (m) {
        expand_csr_kernel<<<grid_for(m), kNT, 0, s>>>(row_off, n, src.p);
        SR_LAUNCH();
    }
    SR_CUDA(cudaStreamSynchronize(s));
    build_graph(g, n, m, src.p, col, w, SERAPH_MEM_DEVICE, flags, P, s);
}

void export_csc(const seraph_graph* g, uint64_t* col_off, uint32_t* row, uint32_t* w,
                uint32_t* out_degree) {
    for (uint32_t p = 0; p < g->num_pages; ++p) {
        const PageMeta& pm = g->pages[p];
        const uint32_t* off = (const uint32_t*)(g->h_struct.p + pm.s_off);
        const uint32_t* c = (const uint32_t*)(g->h_struct.p + pm.s_off + pm.off_bytes);
        if (col_off)
            for (uint64_t i = 0; i < pm.nv; ++i) col_off[pm.vb + i] = pm.e0 + off[i];
        if (row && pm.ne) std::memcpy(row + pm.e0, c, 4 * pm.ne);
        if (w && g->weighted && pm.ne) {
            const uint8_t* hw = g->h_weight.p + pm.w_off;
            for (uint64_t i = 0; i < pm.ne; ++i) {
                uint32_t x = 0;
                std::memcpy(&x, hw + i * g->wbytes, g->wbytes);  // little-endian widths
                w[pm.e0 + i] = x;
            }
        }
    }
    if (col_off) col_off[g->n] = g->m;
    if (out_degree) {
        SR_CUDA(cudaMemcpy(out_degree, g->d_outdeg.p, g->n * 4, cudaMemcpyDeviceToHost));
    }
}

}  // namespace seraph
