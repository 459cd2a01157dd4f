// Rebuild of compact-streamed pages (seraph_params.stream_packed): a chunk
// that is processed in the plain form crosses the host link as, per page, a
// header of two bytes per vertex with offset checkpoints (layout in
// common.cuh) and the page's LEB128 gap stream, and is rebuilt here into its
// plain form (u32 offsets, u32 source ids) inside the ring slot.  A transfer
// encoding of the paper's CSC pages (Sec. 3.1): results are unchanged.
#include <algorithm>

#include "engine.cuh"
#include "leb128.cuh"

namespace seraph {
namespace {

constexpr int kNT = 256;

// The ids of a decoded piece are written out instead of gathered: the code
// at byte j has id run + lid[j] and edge index ord + (codes before j).
__device__ __forceinline__ void piece_write(uint32_t* col, uint32_t st, const uint32_t lid[16],
                                            uint32_t run, uint32_t ord, uint32_t ne) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const uint32_t i = ord + __popc(st & ((1u << j) - 1u));
        if (((st >> j) & 1u) && i < ne) col[i] = run + lid[j];
    }
}

// Decodes the code bytes [B, Eb) of each lane's vertex (when `valid`) into
// col from edge index e0: a vertex of at most 64 code bytes by its own lane,
// longer ones by the whole warp (pieces t, t+32, ... and a warp scan).
// Called by whole warps.
__device__ __forceinline__ void decode_warp(const uint8_t* d, uint32_t* col, uint32_t ne, bool valid,
                                            uint32_t B, uint32_t Eb, uint32_t e0, uint64_t pol) {
    const uint32_t lane = lane_id();
    const bool big = valid && Eb - B > 64u;
    if (valid && !big) {
        const uint32_t A = B & ~15u;
        uint32_t run = 0xFFFFFFFFu, ord = e0;
        for (uint32_t c = A; c < Eb; c += 16) {
            const Piece P = load_piece(d, c, A, Eb, pol);
            const uint32_t st = leb_starts(P.w0, P.w1, P.w2, P.w3, P.pt, c, B, Eb);
            uint32_t lid[16];
            const uint32_t sum = piece_decode(P, st, lid);
            piece_write(col, st, lid, run, ord, ne);
            run += sum;
            ord += __popc(st);
        }
    }
    for (unsigned m = __ballot_sync(kFull, big); m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const uint32_t Bj = __shfl_sync(kFull, B, j), Ej = __shfl_sync(kFull, Eb, j);
        const uint32_t ej = __shfl_sync(kFull, e0, j);
        const uint32_t A = Bj & ~15u;
        const uint32_t pieces = (Ej - A + 15u) >> 4;
        uint32_t run = 0xFFFFFFFFu, ord = ej;
        for (uint32_t it = 0; it < (pieces + 31) / 32; ++it) {
            const uint32_t c = A + 16u * (it * 32 + lane);
            Piece P{0u, 0u, 0u, 0u, 0u, 0u};
            uint32_t st = 0;
            if (c < Ej) {
                P = load_piece(d, c, A, Ej, pol);
                st = leb_starts(P.w0, P.w1, P.w2, P.w3, P.pt, c, Bj, Ej);
            }
            uint32_t lid[16];
            const uint64_t x = ((uint64_t)__popc(st) << 32) | piece_decode(P, st, lid);
            uint64_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(kFull, inc, o);
                if (lane >= (uint32_t)o) inc += y;
            }
            const uint64_t ex = inc - x;
            const uint64_t tot = __shfl_sync(kFull, inc, 31);
            if (st) piece_write(col, st, lid, run + (uint32_t)ex, ord + (uint32_t)(ex >> 32), ne);
            run += (uint32_t)tot;
            ord += (uint32_t)(tot >> 32);
        }
    }
}

// One page streamed compact: `in` = its header (checkpoints, per-vertex
// in-degree and code bytes, escapes; layout in common.cuh) followed by its
// gap stream; `out` = its plain form (off, col with zero padding, s_bytes in
// all).  The regions must not overlap.  A CTA takes a tile of kStreamTile
// vertices, one per thread: a vertex with an in-edge finds its header entry
// by a count of the tile's set bits before it, an escaped vertex its escape
// entry by a count of the escapes before it, a block scan of (in-degree, code bytes)
// from the tile's checkpoint gives each vertex's edge and byte offsets, and
// each warp then decodes its 32 vertices.  Offsets are clamped to the page's
// totals, so a damaged header cannot move a read or a write off the page.
__global__ void __launch_bounds__(kNT) decode_page_kernel(const uint8_t* __restrict__ in,
                                                          uint8_t* __restrict__ out, uint32_t nv,
                                                          uint32_t nesc, uint64_t off_bytes,
                                                          uint64_t s_bytes) {
    static_assert(kStreamTile == kNT, "one vertex per thread");
    __shared__ unsigned long long ws[kNT / 32 + 1];
    __shared__ unsigned s_esc[kNT / 32];
    const uint4* ck = (const uint4*)in;
    const uint32_t T = (nv + kStreamTile - 1) / kStreamTile;
    const uint4 last = ck[T];
    const uint32_t nnz = last.w;
    const uint64_t ckb = stream_ckpt_bytes(nv), bb = stream_bitmap_bytes(nv), hb = stream_hdr_bytes(nnz);
    const uint32_t* bits = (const uint32_t*)(in + ckb);
    const uint16_t* hdr = (const uint16_t*)(in + ckb + bb);
    const uint2* esc = (const uint2*)(in + ckb + bb + hb);
    const uint8_t* d = in + ckb + bb + hb + stream_esc_bytes(nesc);
    uint32_t* ooff = (uint32_t*)out;
    uint32_t* col = (uint32_t*)(out + off_bytes);
    const uint32_t ne = min(last.x, (uint32_t)((s_bytes - off_bytes) / 4)), nb = last.y;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    // the last offset and the zero padding of both arrays (a padding column
    // may be gathered, so it must be a valid vertex id)
    for (uint64_t i = (uint64_t)nv + tid; i < off_bytes / 4; i += stride) ooff[i] = i == nv ? ne : 0u;
    for (uint64_t i = (uint64_t)ne + tid; i < (s_bytes - off_bytes) / 4; i += stride) col[i] = 0u;
    const uint64_t pol = policy_evict_first();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint4 c0 = ck[t];
        const uint32_t v = t * kStreamTile + threadIdx.x;
        const bool valid = v < nv;
        // this vertex's header entry: the tile's set bits before it
        const uint32_t* tb = bits + 8 * (uint64_t)t;
        const uint32_t word = tb[warp];
        uint32_t hi = c0.w + __popc(word & lanemask_lt());
        for (uint32_t w = 0; w < warp; ++w) hi += __popc(tb[w]);
        const uint32_t h = valid && ((word >> lane) & 1u) && hi < nnz ? hdr[hi] : 0u;
        const bool x = h == 0xFFFFu;
        const unsigned m = __ballot_sync(kFull, x);
        if (lane == 0) s_esc[warp] = __popc(m);
        __syncthreads();
        uint32_t k = c0.z + __popc(m & lanemask_lt());
        for (uint32_t w = 0; w < warp; ++w) k += s_esc[w];
        uint32_t deg = h & 0xFFu, len = h >> 8;
        if (x) {
            const uint2 e = k < nesc ? esc[k] : make_uint2(0u, 0u);
            deg = e.x;
            len = e.y;
        }
        unsigned long long tot;
        const unsigned long long ex =
            block_excl_scan<kNT>(((unsigned long long)deg << 32) | len, ws, &tot);
        const uint32_t e0 = min(c0.x + (uint32_t)(ex >> 32), ne);
        const uint32_t B = min(c0.y + (uint32_t)ex, nb), Eb = min(B + len, nb);
        if (valid) ooff[v] = e0;
        decode_warp(d, col, ne, valid, B, Eb, e0, pol);
    }
}

}  // namespace

void launch_decode_page(const uint8_t* in, uint8_t* out, uint32_t nv, uint32_t nesc,
                        uint64_t off_bytes, uint64_t s_bytes, cudaStream_t s) {
    const uint64_t tiles = ((uint64_t)nv + kStreamTile - 1) / kStreamTile;
    const unsigned g = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(tiles, (uint64_t)device_sms() * 8));
    decode_page_kernel<<<g, kNT, 0, s>>>(in, out, nv, nesc, off_bytes, s_bytes);
    SR_LAUNCH();
}

}  // namespace seraph
