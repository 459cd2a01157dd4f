// Device helpers shared by the relax kernels and the page rebuild of
// compact-streamed chunks: L2 eviction policies, streaming loads, and the
// piece-parallel LEB128 decode of the packed page form (SERAPH_COMPRESS).
#pragma once

#include "common.cuh"

namespace seraph {
namespace {

// L2 eviction-priority policies (createpolicy, sm_80+).  Page data of the
// resident chunk is read once per pass (evict-first); the gathered values of
// the lowest-numbered `hot` vertices -- the most-read ones once vertices are
// numbered by out-degree -- are kept (evict-last).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Streaming loads of the resident chunk (read-only while a pass runs; not
// kept in L1).  Not volatile: the compiler may batch them for more loads in
// flight.
__device__ __forceinline__ uint4 ld_stream4(const void* p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ uint2 ld_stream2(const void* p, uint64_t pol) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
        : "=r"(r.x), "=r"(r.y)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ uint32_t ld_stream(const void* p, uint64_t pol) {
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

// ----------------------------------------------------------- packed pages
// A destination's sources are its first id, then each gap to the next id
// minus one, as LEB128 codes (SERAPH_COMPRESS).  Lanes take aligned 16-byte
// pieces of the code bytes and decode the codes that start in their piece:
// a byte starts a code when the byte before it ends one (high bit clear).
// The ids follow from a running sum, across pieces by a scan of the per-piece
// (count, sum of value + 1) pairs.

// Bit i (0..3) set: byte i of w ends a code.
__device__ __forceinline__ uint32_t leb_ends4(uint32_t w) {
    // the four flag bits (7, 15, 23, 31) gathered into bits 28..31 by one
    // multiply: the other partial products land on distinct bits below 24
    return ((~w & 0x80808080u) * 0x00204081u) >> 28;
}

// Bits of the 16 bytes at c that start a code of the range [B, Eb); pt = the
// byte before c ends a code (or c is the range's first piece).
__device__ __forceinline__ uint32_t leb_starts(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                               uint32_t pt, uint32_t c, uint32_t B, uint32_t Eb) {
    const uint32_t T = leb_ends4(w0) | (leb_ends4(w1) << 4) | (leb_ends4(w2) << 8) |
                       (leb_ends4(w3) << 12);
    const uint32_t lo = B > c ? B - c : 0u;                  // < 16
    const uint32_t hi = Eb - c < 16u ? Eb - c : 16u;         // c < Eb
    const uint32_t rng = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
    return ((T << 1) | pt) & rng;
}

// One aligned 16-byte piece of a code range: the piece, the 4 bytes after it
// (when still inside the range) and whether the byte before it ends a code.
struct Piece {
    uint32_t w0, w1, w2, w3, w4, pt;
};

// The 7-bit groups of 4 code bytes packed into 28 bits.
__device__ __forceinline__ uint32_t leb_payload4(uint32_t w) {
    const uint32_t t = (w & 0x007F007Fu) | ((w & 0x7F007F00u) >> 1);  // byte pairs -> 14 bits
    return (t & 0x3FFFu) | ((t >> 2) & 0xFFFC000u);
}

// Every code start of a piece decoded at once.  The 7-bit groups of the 20
// window bytes are packed into one bit stream (byte j's group at bit 7j) and
// their end flags into a second one (a code's last byte flags bit 7j + 6), so
// the code starting at byte j is x & (e ^ (e - 1)) with x, e the 32 bits of
// the two streams from bit 7j: the mask keeps everything up to the first end
// flag (all 32 bits for a 5-byte code, whose value fits them exactly).  The
// byte positions are compile-time constants once unrolled.  lid[j] = sum of
// (value + 1) over the codes starting at or before byte j, i.e. the id of the
// code at j relative to the id before the piece.  Returns the piece's total.
__device__ __forceinline__ uint32_t piece_decode(const Piece& P, uint32_t st, uint32_t lid[16]) {
    const uint32_t w[5] = {P.w0, P.w1, P.w2, P.w3, P.w4};
    uint32_t p[5], q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        p[k] = leb_payload4(w[k]);
        // end flags of the 4 bytes spread to bits 6, 13, 20, 27 (the product
        // terms of distinct bits land on distinct bits: no carries)
        q[k] = (leb_ends4(w[k]) * 0x01041040u) & 0x08102040u;
    }
    const uint32_t sw[6] = {p[0] | (p[1] << 28), (p[1] >> 4) | (p[2] << 24), (p[2] >> 8) | (p[3] << 20),
                            (p[3] >> 12) | (p[4] << 16), p[4] >> 16, 0u};
    const uint32_t se[6] = {q[0] | (q[1] << 28), (q[1] >> 4) | (q[2] << 24), (q[2] >> 8) | (q[3] << 20),
                            (q[3] >> 12) | (q[4] << 16), q[4] >> 16, 0u};
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int o = 7 * j;
        const uint32_t x = __funnelshift_r(sw[o >> 5], sw[(o >> 5) + 1], o & 31);
        const uint32_t e = __funnelshift_r(se[o >> 5], se[(o >> 5) + 1], o & 31);
        const uint32_t v = x & (e ^ (e - 1u));
        acc += ((st >> j) & 1u) ? v + 1u : 0u;
        lid[j] = acc;
    }
    return acc;
}

__device__ __forceinline__ Piece load_piece(const uint8_t* d, uint32_t c, uint32_t A, uint32_t Eb,
                                            uint64_t pol) {
    Piece P;
    const uint4 q = ld_stream4(d + c, pol);
    P.w0 = q.x; P.w1 = q.y; P.w2 = q.z; P.w3 = q.w;
    P.w4 = c + 16u < Eb ? ld_stream(d + c + 16u, pol) : 0u;
    P.pt = c == A ? 1u : ((ld_stream(d + c - 4u, pol) >> 31) ^ 1u);
    return P;
}

}  // namespace
}  // namespace seraph
