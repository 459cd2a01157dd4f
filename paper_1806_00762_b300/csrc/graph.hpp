// Internal graph object: the paged CSC of Sec. 3.1 held in pinned host memory,
// plus the vertex-side arrays that stay resident on the device.
#pragma once

#include <mutex>
#include <vector>

#include "common.cuh"

// Device buffers of a run kept with the graph for the next run (a serving
// loop then allocates nothing after its first call).  Held by one run at a
// time; a concurrent run on the same graph allocates its own.
struct RunWorkspace {
    std::mutex m;
    seraph::DevBuf<uint8_t> ebuf;                // the edge ring
    seraph::DevBuf<unsigned long long> lists;    // compaction lists
    seraph::DevBuf<uint32_t> val, out;           // values; caller-order output staging
    seraph::DevBuf<float> x, contrib, x_next, x_prev, inv_out;
    seraph::DevBuf<uint8_t> state;
    seraph::DevBuf<uint32_t> stamp, front0, front1, big;  // push stage
    seraph::DevBuf<uint8_t> small;               // a run's small device buffers, carved
    seraph::PinnedBuf small_h;                   // its small pinned read-back buffers
    void release() {
        ebuf.release(); lists.release(); val.release(); out.release(); x.release();
        contrib.release(); x_next.release(); x_prev.release(); inv_out.release(); state.release();
        stamp.release(); front0.release(); front1.release(); big.release();
        small.release(); small_h.release();
    }
};

// Static per-page description.  A page is a contiguous destination range
// [vb, vb+nv) with all of its in-edges.  In the pinned structure region it is
//   u32 off[nv+1] (relative to the page's first edge), padded to 16 B,
//   u32 col[ne] (source ids, ascending per destination), padded to 16 B;
// its weights (if any) sit at w_off in the separate weight region.
struct PageMeta {
    uint64_t vb;        // first vertex
    uint64_t nv;        // vertices
    uint64_t ne;        // in-edges
    uint64_t e0;        // global index of the first in-edge
    uint64_t s_off;     // byte offset of the page in the structure region
    uint64_t s_bytes;   // structure bytes (offsets + columns, padded)
    uint64_t off_bytes; // bytes of the padded offset array
    uint64_t w_off;     // byte offset in the weight region
    uint64_t w_bytes;   // weight bytes (ne * weight width, padded), 0 if unweighted
    uint32_t maxdeg;    // largest in-degree in the page
    // Packed structure (SERAPH_COMPRESS), in its own region:
    //   u32 off[nv+1] as above, padded to 16 B,
    //   u32 boff[nv+1] byte offsets into the page's gap stream, padded to 16 B,
    //   the gap stream: per destination, its first source id and then each
    //   gap to the next source minus one, LEB128 (7 bits per byte, low group
    //   first, high bit set on every byte but a value's last), padded to 16 B.
    uint64_t pk_off;    // byte offset of the page in the packed region
    uint64_t pk_bytes;  // packed structure bytes (padded)
    uint64_t pk_data;   // gap-stream bytes (unpadded)
    // Streamed header of the packed page (SERAPH_COMPRESS), in its own region,
    // sent ahead of the page's gap stream when a plain page streams compact:
    //   uint4 ckpt[T+1], T = ceil(nv / kStreamTile): (off, boff, escapes
    //     before, vertices with an in-edge before) at vertex t * kStreamTile,
    //     and (ne, gap-stream bytes, nesc, nnz) at the end;
    //   u32 bits[T][8]: bit i of a tile set when its vertex i has an in-edge;
    //   u16 hdr[nnz]: for each vertex with an in-edge, in order, in-degree |
    //     code bytes << 8 when both are at most 254, else 0xFFFF and the two
    //     counts are the vertex's escape entry;
    //   uint2 esc[nesc]: (in-degree, code bytes) of the escaped vertices in
    //     vertex order;
    // hdr and esc each padded to 16 B.
    uint64_t sh_off;    // byte offset of the header in the header region
    uint64_t sh_bytes;  // header bytes (multiple of 16)
    uint32_t sh_nesc;   // escaped vertices
    uint32_t sh_nnz;    // vertices with an in-edge
};


struct seraph_graph {
    int device = 0;
    uint64_t n = 0, m_raw = 0, m = 0;
    uint32_t num_pages = 0;
    bool weighted = false, symmetrized = false;
    uint32_t max_in_degree = 0;
    uint32_t wbytes = 4;               // stored weight width (1, 2 or 4 bytes)
    std::vector<PageMeta> pages;
    std::vector<uint64_t> vb;          // num_pages + 1 page boundaries
    seraph::PinnedBuf h_struct;        // all page structures, in page order
    seraph::PinnedBuf h_weight;        // all page weights, in page order
    seraph::DevBuf<uint32_t> d_outdeg; // out-degree per vertex (PageRank)
    seraph::DevBuf<uint32_t> d_vb;     // page boundaries (u32) on the device
    seraph::DevBuf<uint32_t> d_zero_in; // bit v set: v has no in-edge
    bool packed = false;               // built with SERAPH_COMPRESS
    seraph::PinnedBuf h_pack;          // all packed page structures, in page order
    seraph::PinnedBuf h_shdr;          // streamed headers of the packed pages, in page order
    seraph::DevBuf<uint8_t> d_pack_tmp; // gap streams while the graph is built
    RunWorkspace ws;                   // buffers kept between runs
    bool reordered = false;            // built with SERAPH_REORDER
    seraph::DevBuf<uint32_t> d_perm;   // internal id -> caller's id (reordered only)
    seraph::DevBuf<uint32_t> d_inv;    // caller's id -> internal id (reordered only)
    // Out-edge CSR of the kept edges in internal ids (SERAPH_OUT_EDGES), in
    // pinned memory that kernels read directly over the host link (the push
    // stage of sparse sweeps): u64 offsets (n+1), u32 destinations ascending
    // per source, weights in the stored width.
    bool out_edges = false;
    seraph::PinnedBuf h_out_off, h_out_col, h_out_w;
    // Which source blocks each page reads: bit b of page p's kPageBlockWords
    // words is set when some in-edge of p comes from a vertex of block b
    // (blocks of src_block consecutive internal ids).  Measures how many
    // pages a change leaves untouched (active-page skipping).
    seraph::DevBuf<uint32_t> d_page_blocks;
    uint32_t src_block = 0;
};

namespace seraph {
constexpr uint32_t kPageBlockWords = 32;  // 1024 source blocks
}

namespace seraph {
struct Adjacency;
}

namespace seraph {
struct Adjacency {
    uint64_t E = 0;
    uint32_t wbytes = 4;
    DevBuf<uint64_t> off;   // n+1 row offsets
    DevBuf<uint32_t> col;   // other endpoint, ascending within a row
    DevBuf<uint32_t> wcol;  // weights if stored 4 bytes wide
    DevBuf<uint8_t> wnar;   // weights if narrowed to 1 or 2 bytes
    const uint8_t* wptr() const { return wbytes < 4 ? wnar.p : (const uint8_t*)wcol.p; }
};
// perm/inv non-null: renumber vertices by non-increasing count in `lo`
// (SERAPH_REORDER), perm = new -> old, inv = old -> new.
void sorted_adjacency(uint64_t n, uint64_t m, const uint32_t* lo, const uint32_t* hi,
                      const uint32_t* w, int mem, bool sym, cudaStream_t s, Adjacency& A,
                      DevBuf<uint32_t>* perm = nullptr, DevBuf<uint32_t>* inv = nullptr);
void build_graph(seraph_graph* g, uint64_t n, uint64_t m, const uint32_t* src,
                 const uint32_t* dst, const uint32_t* w, int mem, uint32_t flags,
                 uint32_t num_pages, cudaStream_t s);
void build_graph_csr(seraph_graph* g, uint64_t n, const uint64_t* row_off, const uint32_t* col,
                     const uint32_t* w, int mem, uint32_t flags, uint32_t num_pages,
                     cudaStream_t s);
// CSR offsets in host memory: n in range, row_off[0] == 0, non-decreasing
// (SERAPH_EINVAL otherwise).  Touches no device.
void check_csr_offsets_host(uint64_t n, const uint64_t* row_off);
void export_csc(const seraph_graph* g, uint64_t* col_off, uint32_t* row, uint32_t* w,
                uint32_t* out_degree);
}  // namespace seraph

// Device-resident out-edge CSR for batched queries (batch.cu).
struct seraph_bgraph {
    int device = 0;
    uint64_t n = 0, m_raw = 0;
    bool weighted = false;
    seraph::Adjacency adj;        // rows = sources
    seraph::Adjacency in_adj;     // rows = destinations (bottom-up BFS rounds), no weights
    int tuned_mapping = 0;        // 0: not tuned yet
    uint32_t tuned_tile = 0;
    uint32_t tuned_delta = 0;     // SSSP near-far width chosen with the mapping (0: none)
};
