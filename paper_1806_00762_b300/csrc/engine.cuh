// Device-side engine of one local pass (Sec. 3.2 pipelined iteration, Sec. 4
// predictive updating): shared declarations between the kernels (engine.cu)
// and the host sweep driver (run.cu).
#pragma once

#include "common.cuh"

namespace seraph {

constexpr int kMaxWindow = 16;
// In-degree classes of the relax mapping: one thread, 4 lanes, 8 lanes, a
// warp, or a whole CTA per vertex.
constexpr int kClasses = 5;

// Where a resident page's arrays currently live (device addresses in the
// edge ring).  Rewritten whenever the page's chunk is (re)loaded.
struct PageLoc {
    const uint32_t* off;  // nv+1 page-relative offsets
    const uint32_t* col;  // ne source ids (16-byte aligned); packed: the gap stream
    const uint8_t* w;     // ne weights, wbytes each (16-byte aligned) or null
    const uint32_t* boff; // packed: nv+1 byte offsets into the gap stream, else null
    uint32_t vb;          // first vertex
    uint32_t nv;          // vertices
};

struct ChunkDesc {
    uint32_t v_begin, v_end;       // destination range of the chunk
    uint32_t first_page, end_page; // pages [first, end)
    uint32_t block_begin;          // first compaction block of this chunk
    uint32_t pad;
};

struct WindowDesc {
    uint32_t nchunks;
    uint32_t nblocks;              // compaction blocks over all chunks
    ChunkDesc c[kMaxWindow];
};

// Counters of one sweep, copied to the host at the sweep boundary.
struct SweepReport {
    unsigned long long changed, attempted, skipped, edges;
    unsigned long long packed_edges, code_bytes;  // in-edges and LEB128 bytes of attempted
                                                  // vertices on packed pages
    unsigned long long clean_pages;  // pages with no in-edge source changed in the sweep
    unsigned int overflow, thr_min, passes_run, passes_skipped;
    double resid, dangling;
};

struct RunState {
    SweepReport cur;
    unsigned int pass_go[2];      // pass decision of the gate kernel
    unsigned int loaded;          // sequence number of the last chunk load done
    unsigned int k_limit;         // learned schedule: passes allowed in this step
    unsigned int step_passes;     // passes run in the current step
    unsigned int pad1;
    unsigned long long prev_changed;  // changes of the previous sweep
    unsigned int pass_changed[2];
    unsigned int list_cnt[2][8];
    unsigned int work[2][8];
    unsigned int thr_cur, thr_prev, sweeps_done, err;
    float base;
    float scale;              // PageRank: 1 / sum(x) applied at the sweep close (1 = none)
    double dsum, rsum;
};

enum { ALG_SSSP = 0, ALG_BFS = 1, ALG_CC = 2, ALG_PR = 3 };

// Per-chunk inputs of the learned scheduler's features.
struct ChunkStatic {
    float nv, ne, maxdeg, bytes_frac;  // vertices, in-edges, max in-degree, bytes / slot
};
struct ChunkDyn {
    unsigned visits, last_passes, gains[4];  // visits so far; passes and first 4 pass gains of the last visit
};

struct AlgoArgs {
    uint32_t* val;            // SSSP/BFS/CC values
    float* x;                 // PageRank values
    float* contrib;           // x / outdeg (0 for dangling)
    float* x_next;            // value computed in the current pass
    const float* inv_out;     // 1 / outdeg or 0
    uint8_t* state;           // weak-prediction state per vertex
    RunState* rs;
    const PageLoc* loc;       // per page
    const uint32_t* vb;       // page boundaries (P+1)
    unsigned long long* list[kClasses];  // entries (page << 32) | v, per class
    unsigned int* step_changed;   // value changes per pipeline step (ring)
    uint32_t step_mask;           // ring size - 1
    uint32_t cls_max[4];      // largest in-degree of classes 0..3 (above: class 4)
    float damping, fail_eps;
    uint64_t fsm_bits;        // next state of (state s, changed c) in bits 3(2s+c)..+2
    uint8_t skip_mask;
    uint8_t pvu;              // SERAPH_PVU_*
    uint8_t wbytes;           // stored weight width: 1, 2 or 4 bytes
    uint8_t hints;            // 1: L2 eviction-priority hints on (see hot)
    uint8_t packed;           // pages hold LEB128 gap streams (SERAPH_COMPRESS)
    uint32_t hot;             // gathers of vertices < hot: L2 evict-last
    uint32_t n;               // vertices
    uint32_t bfs_lb;          // BFS: no attempted vertex can reach a level below this, so a
                              // lane that finds it stops scanning (early-break pull)
    float omega;              // PageRank over-relaxation factor of the apply step (1 = plain)
    uint32_t* chg_stamp;      // push stage on: tag of the sweep in which a vertex last
                              // changed (written with every value change), else null
    uint32_t chg_tag;         // tag of the current sweep
};

// Launchers (engine.cu).  `pass` is the global pass counter (its parity picks
// the double-buffered counters).  Every pass starts with a one-thread gate
// that decides on the device whether the pass runs: it is skipped when
// `check_prev` is set and the previous pass of the step changed nothing, or
// when `idle` is set and load number `want_loaded` has already landed (an
// idle-slot pass is only worth running while the copy is in flight).
// `predict` = 0 runs the pass with prediction off.
void launch_gate(RunState* rs, uint32_t pass, int check_prev, int idle, uint32_t want_loaded,
                 uint32_t j, int learned, unsigned* rec_gains, cudaStream_t s);
// After the last pass of a step: record its gain, update the chunk's state.
void launch_step_epilogue(RunState* rs, ChunkDyn* cd, uint32_t chunk, uint32_t last_pass,
                          uint32_t npass, unsigned* rec_gains, cudaStream_t s);
void launch_compact(int algo, const WindowDesc& wd, const AlgoArgs& a, uint32_t pass,
                    int predict, cudaStream_t s);
void launch_relax(int algo, int kahan, const AlgoArgs& a, uint32_t pass, uint32_t step,
                  int grid, cudaStream_t s);
void launch_pr_apply(const AlgoArgs& a, uint32_t pass, int grid, cudaStream_t s);
void launch_set_locs(PageLoc* loc, const uint32_t* vb, uint32_t first, uint32_t end,
                     const uint64_t* rel_soff, const uint64_t* rel_woff, const uint64_t* off_bytes,
                     uint8_t* sbase, uint8_t* wbase, bool packed, RunState* rs, uint32_t seq,
                     cudaStream_t s);
// Rebuild one page streamed compact (its streamed header -- checkpoints,
// per-vertex in-degree and code bytes, nesc escapes -- then its LEB128 gap
// stream, at `in`, 16-byte aligned) into its plain form (off, col with zero
// padding, s_bytes in all, at `out`, 16-byte aligned); the two regions must
// not overlap.
void launch_decode_page(const uint8_t* in, uint8_t* out, uint32_t nv, uint32_t nesc,
                        uint64_t off_bytes, uint64_t s_bytes, cudaStream_t s);
void launch_init_values(int algo, const AlgoArgs& a, uint64_t n, uint32_t source,
                        const uint32_t* label0, cudaStream_t s);
// out[v] = in[inv[v]]: values of a reordered graph back in the caller's ids.
void launch_unpermute(const uint32_t* in, const uint32_t* inv, uint64_t n, uint32_t* out,
                      cudaStream_t s);
void launch_init_pr(const uint32_t* outdeg, const AlgoArgs& a, float* x_prev, uint64_t n,
                    cudaStream_t s);
void launch_close_min(RunState* rs, SweepReport* out, cudaStream_t s);
// Active-page measurement at a sweep close: the source blocks holding a vertex
// whose stamp is `tag` (changed in the closing sweep; `dirty` = 32 words of
// scratch), then rs->cur.clean_pages += the pages whose source-block bitmap
// (32 words per page) misses all of them.
void launch_count_clean(const uint32_t* stamp, uint64_t n, uint32_t tag, uint32_t bsz,
                        const uint32_t* page_blocks, uint32_t P, uint32_t* dirty, RunState* rs,
                        cudaStream_t s);
void launch_close_pr(const AlgoArgs& a, uint64_t n, float* x_prev, double damping,
                     double* partial, int nparts, SweepReport* out, bool normalize,
                     cudaStream_t s);

}  // namespace seraph
