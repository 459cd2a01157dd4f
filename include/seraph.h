/*
 * seraph.h -- C ABI of the B300 streamed-graph engine (Seraph, arXiv 1806.00762).
 *
 * The problem this library solves (Sec. 1, Sec. 2.1, Sec. 3.1): a graph larger
 * than device memory lives in host memory; the GPU processes subgraphs that
 * stream over the host link while all vertex values stay resident in device
 * memory.  Subgraphs are CSC pages: a contiguous range of destination vertices
 * with all of their incoming edges and no destination-index array (Sec. 3.1
 * "Subgraph Organization").  Each resident page is iterated several times
 * while the next one is in flight ("Pipelined Subgraph Iteration", Sec. 3.2,
 * Fig. 4), and vertices predicted to be converged are skipped ("Predictive
 * Vertex Updating", Sec. 4: strong conditions of Table 1, weak state machine
 * of Fig. 6).
 *
 * Conventions for every call:
 *   - Return 0 (SERAPH_OK) or a negative SERAPH_E* code; no exception crosses
 *     the ABI.  seraph_last_error() gives a message for the calling thread.
 *   - Input arrays are caller-owned and only read during the call (they are
 *     copied).  Output buffers are caller-owned.  The library owns the pinned
 *     host pages and every device allocation it makes, and frees them in
 *     seraph_graph_free / at the end of seraph_run.
 *   - `mem` says where a pointer lives: SERAPH_MEM_HOST (pageable or pinned
 *     host memory) or SERAPH_MEM_DEVICE (device memory of the current CUDA
 *     device, e.g. a torch tensor's data_ptr()).
 *   - `stream` is a cudaStream_t (NULL = the library's own stream).  Calls are
 *     synchronous with respect to the host: they return when results are ready.
 *   - Vertex ids are uint32; n <= 2^32 - 2.  0xFFFFFFFF means "unreachable".
 *   - Requires a CUDA device of compute capability 10.3 (B300, sm_103a).
 */
#ifndef SERAPH_H
#define SERAPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define SERAPH_OK         0
#define SERAPH_EINVAL    -1   /* bad argument                                   */
#define SERAPH_ENOMEM    -2   /* host (pinned) or device allocation failed      */
#define SERAPH_EBUDGET   -3   /* a page does not fit a ring slot of the budget  */
#define SERAPH_ECUDA     -4   /* CUDA runtime error (message has the details)   */
#define SERAPH_ETIMEOUT  -5   /* a bounded wait ran out                         */
#define SERAPH_EOVERFLOW -6   /* an SSSP distance does not fit below 2^32-1, or
                                 a page holds 2^32 or more edges                 */
#define SERAPH_ENOTCONV  -7   /* max_sweeps reached before the fixpoint (SSSP,
                                 BFS, CC); PageRank stops at max_sweeps with
                                 SERAPH_OK and stats->converged = 0              */

#define SERAPH_INF 0xFFFFFFFFu

enum seraph_algo { SERAPH_SSSP = 0, SERAPH_BFS = 1, SERAPH_CC = 2, SERAPH_PAGERANK = 3 };
enum seraph_mem  { SERAPH_MEM_HOST = 0, SERAPH_MEM_DEVICE = 1 };
/* Predictive vertex updating (Sec. 4). */
enum seraph_pvu  { SERAPH_PVU_OFF = 0, SERAPH_PVU_STRONG = 1, SERAPH_PVU_WEAK = 2 };
/* Schedule of the local passes (Sec. 3.2). */
enum seraph_sched { SERAPH_SCHED_FIXED = 0, SERAPH_SCHED_LEARNED = 1 };
/* Chunk order across sweeps.  CYCLIC: every sweep streams chunks 0..C-1 and
 * the window wraps from the last chunk to the first.  ZIGZAG: sweeps
 * alternate direction, so the window resident at the end of one sweep opens
 * the next one and is not streamed again (C - window loads per sweep). */
enum seraph_order { SERAPH_ORDER_CYCLIC = 0, SERAPH_ORDER_ZIGZAG = 1 };

/* Graph flags. */
#define SERAPH_SYMMETRIZE 1u  /* add (v,u) for every (u,v): the undirected view
                                 that weakly connected components run on      */
#define SERAPH_REORDER    2u  /* number vertices internally in order of
                                 non-increasing out-degree (ties: ascending
                                 id) before the page cut.  A layout choice,
                                 not in the paper: the gathered source values
                                 of the most-read vertices become one compact
                                 range that stays in L2.  Results, sources and
                                 labels stay in the caller's ids; only the
                                 page contents (export_csc, page_bounds) are
                                 in internal ids (see seraph_graph_export_perm) */
#define SERAPH_COMPRESS   4u  /* also keep every page in a packed form: per
                                 destination its first source id, then each
                                 gap to the next source minus one, as LEB128
                                 bytes (7 bits per byte, low group first, high
                                 bit set on all but a value's last byte), with
                                 u32 page-relative byte offsets per vertex
                                 beside the u32 edge offsets.  A lossless
                                 encoding of the compact page of Sec. 3.1 that
                                 streams ~2 bytes per edge instead of 4; runs
                                 pick the form with seraph_params.columns    */

#define SERAPH_OUT_EDGES  8u  /* also keep the kept edges as an out-edge CSR in
                                 pinned host memory (u64 offsets per source,
                                 u32 destinations ascending, weights in the
                                 stored width), read directly by the GPU over
                                 the host link: the push stage of sparse
                                 sweeps (seraph_params.push) needs it        */

typedef struct seraph_graph seraph_graph;  /* opaque, library-owned */

typedef struct seraph_graph_info {
    uint64_t n;                 /* vertices                                  */
    uint64_t m_raw;             /* edges given (after SYMMETRIZE doubling)   */
    uint64_t m;                 /* edges kept: self-loops dropped, duplicate
                                   (u,v) collapsed to the smallest weight    */
    uint64_t struct_bytes;      /* pinned bytes of all page structures       */
    uint64_t weight_bytes;      /* pinned bytes of all page weights (0 if none) */
    uint64_t max_page_struct_bytes;
    uint64_t max_page_weight_bytes;
    uint32_t num_pages;
    uint32_t weighted;
    uint32_t symmetrized;
    uint32_t max_in_degree;
    uint32_t weight_width;      /* bytes per stored weight: 1, 2 or 4 (the
                                   narrowest that holds the largest weight) */
    uint32_t reordered;         /* 1 if built with SERAPH_REORDER            */
    uint32_t packed;            /* 1 if built with SERAPH_COMPRESS           */
    uint32_t reserved;
    uint64_t packed_bytes;      /* pinned bytes of all packed page structures */
    uint64_t packed_data_bytes; /* gap-stream bytes of all pages (unpadded)  */
    uint64_t max_page_packed_bytes;
    uint64_t out_edge_bytes;    /* pinned bytes of the out-edge CSR (0 without
                                   SERAPH_OUT_EDGES)                         */
} seraph_graph_info;

/*
 * Build a paged CSC graph from a raw edge list (Sec. 3.1 "Subgraph
 * Organization").  On the GPU: sort by (destination, source), drop self-loops,
 * collapse duplicates keeping the smallest weight, build the column offsets,
 * cut `num_pages` destination ranges balanced on (vertices + in-edges) --
 * page j starts at the smallest v with (v + in_offset[v]) * P >= j * (n + m)
 * -- and copy each page into library-owned pinned host memory as
 *   structure: u32 offsets relative to the page (nv+1, padded to 16 B),
 *              u32 source ids (ne, padded to 16 B);
 *   weights:   ne weights of 1, 2 or 4 bytes -- the narrowest width that holds
 *              the largest weight, a lossless encoding that keeps the streamed
 *              data compact (padded to 16 B) -- in a separate region so that
 *              unweighted algorithms stream structure only.
 * src/dst/w: m entries each in `mem`; w may be NULL (unweighted).  Every id
 * must be < n (SERAPH_EINVAL otherwise).  Out-degrees are kept resident on the
 * device for PageRank.  num_pages in [1, 2^20].
 */
int seraph_graph_from_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            const uint32_t* w, int mem, uint32_t flags, uint32_t num_pages,
                            void* stream, seraph_graph** out);

/* Same, from a CSR (row_off: n+1 uint64 offsets; col: row_off[n] ids; w NULL
 * or row_off[n] weights), all in `mem`.  row_off must start at 0 and never
 * decrease (SERAPH_EINVAL otherwise; offsets in host memory are checked
 * before any device call, offsets in device memory by a kernel before they
 * are used). */
int seraph_graph_from_csr(uint64_t n, const uint64_t* row_off, const uint32_t* col,
                          const uint32_t* w, int mem, uint32_t flags, uint32_t num_pages,
                          void* stream, seraph_graph** out);

int  seraph_graph_get_info(const seraph_graph* g, seraph_graph_info* info);

/* Page boundaries: vb[0..num_pages] (host array of num_pages+1 uint64). */
int  seraph_graph_page_bounds(const seraph_graph* g, uint64_t* vb);

/* Copy the CSC held in the pinned pages into host arrays (verification):
 * col_off[n+1] global in-edge offsets, row[m] sources (ascending within each
 * destination), w[m] weights (may be NULL), out_degree[n] (may be NULL). */
int  seraph_graph_export_csc(const seraph_graph* g, uint64_t* col_off, uint32_t* row,
                             uint32_t* w, uint32_t* out_degree);

/* The internal vertex order: perm[i] = the caller's id of internal vertex i
 * (host array of n uint32).  The identity unless built with SERAPH_REORDER.
 * With it, i < j implies outdeg(perm[i]) > outdeg(perm[j]), or equal
 * out-degrees and perm[i] < perm[j]; out-degrees count kept edges (after
 * SYMMETRIZE, self-loop removal and deduplication). */
int  seraph_graph_export_perm(const seraph_graph* g, uint32_t* perm);

/* The packed gap streams (SERAPH_COMPRESS graphs; SERAPH_EINVAL otherwise),
 * pages concatenated without padding: boff[n+1] global byte offsets of each
 * destination's bytes, data[packed_data_bytes].  Either may be NULL. */
int  seraph_graph_export_packed(const seraph_graph* g, uint64_t* boff, uint8_t* data);

/* The out-edge CSR (SERAPH_OUT_EDGES graphs; SERAPH_EINVAL otherwise), in
 * internal ids: out_off[n+1], out_col[m] (destinations ascending per
 * source), out_w[m] weights (may be NULL; ignored for unweighted graphs). */
int  seraph_graph_export_out_edges(const seraph_graph* g, uint64_t* out_off, uint32_t* out_col,
                                   uint32_t* out_w);

/* A run keeps its device buffers (edge ring, vertex arrays, lists) with the
 * graph for the next run, so repeated runs allocate nothing; this returns
 * them to the device (seraph_graph_free does too).  Must not overlap a run on
 * the same graph. */
int  seraph_graph_release_buffers(seraph_graph* g);

void seraph_graph_free(seraph_graph* g);

/*
 * Run parameters.  Fill with seraph_params_default(), then override.
 *
 * Streaming (Sec. 3.2, Fig. 4): the device edge buffer of `budget_bytes` is a
 * ring of `slots` (default window+1) slots.  Pages are packed in order into
 * chunks of at most one slot.  Chunks outside the window stay resident as
 * long as the schedule's look-ahead says they are needed sooner than the
 * others (furthest-next-use eviction).  Step t runs `passes` local passes over the `window` most recent
 * chunks while the next chunk copies into the free slot, then the oldest chunk
 * leaves the window: with passes = 1 every chunk gets `window` passes per
 * sweep and shares them with its neighbours (the sliding "super subgraph");
 * window = 1, passes = k is the double-buffer variant.  If all chunks fit in
 * the ring at once they are loaded once and never re-streamed.  A sweep runs
 * the window over every chunk once, in the direction given by `order`.
 *
 * Termination: SSSP/BFS/CC stop once every chunk has been processed with
 * prediction off after the last value change anywhere (the all-pull
 * retrieval of Sec. 4.3: a prediction-off sweep is run whenever a predicted
 * sweep changes nothing); PageRank stops when the FP64 L1 change between two
 * sweep ends is < tol, or at max_sweeps.
 */
typedef struct seraph_params {
    int32_t  algo;              /* seraph_algo                                */
    uint32_t source;            /* SSSP/BFS source vertex                     */
    uint64_t budget_bytes;      /* device edge-buffer budget                  */
    uint32_t window;            /* chunks resident in the compute window, 1..16 */
    uint32_t passes;            /* local passes per step, 1..64               */
    int32_t  pvu;               /* seraph_pvu                                 */
    uint32_t verify;            /* 1: finish with a prediction-off sweep (must
                                   stay 1 for weak prediction)                */
    uint8_t  fsm_next[12];      /* weak state machine: next state =
                                   fsm_next[2*state + changed]; dormant states
                                   use column 0 as their unconditional tick   */
    uint8_t  fsm_skip_mask;     /* bit s set: state s skips the update        */
    uint8_t  kahan;             /* PageRank: 1 = compensated FP32 sums        */
    uint8_t  pr_normalize;      /* PageRank (not in the paper): 1 = at every
                                   sweep end whose total sum(x) is off 1 by
                                   more than 2^-22, scale x (and x / outdeg)
                                   by 1 / sum(x).  The fixpoint sums to 1
                                   (summing its equation over all vertices
                                   gives sum = (1-d) + d sum), so it never
                                   moves; the scaling removes the error along
                                   the fixpoint's own direction, which the
                                   steps' in-place (Gauss-Seidel) updates with
                                   a dangling mass one sweep old leave behind
                                   and which otherwise decays only by about d
                                   per sweep.  0 = off                        */
    uint8_t  pad0;
    uint32_t max_sweeps;
    double   damping;           /* PageRank d                                 */
    double   tol;               /* PageRank stop: L1 change < tol             */
    double   pr_fail_eps;       /* PageRank weak prediction: an update "fails"
                                   when |dx| <= pr_fail_eps * x               */
    double   pr_pvu_off_below;  /* PageRank: prediction off once L1 change < this */
    uint32_t thread_max_deg;    /* in-degree <= this: one thread per vertex   */
    uint32_t warp_max_deg;      /* <= this: one warp (or a smaller lane group,
                                   see group*_max_deg); above: one CTA       */
    int32_t  sched;             /* seraph_sched                               */
    uint32_t timeout_ms;        /* bound on every host wait                   */
    uint32_t profile;           /* 1: time every relax kernel and step with
                                   CUDA events (fills relax_ms, copy_ms, ...) */
    uint32_t order;             /* seraph_order: chunk order across sweeps     */
    uint32_t max_passes;        /* idle-slot filling (Sec. 3.2): after `passes`
                                   passes keep running passes over the window,
                                   up to this many per step, while the next
                                   chunk is still in flight and the last pass
                                   changed something (<= passes: off)          */
    uint32_t slots;             /* ring slots the budget is split into, >=
                                   window + 1 (0 = window + 1).  Slots beyond
                                   the window keep chunks resident across
                                   sweeps so they are not streamed again      */
    uint32_t group4_max_deg;    /* in-degree <= this (and > thread_max_deg):
                                   4 lanes per vertex                         */
    uint32_t group8_max_deg;    /* <= this: 8 lanes per vertex; require
                                   thread <= group4 <= group8 <= warp          */
    void*    sched_model;       /* seraph_sched_model* for SERAPH_SCHED_LEARNED */
    void*    stream;            /* cudaStream_t for compute, NULL = own       */
    void*    trace;             /* seraph_trace* to fill, or NULL             */
    uint32_t columns;           /* page form streamed: SERAPH_COLUMNS_AUTO
                                   (packed when the graph has it), _PLAIN (u32
                                   source ids), _PACKED (LEB128 gaps) or
                                   _HYBRID (packed prefix of the pages)      */
    uint32_t pad1;
    uint64_t l2_hot_bytes;      /* L2 residency hint (not in the paper): the
                                   gathered values of vertices with internal
                                   id < l2_hot_bytes / 4 are read with L2
                                   evict-last priority and streamed page data
                                   with evict-first, so the most-read values
                                   stay in L2 (pair with SERAPH_REORDER, which
                                   puts them first); a graph's first such run
                                   raises the context's persisting-L2 limit to
                                   that size, and it stays raised until the
                                   last graph holding it is freed or has its
                                   buffers released, when the earlier value
                                   comes back.  0 = no hints;
                                   the default SERAPH_L2_HOT_AUTO = 3/8 of
                                   the device's L2.  Never changes a result. */
    double   pr_omega;          /* PageRank over-relaxation (not in the paper):
                                   a pass publishes x + omega (x_new - x),
                                   clamped at 0, instead of x_new (successive
                                   over-relaxation of the in-place steps; the
                                   fixpoint is the same) until a sweep
                                   changes x by less than pr_pvu_off_below
                                   (L1); later sweeps publish x_new.  0 or 1
                                   = plain updates; must lie in [0, 2)     */
    uint32_t push;              /* dense -> sparse switch (Sec. 3.1, the
                                   heterogeneous execution model: sparse
                                   iterations push from the active vertices):
                                   1 = after a sweep in which every
                                   non-final vertex was relaxed (prediction
                                   off, or strong) and at most push_below
                                   vertices changed, the run leaves the pages
                                   and pushes from the changed vertices over
                                   the graph's out-edge CSR (SERAPH_OUT_EDGES),
                                   round by round on the GPU, until a round
                                   changes nothing: the fixpoint.  SSSP, BFS
                                   and CC (on a symmetrized graph).  0 = off */
    uint32_t pad2;
    uint64_t push_below;        /* switch threshold in changed vertices (0 =
                                   n / 256)                                  */
    uint32_t count_clean;       /* measurement (SSSP, BFS, CC): 1 = at every
                                   sweep close count the pages none of whose
                                   in-edge sources changed in that sweep (the
                                   pages active-page skipping could leave out
                                   of the next sweep), into stats.clean_pages;
                                   sources are grouped in 1024 blocks of
                                   consecutive ids, so the count is a lower
                                   bound                                     */
    uint32_t stream_packed;     /* 1 (graphs built with SERAPH_COMPRESS): a
                                   chunk processed in the plain form streams
                                   compact into the far end of its ring slot
                                   -- per page a header of one bit per vertex
                                   (has an in-edge) and two bytes per vertex
                                   that has one (in-degree, LEB128 code
                                   bytes; larger counts in an escape list)
                                   with the offsets of every 256th vertex,
                                   then the page's gap stream -- and is
                                   rebuilt on the
                                   device into the plain form, page by page
                                   (each page's plain bytes end before its
                                   staged bytes start), so the host link
                                   carries neither offset array nor the
                                   4-byte columns; chunks that cannot be laid
                                   out so stream plain.  Chunks are cut with
                                   one staged page of slack.  A transfer
                                   encoding (not in the paper): results
                                   unchanged.  0 = off                       */
} seraph_params;

#define SERAPH_L2_HOT_AUTO UINT64_MAX
#define SERAPH_COLUMNS_AUTO   0u
#define SERAPH_COLUMNS_PLAIN  1u
#define SERAPH_COLUMNS_PACKED 2u
#define SERAPH_COLUMNS_HYBRID 3u  /* the first pages packed, the rest plain: the
                                     fewest packed pages with which every chunk
                                     stays resident in the ring (window 1)   */

typedef struct seraph_stats {
    uint32_t sweeps;            /* sweeps run                                 */
    uint32_t steps;             /* pipeline steps                             */
    uint32_t passes_run;        /* local passes executed                      */
    uint32_t passes_skipped;    /* local passes skipped on the device flag    */
    uint32_t chunks;            /* chunks per sweep                           */
    uint32_t resident;          /* 1 if all chunks stayed loaded              */
    uint32_t converged;         /* 1 if the stop rule was met                 */
    uint32_t verify_sweeps;     /* sweeps run with prediction off for the stop */
    uint64_t bytes_streamed;    /* host->device page bytes                    */
    uint64_t edges_relaxed;     /* in-edges read by attempted vertices        */
    uint64_t vertices_attempted;
    uint64_t vertices_skipped;  /* skipped by prediction                      */
    uint64_t changes;           /* value changes (PageRank: |dx| > eps*x)     */
    double   time_ms;           /* device time: first copy -> stop decided    */
    double   copy_ms;           /* sum of copy durations                      */
    double   compute_ms;        /* sum of step compute durations              */
    double   wall_ms;           /* host time of the whole call                */
    double   residual;          /* PageRank: last FP64 L1 change              */
    double   relax_ms;          /* sum of relax-kernel durations (events)     */
    uint64_t relax_launches;    /* relax kernels launched                     */
    uint64_t kernel_launches;   /* all library kernels launched by the run    */
    uint64_t packed_edges;      /* part of edges_relaxed read from packed pages */
    uint64_t code_bytes;        /* their LEB128 code bytes (the column bytes a
                                   relax pass reads for them, against 4 per
                                   edge on plain pages)                       */
    uint64_t push_edges;        /* out-edges read by the push stage           */
    uint32_t push_rounds;       /* push rounds with a non-empty frontier      */
    uint32_t push_sweep;        /* sweeps run before the switch (0: none)     */
    uint64_t clean_pages;       /* count_clean: pages, summed over sweeps,
                                   with no in-edge source block changed in
                                   the sweep                                 */
} seraph_stats;

int seraph_params_default(seraph_params* p, int algo);

/*
 * Run `p->algo` to its fixpoint over the paged graph.
 * out_values: n entries in out_mem -- uint32 distances / levels / labels, or
 * float32 PageRank values.  stats may be NULL.
 * Errors: SERAPH_EINVAL (bad params, e.g. strong prediction with PageRank, or
 * source >= n), SERAPH_EBUDGET (a page larger than one ring slot),
 * SERAPH_EOVERFLOW, SERAPH_ENOTCONV, SERAPH_ETIMEOUT, SERAPH_ECUDA.
 */
int seraph_run(seraph_graph* g, const seraph_params* p, void* out_values, int out_mem,
               seraph_stats* stats);

/*
 * No-allocation pull fixpoint (the paper has no counterpart).
 *
 * For callers that cannot call cudaMalloc: code whose device memory is owned
 * by a framework's allocator or memory planner, or a latency-critical loop
 * where cudaMalloc/cudaFree (which synchronise the device and can fail under
 * memory pressure) are not allowed.  Runs the pull relaxation of seraph_run --
 * each vertex takes the minimum over its in-edges, one warp per vertex -- to
 * its fixpoint over a CSC already in device memory, and allocates nothing:
 * its only scratch is a file-scope device array sized for
 * SERAPH_NOALLOC_MAX_VERTICES vertices, held by every GPU that loads the
 * library until the process exits.
 *
 * algo: SERAPH_SSSP, SERAPH_BFS or SERAPH_CC.  col_off[n+1] (uint64) and
 * row[col_off[n]] (source ids, any order within a destination) and w (NULL =
 * unit weights) are caller-owned device arrays; values[n] receives the
 * distances / levels / labels (caller-owned device array); passes_out (host,
 * may be NULL) receives the number of passes.  For CC pass the symmetric
 * graph.  Before anything else is read through the CSC a kernel checks it:
 * col_off must start at 0 and never decrease and every row id must be < n
 * (SERAPH_EINVAL otherwise, values untouched); row must hold col_off[n]
 * entries (and w, when given, as many), which no call can check.  Errors:
 * SERAPH_EINVAL (n > SERAPH_NOALLOC_MAX_VERTICES, bad algo, NULL pointers,
 * source >= n, the CSC check above), SERAPH_EOVERFLOW, SERAPH_ECUDA.
 *
 * The first call on each device resolves the scratch array's device address
 * (cudaGetSymbolAddress).  Every pass ends with a host read of its change
 * count, so a call returns only once its fixpoint is reached.  All calls share the scratch array and each clears it on entry, so calls
 * that overlap on the GPU race: serialise them.
 */
#define SERAPH_NOALLOC_MAX_VERTICES (1u << 20)
int seraph_pull_fixpoint_noalloc(int algo, uint64_t n, const uint64_t* col_off,
                                 const uint32_t* row, const uint32_t* w, uint32_t source,
                                 uint32_t* values, uint32_t* passes_out, void* stream);

/*
 * Random-gather probe (not in the paper; a measurement aid).
 *
 * Times the relax kernels' inner operation in isolation: n_gathers 4-byte
 * reads of a device array of n_values values, at indexes that stream in
 * order (16-byte loads, L2 evict-first) and are drawn by a counter-based hash
 * uniformly from [0, hot_values) with probability hot_frac, else from
 * [hot_values, n_values).  Reads of the hot range carry L2 evict-last hints
 * under a persisting-L2 set-aside of 4 * hot_values bytes (the context's
 * previous limit comes back on return), as in seraph_run.  One warm-up
 * launch, then `reps` timed launches (CUDA events on `stream`, NULL = the
 * default stream); *best_seconds (host) receives the fastest.  With every
 * index in a range far smaller than L2 it measures the rate of random gathers
 * that hit L2 -- the ceiling of a pull pass whose gathers all hit -- and with
 * cold indexes the cost of DRAM misses.
 *
 * Allocates 4 * n_values + 4.5 * n_gathers bytes of device memory for the
 * call.  Errors: SERAPH_EINVAL (n_values 0 or >= 2^32, n_gathers not a
 * positive multiple of 8, hot_values > n_values, hot_frac outside [0, 1],
 * reps 0, best_seconds NULL -- all checked before any device call),
 * SERAPH_ENOMEM, SERAPH_ECUDA.
 */
int seraph_gather_probe(uint64_t n_values, uint64_t n_gathers, uint64_t hot_values,
                        double hot_frac, uint32_t reps, void* stream, double* best_seconds);

/*
 * Learned scheduler (not in the paper; its closest counterpart is the
 * fine-grained idle-slot scheduling of Sec. 3.2).  A 16 -> 64 -> 64 -> 17 MLP
 * with GELU, BF16 weights and FP32 accumulation (FP32 master weights, Adam),
 * trained and run by the library's own kernels.  Inputs: 16 per-chunk
 * features of a pipeline step (SERAPH_SCHED_FEATURE_* below).  Outputs: the
 * number of local passes k in [1,16] for the step (argmax of 16 logits) and a
 * streaming priority (predicted first-pass gain).  With params.sched =
 * SERAPH_SCHED_LEARNED (window must be 1) the device caps each step's passes
 * at the predicted k (no host round trip).  For SSSP/BFS/CC the priority
 * orders the stream: each sweep takes the chunks already in the ring first,
 * then the others, each group by decreasing predicted gain (PageRank keeps
 * the base cyclic or zigzag order); a chunk predicted to change nothing
 * (priority < 0.02) may be skipped, for at most three sweeps in a row and
 * never when verify = 0, which the stop rule (every chunk processed after the
 * last change) makes safe.  The fixed schedule remains the fallback and the
 * yardstick.
 */
#define SERAPH_SCHED_FEATURES 16
#define SERAPH_SCHED_OUTPUTS 17
#define SERAPH_SCHED_PARAMS 6353   /* 64*16+64 + 64*64+64 + 17*64+17 */

typedef struct seraph_sched_model seraph_sched_model;  /* opaque */

/* A trace of pipeline steps filled by seraph_run (params.trace; window must
 * be 1): per step the 16 features seen at the step's start and the number of
 * value changes in each of its passes (up to 16; 0 for passes not run). */
typedef struct seraph_trace {
    uint64_t capacity;          /* rows the caller allocated                 */
    uint64_t count;             /* rows written (output)                     */
    float*    features;         /* host, capacity x 16                       */
    uint32_t* gains;            /* host, capacity x 16                       */
    uint32_t* vertices;         /* host, capacity: vertices of the chunk     */
} seraph_trace;

/* New model with Glorot-uniform weights from a seeded splitmix64 stream.
 * fp32 != 0: debug mode, the forward pass uses the FP32 master weights. */
int  seraph_sched_create(uint64_t seed, int fp32, seraph_sched_model** out);
int  seraph_sched_get_params(const seraph_sched_model* m, float* params /* host, PARAMS */);
int  seraph_sched_set_params(seraph_sched_model* m, const float* params /* host, PARAMS */);
/* Mean loss over n samples and its gradient w.r.t. the master weights:
 * CE(softmax(logits), k-1) + (priority_out - prio)^2.  x: n x 16, k: n
 * (1..16), prio: n, all in `mem`; loss and grad (PARAMS floats) on the host. */
int  seraph_sched_loss_grad(seraph_sched_model* m, const float* x, const int32_t* k,
                            const float* prio, uint64_t n, int mem, float* loss, float* grad);
/* `epochs` passes of Adam over shuffled mini-batches; losses[e] (host, may be
 * NULL) receives the mean batch loss of epoch e. */
int  seraph_sched_train(seraph_sched_model* m, const float* x, const int32_t* k, const float* prio,
                        uint64_t n, int mem, uint32_t epochs, uint32_t batch, float lr,
                        uint64_t seed, float* losses);
/* Predictions for n feature rows (x in `mem`; outputs in the same memory). */
int  seraph_sched_infer(const seraph_sched_model* m, const float* x, uint64_t n, int mem,
                        int32_t* k_out, float* prio_out);
/* Training targets from a trace: k = smallest number of passes that captures
 * at least `share` of the step's changes (1..16); priority = log2(1 + first
 * pass changes) / 24.  Host arrays of trace->count entries. */
int  seraph_sched_targets(const seraph_trace* t, float share, int32_t* k_out, float* prio_out);
void seraph_sched_free(seraph_sched_model* m);

/*
 * Batched queries (not in the paper; a serving pattern): many BFS /
 * SSSP queries over many graphs resident in device memory, run by one
 * persistent kernel that is captured in a CUDA graph.  Each query advances
 * in frontier rounds (push relaxation over the out-edge CSR, label
 * correcting, so the results are the exact distances / levels); the tiles of
 * every query's rounds share one task ring.  The tile mapping -- one thread,
 * one warp, or the whole CTA (edge-balanced) per frontier vertex -- and the
 * tile size are chosen per graph by an autotuner that times each candidate
 * on the graph's own queries (cached in the graph for later calls).
 */
typedef struct seraph_bgraph seraph_bgraph;   /* device-resident out-edge CSR */

enum seraph_mapping { SERAPH_MAP_AUTO = 0, SERAPH_MAP_THREAD = 1, SERAPH_MAP_WARP = 2,
                      SERAPH_MAP_CTA = 3 };

typedef struct seraph_query {
    uint32_t graph;             /* index into the graphs array                */
    int32_t  algo;              /* SERAPH_SSSP or SERAPH_BFS                  */
    uint32_t source;
    uint32_t reserved;
    uint32_t* out;              /* n_graph distances / levels, in out_mem     */
} seraph_query;

typedef struct seraph_batch_params {
    int32_t  mapping;           /* seraph_mapping; AUTO = autotune per graph  */
    uint32_t tile;              /* frontier vertices per task (0 = 256)       */
    uint32_t use_graph;         /* 1: capture the launch in a CUDA graph      */
    uint32_t replays;           /* timed repetitions (>= 1)                   */
    uint32_t timeout_ms;        /* bound on every wait, device and host       */
    uint32_t delta;             /* SSSP near-far bucket width: an improved
                                   vertex whose distance is below the current
                                   split joins the next round, the rest wait
                                   in a far pile until the split rises by
                                   delta; BFS ignores it.  0 = per graph: with
                                   mapping AUTO the autotuner times 64, 128,
                                   256 and 512 on the graph's SSSP queries and
                                   keeps the fastest (cached with the
                                   mapping), otherwise 64                    */
    void*    stream;            /* cudaStream_t, NULL = own                   */
    uint32_t bfs_pull_div;      /* BFS direction switch (Beamer et al.): a
                                   round whose frontier exceeds n / div runs
                                   bottom-up -- every unvisited vertex looks
                                   for a parent among its in-neighbours --
                                   instead of pushing (0 = 5; 1 = never)     */
    uint32_t group;             /* 1 (default): queries of one graph and one
                                   algorithm run in lockstep groups of up to
                                   8 -- one frontier of vertices for the
                                   group, per vertex the sub-queries that
                                   hold it, distances interleaved -- so one
                                   read of a vertex's out-edges serves every
                                   sub-query that holds it and a
                                   destination's distances share one sector
                                   (the group shares the near-far split; edge-
                                   balanced CTA tiles of at most 512 vertices
                                   whatever the mapping).  Exact distances
                                   either way.  0 = one record per query     */
} seraph_batch_params;

typedef struct seraph_batch_stats {
    double   time_ms;           /* one batched launch (mean over replays)     */
    double   tune_ms;           /* autotuning time (0 when cached)            */
    uint64_t edges;             /* out-edges relaxed by all queries           */
    uint64_t tasks;             /* tiles processed                            */
    uint32_t rounds_max;        /* most frontier rounds of any query          */
    uint32_t graph_captured;    /* 1 if the launch ran from a CUDA graph      */
    uint32_t mapping[16];       /* chosen mapping of graphs 0..15             */
    uint32_t tile[16];          /* chosen tile of graphs 0..15                */
} seraph_batch_stats;

/* Resident out-edge CSR (self-loops dropped, duplicates keep the smallest
 * weight, weights in the narrowest lossless width); arguments as for
 * seraph_graph_from_edges. */
int  seraph_bgraph_from_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                              const uint32_t* w, int mem, void* stream, seraph_bgraph** out);
void seraph_bgraph_free(seraph_bgraph* g);
int  seraph_batch_params_default(seraph_batch_params* p);
/* Run nq queries over ng graphs (one device).  Errors: SERAPH_EINVAL,
 * SERAPH_ETIMEOUT (a bounded wait in the kernel ran out), SERAPH_ECUDA. */
int  seraph_batch_run(seraph_bgraph* const* graphs, uint32_t ng, const seraph_query* queries,
                      uint32_t nq, int out_mem, const seraph_batch_params* p,
                      seraph_batch_stats* stats);

/* A prepared batch for serving loops: the same queries (sources may change)
 * run again and again without re-planning.  seraph_batch_plan_create does
 * what seraph_batch_run does before its launch -- checks, autotuning (cached
 * in the graphs), grouping, the device tables, the per-query arrays, the
 * captured launch when params.use_graph -- once; every queries[i].out must be
 * a caller-owned DEVICE array of n_graph uint32, written by every run (the
 * caller reads it back however it likes, e.g. on its own stream while the
 * next run computes).  The graphs must outlive the plan; params.replays is
 * ignored (one launch per run); runs go to params.stream (NULL = the plan's
 * own) and must not overlap.
 * seraph_batch_plan_run: one launch; `sources` (host, nq values, NULL = as
 * before) replaces the queries' sources first (checked against n; SERAPH_EINVAL
 * with nothing run otherwise).  It allocates nothing unless new sources change
 * a group's round-0 task count (a tile smaller than the group with repeated
 * sources), when the plan is rebuilt.  Returns after the launch completes;
 * stats as for seraph_batch_run (tune_ms 0).  Errors as seraph_batch_run. */
typedef struct seraph_batch_plan seraph_batch_plan;
int  seraph_batch_plan_create(seraph_bgraph* const* graphs, uint32_t ng,
                              const seraph_query* queries, uint32_t nq,
                              const seraph_batch_params* p, seraph_batch_plan** plan);
int  seraph_batch_plan_run(seraph_batch_plan* plan, const uint32_t* sources,
                           seraph_batch_stats* stats);
void seraph_batch_plan_free(seraph_batch_plan* plan);

/*
 * Host-side fault injection and accounting, for tests of the failure paths
 * (not in the paper).  Every failure is made on the host; nothing here makes
 * the device fault or wait.
 *
 * seraph_debug_fail_pinned_alloc(k): the k-th pinned host allocation the
 * library makes from now on (k >= 1; process-wide, any thread) fails as if
 * the host had no pinned memory left, and the call that made it returns
 * SERAPH_ENOMEM after freeing what it had taken.  k = 0 disarms.  Returns
 * SERAPH_OK.
 * seraph_debug_pinned_bytes(): pinned host bytes the library holds right now
 * (all graphs, runs and buffers of the process), so that a test can check
 * that a failed call gave back everything it allocated.
 * seraph_debug_l2_setaside(bytes): the current context's persisting-L2
 * set-aside limit (cudaLimitPersistingL2CacheSize) in *bytes.  Runs that keep
 * their hot range in L2 raise it once per graph and leave it raised until the
 * graph is freed or its buffers released; then the earlier value comes back.
 * Returns SERAPH_ECUDA if the limit cannot be read.
 */
int      seraph_debug_fail_pinned_alloc(uint32_t k);
uint64_t seraph_debug_pinned_bytes(void);
int      seraph_debug_l2_setaside(uint64_t* bytes);

/* Message for the last failing call on this thread ("" if none). */
const char* seraph_last_error(void);

/* Library version string. */
const char* seraph_version(void);

#ifdef __cplusplus
}
#endif
#endif
