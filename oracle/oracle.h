/*
 * oracle.h -- plain, slow, obviously correct CPU reference for the Seraph
 * streamed-graph hot path (arXiv 1806.00762).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product library shares no code, header, table or helper with it.
 *
 * Every result the paper's method reaches is a plain definition, so the
 * oracle writes that definition out:
 *   - SSSP: Dijkstra on the directed weighted graph (evaluation section,
 *     "Graph Algorithms"); distances accumulated in 64 bits.
 *   - BFS: FIFO-queue breadth-first levels on the directed graph (same).
 *   - CC: weakly connected components (Table 1 names WCC), label = minimum
 *     vertex id of the component, by union-find.
 *   - PageRank (named in Sec. 4.3 as the case needing weak prediction):
 *     FP64 power iteration with uniform redistribution of dangling mass,
 *     x' = (1-d)/n + d (sum_{u->v} x_u/outdeg(u) + D/n), D = sum over
 *     out-degree-0 vertices of x_u.
 *   - Graph build: self-loops dropped, duplicate (u,v) collapsed keeping the
 *     smallest weight; CSR rows ascending by destination.
 *   - CSC pages (Sec. 3.1 "Subgraph Organization"): transpose with sources
 *     ascending in each column; pages cut by destination range so that each
 *     holds about E/P in-edges.
 *   - Certificates for sizes where a full run is too slow: the SSSP/BFS
 *     optimality conditions checked edge by edge over the raw edge stream.
 *
 * Unreachable distances/levels are 0xFFFFFFFF.  Return codes: 0 = ok,
 * -6 = a distance does not fit below 0xFFFFFFFF.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_INF 0xFFFFFFFFu

/* Build a simple directed CSR from raw edges.  row_off has n+1 entries, col
 * and wout (if w != NULL) have room for m entries.  Returns the edge count E. */
uint64_t oracle_build_csr(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                          const uint32_t* w, uint64_t* row_off, uint32_t* col, uint32_t* wout);

/* CSC (in-edges) of a CSR: col_off[n+1], row[E] (sources ascending within a
 * column), wcsc[E] if w != NULL. */
void oracle_csc(uint64_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                uint64_t* col_off, uint32_t* row, uint32_t* wcsc);

/* Destination-range page cut: vb[0]=0, vb[P]=n, vb[j] = smallest v with
 * col_off[v] * P >= j * E for 0<j<P. */
void oracle_page_cut(uint64_t n, const uint64_t* col_off, uint32_t P, uint64_t* vb);

int  oracle_sssp(uint64_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                 uint32_t source, uint32_t* dist);
void oracle_bfs(uint64_t n, const uint64_t* row_off, const uint32_t* col, uint32_t source,
                uint32_t* level);
void oracle_cc(uint64_t n, const uint64_t* row_off, const uint32_t* col, uint32_t* label);
void oracle_cc_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                     uint32_t* label);

/* FP64 PageRank.  Runs until the L1 change of one iteration is < tol or
 * maxit iterations; x receives the result.  Returns iterations run; *resid
 * gets the last L1 change.  Uses OpenMP over destination vertices (each
 * vertex sums its in-edges in CSC order, so the result is deterministic). */
int oracle_pagerank(uint64_t n, const uint64_t* row_off, const uint32_t* col, double d,
                    double tol, int maxit, double* x, double* resid);

/* One PageRank map application y = F(x) in FP64 (same definition). */
void oracle_pagerank_apply(uint64_t n, const uint64_t* row_off, const uint32_t* col, double d,
                           const double* x, double* y);

/* FP64 PageRank step certificate for graphs too large for one CSR build.
 *
 * One map application T(x)_v = (1-d)/n + d (sum_{u->v} x_u/outdeg(u) + D/n)
 * (the PageRank definition above) is assembled from a raw edge stream that
 * the caller replays, bucket by bucket: destinations are split into
 * `nbuckets` classes by a multiplicative hash, and for each class the caller
 * streams every raw edge through oracle_pr_bucket_keys, which keeps the keys
 * (dst << 32 | src) of the class's edges (self-loops dropped) in
 * keys[at..]; cap bounds the buffer (returns UINT64_MAX when it would
 * overflow, else the new key count).  oracle_pr_bucket_apply then sorts the
 * keys (in `nsub` parts split by the same hash, tmp = scratch of k entries),
 * drops duplicate edges and, for every distinct edge (u, v),
 *   mode 0: outdeg[u] += 1 (a first round over all classes gives the kept
 *           out-degrees),
 *   mode 1: s[j n + v] += x[j n + u] / outdeg[u] for each of the nx
 *           vectors x (rows of n), each destination's in-edges added in
 *           ascending source order (a second round gives the pull sums).
 * Returns the number of distinct edges of the class.  The caller forms
 * T(x) from s, the dangling mass D and d.  Since T is an affine map whose
 * linear part is d times a column-stochastic matrix, ||T x - T y||_1 <=
 * d ||x - y||_1, so ||x - x*||_1 <= ||T x - x||_1 / (1 - d) for any x: the
 * step residual bounds the distance to the fixpoint. */
uint64_t oracle_pr_bucket_keys(uint64_t count, const uint32_t* src, const uint32_t* dst,
                               uint32_t bucket, uint32_t nbuckets, uint64_t* keys, uint64_t at,
                               uint64_t cap);
uint64_t oracle_pr_bucket_apply(uint64_t k, uint64_t* keys, uint64_t* tmp, uint32_t nsub, int mode,
                                uint32_t* outdeg, uint64_t n, uint32_t nx, const double* x, double* s);

/* SSSP/BFS certificate over a stream of raw edges (self-loops ignored; w may
 * be NULL for unit weights).  Counts edges with dist[v] > dist[u] + w (the
 * triangle inequality violated) and marks tight[v] = 1 when
 * dist[v] == dist[u] + w with dist[u] finite.  Returns the violation count. */
uint64_t oracle_sp_check_edges(uint64_t count, const uint32_t* src, const uint32_t* dst,
                               const uint32_t* w, const uint32_t* dist, uint8_t* tight);

/* Final certificate step: dist[source] == 0 and every other vertex with a
 * finite value has a tight in-edge.  Returns the number of failing vertices. */
uint64_t oracle_sp_check_tight(uint64_t n, uint32_t source, const uint32_t* dist,
                               const uint8_t* tight);

#ifdef __cplusplus
}
#endif
#endif
