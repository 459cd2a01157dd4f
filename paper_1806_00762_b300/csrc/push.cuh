// Push stage of sparse sweeps (Sec. 3.1, heterogeneous execution model):
// once a pull sweep in which every non-final vertex was relaxed changes only
// a few vertices, the remaining work is pushed from those vertices over the
// out-edge CSR (SERAPH_OUT_EDGES, pinned host memory read directly by the
// kernels), round by round, instead of streaming and pulling every page.
//
// Why it is exact: if every destination v was relaxed (or is final) at some
// step after the start of sweep T, an edge (u, v) can violate val[v] <=
// val[u] (+) w only if u changed since then (otherwise v saw u's current
// value when it was relaxed, and v only decreases afterwards).  A round
// relaxes every out-edge of its frontier and collects the vertices it
// improved; an edge from a vertex that did not improve in the round cannot
// be violated afterwards.  A round with an empty frontier therefore leaves no
// violated edge: the least fixpoint (shortest distances, BFS levels, minimum
// component labels).
#pragma once

#include "engine.cuh"

namespace seraph {

// Frontier vertices with more out-edges than this are walked by the whole
// grid instead of one warp; fewer than m / kPushWarpMax + 1 vertices qualify.
constexpr uint64_t kPushWarpMax = 2048;

struct PushState {
    unsigned cnt[2];          // frontier sizes (double-buffered by round parity)
    unsigned nbig;            // frontier vertices of the round with > kPushWarpMax out-edges
    unsigned ovf;             // an SSSP candidate did not fit below 2^32-1
    unsigned rounds;          // rounds with a non-empty frontier
    unsigned pad;
    unsigned long long edges; // out-edges read
    unsigned long long changes;  // vertices improved (once per round)
};

struct PushArgs {
    const uint64_t* out_off;  // n+1 out-edge offsets (pinned host, device-readable)
    const uint32_t* out_col;  // destinations
    const uint8_t* out_w;     // weights, wbytes each, or null
    uint32_t wbytes;
    uint32_t n;
    uint32_t* val;            // values (device)
    uint32_t* stamp;          // tag of the sweep / round in which a vertex last changed
    uint32_t* front[2];       // frontier lists, n entries each
    uint32_t* big;            // high out-degree vertices of the current round
    uint32_t big_cap;
    PushState* ps;
};

// Frontier of round 0: every vertex whose stamp is `tag` or later (the vertices
// changed since the earliest sweep that some chunk was last validly processed in).
void launch_push_frontier(const PushArgs& a, uint32_t tag, cudaStream_t s);
// Round r over front[r & 1] into front[(r + 1) & 1]; improved vertices get
// stamp `tag` (unique per round).  Does nothing when the frontier is empty.
void launch_push_round(int algo, const PushArgs& a, uint32_t r, uint32_t tag, cudaStream_t s);

}  // namespace seraph
