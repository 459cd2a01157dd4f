/*
 * oracle.c -- plain CPU reference for the Seraph hot path.
 * TEST INFRASTRUCTURE ONLY (see oracle.h): never linked into the product.
 *
 * Each function follows the definition cited in oracle.h.  No blocking, no
 * fusion, no reordering beyond what those definitions state.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- graph */

typedef struct { uint64_t key; uint32_t w; } kw_t;

static int cmp_kw(const void* pa, const void* pb)
{
    const kw_t* a = (const kw_t*)pa;
    const kw_t* b = (const kw_t*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->w != b->w) return a->w < b->w ? -1 : 1;
    return 0;
}

uint64_t oracle_build_csr(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                          const uint32_t* w, uint64_t* row_off, uint32_t* col, uint32_t* wout)
{
    kw_t* a = (kw_t*)malloc((m ? m : 1) * sizeof(kw_t));
    uint64_t k = 0;
    for (uint64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;                 /* drop self-loops */
        a[k].key = ((uint64_t)src[i] << 32) | dst[i];
        a[k].w = w ? w[i] : 0;
        ++k;
    }
    qsort(a, k, sizeof(kw_t), cmp_kw);                  /* by (src, dst, w) */
    memset(row_off, 0, (n + 1) * sizeof(uint64_t));
    uint64_t E = 0;
    for (uint64_t i = 0; i < k; ++i) {
        if (i > 0 && a[i].key == a[i - 1].key) continue; /* duplicate: keep min w */
        uint32_t u = (uint32_t)(a[i].key >> 32);
        col[E] = (uint32_t)a[i].key;
        if (w && wout) wout[E] = a[i].w;
        row_off[u + 1] += 1;
        ++E;
    }
    for (uint64_t v = 0; v < n; ++v) row_off[v + 1] += row_off[v];
    free(a);
    return E;
}

void oracle_csc(uint64_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                uint64_t* col_off, uint32_t* row, uint32_t* wcsc)
{
    memset(col_off, 0, (n + 1) * sizeof(uint64_t));
    uint64_t E = row_off[n];
    for (uint64_t e = 0; e < E; ++e) col_off[col[e] + 1] += 1;
    for (uint64_t v = 0; v < n; ++v) col_off[v + 1] += col_off[v];
    uint64_t* fill = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    memcpy(fill, col_off, n * sizeof(uint64_t));
    for (uint64_t u = 0; u < n; ++u) {
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint64_t pos = fill[col[e]]++;
            row[pos] = (uint32_t)u;
            if (w && wcsc) wcsc[pos] = w[e];
        }
    }
    free(fill);
}

void oracle_page_cut(uint64_t n, const uint64_t* col_off, uint32_t P, uint64_t* vb)
{
    /* cost(v) = v + col_off[v]: vertices (one offset each) plus in-edges. */
    uint64_t total = n + col_off[n];
    vb[0] = 0;
    vb[P] = n;
    uint64_t v = 0;
    for (uint32_t j = 1; j < P; ++j) {
        while (v < n && (v + col_off[v]) * (uint64_t)P < (uint64_t)j * total) ++v;
        vb[j] = v;
    }
}

/* ----------------------------------------------------------------- SSSP */

typedef struct {
    uint32_t* heap;   /* vertex ids */
    int64_t* pos;     /* -1: never inserted, -2: settled, else heap slot */
    const uint64_t* key;
    uint64_t size;
} heap_t;

static void heap_swap(heap_t* h, uint64_t i, uint64_t j)
{
    uint32_t a = h->heap[i], b = h->heap[j];
    h->heap[i] = b; h->heap[j] = a;
    h->pos[b] = (int64_t)i; h->pos[a] = (int64_t)j;
}

static void heap_up(heap_t* h, uint64_t i)
{
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h->key[h->heap[p]] <= h->key[h->heap[i]]) break;
        heap_swap(h, i, p);
        i = p;
    }
}

static void heap_down(heap_t* h, uint64_t i)
{
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->size && h->key[h->heap[l]] < h->key[h->heap[m]]) m = l;
        if (r < h->size && h->key[h->heap[r]] < h->key[h->heap[m]]) m = r;
        if (m == i) break;
        heap_swap(h, i, m);
        i = m;
    }
}

int oracle_sssp(uint64_t n, const uint64_t* row_off, const uint32_t* col, const uint32_t* w,
                uint32_t source, uint32_t* dist)
{
    uint64_t* d = (uint64_t*)malloc(n * sizeof(uint64_t));
    heap_t h;
    h.heap = (uint32_t*)malloc(n * sizeof(uint32_t));
    h.pos = (int64_t*)malloc(n * sizeof(int64_t));
    h.key = d;
    h.size = 0;
    for (uint64_t v = 0; v < n; ++v) { d[v] = UINT64_MAX; h.pos[v] = -1; }
    d[source] = 0;
    h.heap[0] = source; h.pos[source] = 0; h.size = 1;
    while (h.size > 0) {
        uint32_t u = h.heap[0];
        heap_swap(&h, 0, h.size - 1);
        h.size -= 1;
        h.pos[u] = -2;
        if (h.size > 0) heap_down(&h, 0);
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint32_t v = col[e];
            if (h.pos[v] == -2) continue;
            uint64_t nd = d[u] + (uint64_t)(w ? w[e] : 1);
            if (nd < d[v]) {
                d[v] = nd;
                if (h.pos[v] == -1) {
                    h.heap[h.size] = v; h.pos[v] = (int64_t)h.size; h.size += 1;
                }
                heap_up(&h, (uint64_t)h.pos[v]);
            }
        }
    }
    int rc = 0;
    for (uint64_t v = 0; v < n; ++v) {
        if (d[v] == UINT64_MAX) dist[v] = ORACLE_INF;
        else if (d[v] >= ORACLE_INF) { dist[v] = ORACLE_INF; rc = -6; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(h.heap); free(h.pos);
    return rc;
}

/* ------------------------------------------------------------------ BFS */

void oracle_bfs(uint64_t n, const uint64_t* row_off, const uint32_t* col, uint32_t source,
                uint32_t* level)
{
    uint32_t* queue = (uint32_t*)malloc(n * sizeof(uint32_t));
    for (uint64_t v = 0; v < n; ++v) level[v] = ORACLE_INF;
    uint64_t head = 0, tail = 0;
    level[source] = 0;
    queue[tail++] = source;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint32_t v = col[e];
            if (level[v] == ORACLE_INF) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
}

/* ------------------------------------------------------------------- CC */

static uint32_t uf_find(uint32_t* parent, uint32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];   /* path halving */
        x = parent[x];
    }
    return x;
}

void oracle_cc(uint64_t n, const uint64_t* row_off, const uint32_t* col, uint32_t* label)
{
    uint32_t* parent = label;            /* the label array doubles as the forest */
    for (uint64_t v = 0; v < n; ++v) parent[v] = (uint32_t)v;
    for (uint64_t u = 0; u < n; ++u) {
        for (uint64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            uint32_t a = uf_find(parent, (uint32_t)u), b = uf_find(parent, col[e]);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;   /* root = min id */
        }
    }
    for (uint64_t v = 0; v < n; ++v) label[v] = uf_find(parent, (uint32_t)v);
}

/* The same union-find over a raw edge list: every (src[i], dst[i]) joins its
 * two endpoints, whatever its direction, self-loops and duplicates included
 * (they join nothing new).  Weakly connected components with min-id labels,
 * without building a CSR first. */
void oracle_cc_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                     uint32_t* label)
{
    uint32_t* parent = label;
    for (uint64_t v = 0; v < n; ++v) parent[v] = (uint32_t)v;
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = uf_find(parent, src[i]), b = uf_find(parent, dst[i]);
        if (a == b) continue;
        if (a < b) parent[b] = a; else parent[a] = b;
    }
    for (uint64_t v = 0; v < n; ++v) label[v] = uf_find(parent, (uint32_t)v);
}

/* ------------------------------------------------------------- PageRank */

typedef struct {
    uint64_t* col_off;
    uint32_t* row;
    double* inv_out;
    uint8_t* dangling;
} pr_graph_t;

static void pr_graph_init(uint64_t n, const uint64_t* row_off, const uint32_t* col,
                          pr_graph_t* g)
{
    uint64_t E = row_off[n];
    g->col_off = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    g->row = (uint32_t*)malloc((E ? E : 1) * sizeof(uint32_t));
    g->inv_out = (double*)malloc(n * sizeof(double));
    g->dangling = (uint8_t*)malloc(n);
    oracle_csc(n, row_off, col, NULL, g->col_off, g->row, NULL);
    for (uint64_t u = 0; u < n; ++u) {
        uint64_t od = row_off[u + 1] - row_off[u];
        g->dangling[u] = od == 0;
        g->inv_out[u] = od ? 1.0 / (double)od : 0.0;
    }
}

static void pr_graph_free(pr_graph_t* g)
{
    free(g->col_off); free(g->row); free(g->inv_out); free(g->dangling);
}

static void pr_step(uint64_t n, const pr_graph_t* g, double d, const double* x, double* y)
{
    double D = 0.0;
    for (uint64_t u = 0; u < n; ++u) if (g->dangling[u]) D += x[u];
    double base = (1.0 - d) / (double)n + d * D / (double)n;
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        double s = 0.0;
        for (uint64_t e = g->col_off[v]; e < g->col_off[v + 1]; ++e) {
            uint32_t u = g->row[e];
            s += x[u] * g->inv_out[u];
        }
        y[v] = base + d * s;
    }
}

void oracle_pagerank_apply(uint64_t n, const uint64_t* row_off, const uint32_t* col, double d,
                           const double* x, double* y)
{
    pr_graph_t g;
    pr_graph_init(n, row_off, col, &g);
    pr_step(n, &g, d, x, y);
    pr_graph_free(&g);
}

int oracle_pagerank(uint64_t n, const uint64_t* row_off, const uint32_t* col, double d,
                    double tol, int maxit, double* x, double* resid)
{
    if (n == 0) { *resid = 0.0; return 0; }
    pr_graph_t g;
    pr_graph_init(n, row_off, col, &g);
    double* y = (double*)malloc(n * sizeof(double));
    for (uint64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    int it = 0;
    double r = INFINITY;
    while (it < maxit) {
        pr_step(n, &g, d, x, y);
        r = 0.0;
        for (uint64_t v = 0; v < n; ++v) r += fabs(y[v] - x[v]);
        memcpy(x, y, n * sizeof(double));
        ++it;
        if (r < tol) break;
    }
    *resid = r;
    free(y);
    pr_graph_free(&g);
    return it;
}

/* --------------------------------------------------------- certificates */

uint64_t oracle_sp_check_edges(uint64_t count, const uint32_t* src, const uint32_t* dst,
                               const uint32_t* w, const uint32_t* dist, uint8_t* tight)
{
    uint64_t bad = 0;
    #pragma omp parallel for reduction(+ : bad) schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) {
        uint32_t u = src[i], v = dst[i];
        if (u == v || dist[u] == ORACLE_INF) continue;
        uint64_t cand = (uint64_t)dist[u] + (w ? w[i] : 1u);
        if ((uint64_t)dist[v] > cand) bad += 1;          /* dist[v] == INF counts */
        else if ((uint64_t)dist[v] == cand) {
            #pragma omp atomic write
            tight[v] = 1;
        }
    }
    return bad;
}

uint64_t oracle_sp_check_tight(uint64_t n, uint32_t source, const uint32_t* dist,
                               const uint8_t* tight)
{
    uint64_t bad = dist[source] != 0;
    for (uint64_t v = 0; v < n; ++v)
        if (v != source && dist[v] != ORACLE_INF && !tight[v]) bad += 1;
    return bad;
}

/* ------------------------------------------- PageRank step certificate */

/* Destination hash shared by the two levels of the certificate's partition
 * (Knuth's multiplicative hashing with the 32-bit golden-ratio constant). */
static uint32_t pr_dst_hash(uint32_t v) { return v * 0x9E3779B1u; }

static uint32_t pr_bucket_of(uint32_t v, uint32_t nbuckets)
{
    return (uint32_t)(((uint64_t)pr_dst_hash(v) * nbuckets) >> 32);
}

uint64_t oracle_pr_bucket_keys(uint64_t count, const uint32_t* src, const uint32_t* dst,
                               uint32_t bucket, uint32_t nbuckets, uint64_t* keys, uint64_t at,
                               uint64_t cap)
{
    uint64_t cnt[257];
    int nt_used = 1;
    int over = 0;
    int want = 1;
#ifdef _OPENMP
    want = omp_get_max_threads() < 256 ? omp_get_max_threads() : 256;
#endif
    memset(cnt, 0, sizeof(cnt));
    #pragma omp parallel num_threads(want)
    {
        int t = 0, nt = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        uint64_t lo = count * (uint64_t)t / (uint64_t)nt, hi = count * (uint64_t)(t + 1) / (uint64_t)nt;
        uint64_t c = 0;
        for (uint64_t i = lo; i < hi; ++i)
            if (src[i] != dst[i] && pr_bucket_of(dst[i], nbuckets) == bucket) ++c;
        cnt[t + 1] = c;
        #pragma omp barrier
        #pragma omp single
        {
            nt_used = nt;
            for (int j = 0; j < nt; ++j) cnt[j + 1] += cnt[j];
            over = at + cnt[nt] > cap;
        }
        if (!over) {
            uint64_t o = at + cnt[t];
            for (uint64_t i = lo; i < hi; ++i)
                if (src[i] != dst[i] && pr_bucket_of(dst[i], nbuckets) == bucket)
                    keys[o++] = ((uint64_t)dst[i] << 32) | src[i];
        }
    }
    return over ? UINT64_MAX : at + cnt[nt_used];
}

static int cmp_u64(const void* pa, const void* pb)
{
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    return a < b ? -1 : (a > b);
}

uint64_t oracle_pr_bucket_apply(uint64_t k, uint64_t* keys, uint64_t* tmp, uint32_t nsub, int mode,
                                uint32_t* outdeg, uint64_t n, uint32_t nx, const double* x, double* s)
{
    /* split by a second hash level so that each destination lands in one
     * part (mode 1 sums without races), then sort each part */
    uint64_t* start = (uint64_t*)calloc((size_t)nsub + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < k; ++i) start[((pr_dst_hash((uint32_t)(keys[i] >> 32)) >> 8) % nsub) + 1] += 1;
    for (uint32_t p = 0; p < nsub; ++p) start[p + 1] += start[p];
    uint64_t* fill = (uint64_t*)malloc((size_t)nsub * sizeof(uint64_t));
    memcpy(fill, start, (size_t)nsub * sizeof(uint64_t));
    for (uint64_t i = 0; i < k; ++i)
        tmp[fill[(pr_dst_hash((uint32_t)(keys[i] >> 32)) >> 8) % nsub]++] = keys[i];
    free(fill);
    uint64_t distinct = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+ : distinct)
    for (int64_t p = 0; p < (int64_t)nsub; ++p) {
        uint64_t* a = tmp + start[p];
        uint64_t len = start[p + 1] - start[p];
        qsort(a, len, sizeof(uint64_t), cmp_u64);
        for (uint64_t i = 0; i < len; ++i) {
            if (i > 0 && a[i] == a[i - 1]) continue;      /* duplicate edge */
            uint32_t u = (uint32_t)a[i], v = (uint32_t)(a[i] >> 32);
            ++distinct;
            if (mode == 0) {
                #pragma omp atomic
                outdeg[u] += 1;
            } else {
                for (uint32_t j = 0; j < nx; ++j)
                    s[j * n + v] += x[j * n + u] / (double)outdeg[u];
            }
        }
    }
    free(start);
    return distinct;
}
