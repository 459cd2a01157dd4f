// extern "C" entry points of include/seraph.h.  Every call catches
// exceptions, records a thread-local message and returns a SERAPH_E* code.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>
#include <new>
#include <string>

#include "graph.hpp"
#include "mlp.cuh"


namespace seraph {
int run_graph(seraph_graph* g, const seraph_params* P, void* out, int out_mem, seraph_stats* st);
void bgraph_build(seraph_bgraph* g, uint64_t n, uint64_t m, const uint32_t* src,
                  const uint32_t* dst, const uint32_t* w, int mem, cudaStream_t s);
int batch_run(seraph_bgraph* const* graphs, uint32_t ng, const seraph_query* q, uint32_t nq,
              int out_mem, const seraph_batch_params* P, seraph_batch_stats* st);
int batch_plan_create(seraph_bgraph* const* graphs, uint32_t ng, const seraph_query* q, uint32_t nq,
                      const seraph_batch_params* P, seraph_batch_plan** out);
int batch_plan_run(seraph_batch_plan* plan, const uint32_t* sources, seraph_batch_stats* st);
void batch_plan_free(seraph_batch_plan* plan);
}


namespace {

thread_local std::string g_last_error;

template <class F>
int guarded(F&& f) {
    try {
        g_last_error.clear();
        return f();
    } catch (const seraph::Error& e) {
        g_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return SERAPH_ENOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return SERAPH_EINVAL;
    } catch (...) {
        g_last_error = "unknown error";
        return SERAPH_EINVAL;
    }
}

}  // namespace

namespace seraph {
void set_last_error(const char* msg) { g_last_error = msg; }

namespace {
std::atomic<int64_t> g_pinned_fail_in{0};   // 0: off; k: the k-th allocation from now fails
std::atomic<int64_t> g_pinned_bytes{0};
}  // namespace

bool take_injected_pinned_failure() {
    int64_t k = g_pinned_fail_in.load();
    while (k > 0) {
        if (g_pinned_fail_in.compare_exchange_weak(k, k - 1)) return k == 1;
    }
    return false;
}

void note_pinned_bytes(int64_t delta) { g_pinned_bytes += delta; }

namespace {
std::mutex g_l2_mu;
std::set<const void*> g_l2_holders;
bool g_l2_raised = false;
size_t g_l2_orig = 0, g_l2_now = 0;
}  // namespace

void l2_setaside_hold(const void* holder, int device, uint64_t bytes) {
    std::lock_guard<std::mutex> lk(g_l2_mu);
    int maxp = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, device) != cudaSuccess ||
        maxp <= 0) {
        (void)cudaGetLastError();
        return;
    }
    const size_t want = bytes < (uint64_t)maxp ? (size_t)bytes : (size_t)maxp;
    if (!g_l2_raised) {
        if (cudaDeviceGetLimit(&g_l2_orig, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        g_l2_now = g_l2_orig;
    }
    if (g_l2_now < want) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        g_l2_now = want;
        g_l2_raised = true;
    }
    if (g_l2_raised) g_l2_holders.insert(holder);
}

void l2_setaside_drop(const void* holder) {
    std::lock_guard<std::mutex> lk(g_l2_mu);
    if (!g_l2_holders.erase(holder) || !g_l2_holders.empty() || !g_l2_raised) return;
    (void)cudaCtxResetPersistingL2Cache();
    (void)cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_orig);
    (void)cudaGetLastError();
    g_l2_raised = false;
}
}  // namespace seraph

extern "C" {

const char* seraph_last_error(void) { return g_last_error.c_str(); }

const char* seraph_version(void) { return "seraph-b300 0.1 (sm_103a)"; }

int seraph_debug_fail_pinned_alloc(uint32_t k) {
    seraph::g_pinned_fail_in.store((int64_t)k);
    return SERAPH_OK;
}

uint64_t seraph_debug_pinned_bytes(void) {
    const int64_t b = seraph::g_pinned_bytes.load();
    return b > 0 ? (uint64_t)b : 0u;
}

int seraph_debug_l2_setaside(uint64_t* bytes) {
    return guarded([&] {
        SR_CHECK(bytes, SERAPH_EINVAL, "bytes must not be NULL");
        size_t v = 0;
        SR_CUDA(cudaDeviceGetLimit(&v, cudaLimitPersistingL2CacheSize));
        *bytes = v;
        return SERAPH_OK;
    });
}

int seraph_graph_from_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            const uint32_t* w, int mem, uint32_t flags, uint32_t num_pages,
                            void* stream, seraph_graph** out) {
    return guarded([&] {
        SR_CHECK(out != nullptr, SERAPH_EINVAL, "out must not be NULL");
        *out = nullptr;
        seraph::Stream s;
        s.use(stream);
        seraph_graph* g = new seraph_graph();
        try {
            seraph::build_graph(g, n, m, src, dst, w, mem, flags, num_pages, s.s);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
        return SERAPH_OK;
    });
}

int seraph_graph_from_csr(uint64_t n, const uint64_t* row_off, const uint32_t* col,
                          const uint32_t* w, int mem, uint32_t flags, uint32_t num_pages,
                          void* stream, seraph_graph** out) {
    return guarded([&] {
        SR_CHECK(out != nullptr, SERAPH_EINVAL, "out must not be NULL");
        *out = nullptr;
        // host offsets are checked before any device work (device offsets by
        // a kernel in build_graph_csr)
        if (mem == SERAPH_MEM_HOST) seraph::check_csr_offsets_host(n, row_off);
        seraph::Stream s;
        s.use(stream);
        seraph_graph* g = new seraph_graph();
        try {
            seraph::build_graph_csr(g, n, row_off, col, w, mem, flags, num_pages, s.s);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
        return SERAPH_OK;
    });
}

int seraph_graph_get_info(const seraph_graph* g, seraph_graph_info* info) {
    return guarded([&] {
        SR_CHECK(g && info, SERAPH_EINVAL, "null argument");
        std::memset(info, 0, sizeof(*info));
        info->n = g->n;
        info->m_raw = g->m_raw;
        info->m = g->m;
        info->struct_bytes = g->h_struct.bytes;
        info->weight_bytes = g->h_weight.bytes;
        for (const auto& p : g->pages) {
            info->max_page_struct_bytes = std::max(info->max_page_struct_bytes, p.s_bytes);
            info->max_page_weight_bytes = std::max(info->max_page_weight_bytes, p.w_bytes);
        }
        info->num_pages = g->num_pages;
        info->weighted = g->weighted;
        info->symmetrized = g->symmetrized;
        info->max_in_degree = g->max_in_degree;
        info->weight_width = g->weighted ? g->wbytes : 0;
        info->reordered = g->reordered;
        info->packed = g->packed;
        info->out_edge_bytes = g->h_out_off.bytes + g->h_out_col.bytes + g->h_out_w.bytes;
        if (g->packed) {
            info->packed_bytes = g->h_pack.bytes;
            for (const auto& p : g->pages) {
                info->packed_data_bytes += p.pk_data;
                info->max_page_packed_bytes = std::max(info->max_page_packed_bytes, p.pk_bytes);
            }
        }
        return SERAPH_OK;
    });
}

int seraph_graph_page_bounds(const seraph_graph* g, uint64_t* vb) {
    return guarded([&] {
        SR_CHECK(g && vb, SERAPH_EINVAL, "null argument");
        std::memcpy(vb, g->vb.data(), g->vb.size() * sizeof(uint64_t));
        return SERAPH_OK;
    });
}

int seraph_graph_export_csc(const seraph_graph* g, uint64_t* col_off, uint32_t* row, uint32_t* w,
                            uint32_t* out_degree) {
    return guarded([&] {
        SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
        SR_CHECK(w == nullptr || g->weighted, SERAPH_EINVAL, "graph has no weights");
        seraph::export_csc(g, col_off, row, w, out_degree);
        return SERAPH_OK;
    });
}

int seraph_graph_export_perm(const seraph_graph* g, uint32_t* perm) {
    return guarded([&] {
        SR_CHECK(g && perm, SERAPH_EINVAL, "null argument");
        if (g->reordered) {
            SR_CUDA(cudaSetDevice(g->device));
            SR_CUDA(cudaMemcpy(perm, g->d_perm.p, g->n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        } else {
            for (uint64_t i = 0; i < g->n; ++i) perm[i] = (uint32_t)i;
        }
        return SERAPH_OK;
    });
}

int seraph_graph_export_packed(const seraph_graph* g, uint64_t* boff, uint8_t* data) {
    return guarded([&] {
        SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
        SR_CHECK(g->packed, SERAPH_EINVAL, "graph was built without SERAPH_COMPRESS");
        uint64_t base = 0;
        for (const auto& pm : g->pages) {
            const uint8_t* h = g->h_pack.p + pm.pk_off;
            const uint32_t* rel = (const uint32_t*)(h + pm.off_bytes);
            if (boff)
                for (uint64_t i = 0; i < pm.nv; ++i) boff[pm.vb + i] = base + rel[i];
            if (data && pm.pk_data) std::memcpy(data + base, h + 2 * pm.off_bytes, pm.pk_data);
            base += pm.pk_data;
        }
        if (boff) boff[g->n] = base;
        return SERAPH_OK;
    });
}

int seraph_graph_export_out_edges(const seraph_graph* g, uint64_t* out_off, uint32_t* out_col,
                                  uint32_t* out_w) {
    return guarded([&] {
        SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
        SR_CHECK(g->out_edges, SERAPH_EINVAL, "graph was built without SERAPH_OUT_EDGES");
        if (out_off) std::memcpy(out_off, g->h_out_off.p, 8 * (g->n + 1));
        if (out_col && g->m) std::memcpy(out_col, g->h_out_col.p, 4 * g->m);
        if (out_w && g->weighted && g->m) {
            for (uint64_t i = 0; i < g->m; ++i) {
                uint32_t x = 0;
                std::memcpy(&x, g->h_out_w.p + i * g->wbytes, g->wbytes);  // little-endian widths
                out_w[i] = x;
            }
        }
        return SERAPH_OK;
    });
}

int seraph_graph_release_buffers(seraph_graph* g) {
    return guarded([&] {
        SR_CHECK(g != nullptr, SERAPH_EINVAL, "null graph");
        std::lock_guard<std::mutex> lk(g->ws.m);
        SR_CUDA(cudaSetDevice(g->device));
        g->ws.release();
        seraph::l2_setaside_drop(g);
        return SERAPH_OK;
    });
}

void seraph_graph_free(seraph_graph* g) {
    if (!g) return;
    try {
        cudaSetDevice(g->device);
        seraph::l2_setaside_drop(g);
        delete g;
    } catch (...) {
    }
}

int seraph_params_default(seraph_params* p, int algo) {
    return guarded([&] {
        SR_CHECK(p != nullptr, SERAPH_EINVAL, "null params");
        std::memset(p, 0, sizeof(*p));
        p->algo = algo;
        p->source = 0;
        p->budget_bytes = 2ull << 30;
        p->window = 4;
        p->passes = 1;
        p->pvu = SERAPH_PVU_OFF;
        p->verify = 1;
        // Weak state machine (Fig. 6): 0,1,5 attempt; 2,3,4 are dormant.
        //   0 -ok-> 0, 0 -fail-> 5;   5 -ok-> 0, 5 -fail-> 3;
        //   3 -> 2 -> 1 (two dormant passes);  1 -ok-> 0, 1 -fail-> 4;
        //   4 -> 3 (punishment: one more dormant pass).
        // Column 1 of a dormant state is its valid-update edge (-> 0).
        const uint8_t fsm[12] = {5, 0, 4, 0, 1, 0, 2, 0, 3, 0, 3, 0};
        std::memcpy(p->fsm_next, fsm, 12);
        p->fsm_skip_mask = (1u << 2) | (1u << 3) | (1u << 4);
        p->kahan = 1;
        p->pr_normalize = 1;
        p->max_sweeps = algo == SERAPH_PAGERANK ? 100 : 1000000;
        p->damping = 0.85;
        p->tol = 1e-7;
        p->pr_fail_eps = 1.0 / (1 << 20);
        p->pr_pvu_off_below = 1e-6;
        p->thread_max_deg = 8;
        p->group4_max_deg = 32;
        p->group8_max_deg = 128;
        p->warp_max_deg = 4096;
        p->sched = SERAPH_SCHED_FIXED;
        p->timeout_ms = 600000;
        p->l2_hot_bytes = SERAPH_L2_HOT_AUTO;
        p->pr_omega = 1.0;
        return SERAPH_OK;
    });
}

int seraph_run(seraph_graph* g, const seraph_params* p, void* out_values, int out_mem,
               seraph_stats* stats) {
    return guarded([&] { return seraph::run_graph(g, p, out_values, out_mem, stats); });
}

}  // extern "C"

// ------------------------------------------------------ learned scheduler

namespace {

template <class T>
const T* dev_input(const T* p, uint64_t count, int mem, seraph::DevBuf<T>& hold) {
    if (mem == SERAPH_MEM_DEVICE) return p;
    hold.alloc(count ? count : 1);
    if (count) SR_CUDA(cudaMemcpy(hold.p, p, count * sizeof(T), cudaMemcpyHostToDevice));
    return hold.p;
}

uint64_t mix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int seraph_sched_create(uint64_t seed, int fp32, seraph_sched_model** out) {
    return guarded([&] {
        SR_CHECK(out != nullptr, SERAPH_EINVAL, "out must not be NULL");
        *out = nullptr;
        int dev = 0;
        SR_CUDA(cudaGetDevice(&dev));
        auto* m = new seraph_sched_model(seed, fp32 != 0);
        m->device = dev;
        *out = m;
        return SERAPH_OK;
    });
}

int seraph_sched_get_params(const seraph_sched_model* m, float* params) {
    return guarded([&] {
        SR_CHECK(m && params, SERAPH_EINVAL, "null argument");
        m->model.get_params(params);
        return SERAPH_OK;
    });
}

int seraph_sched_set_params(seraph_sched_model* m, const float* params) {
    return guarded([&] {
        SR_CHECK(m && params, SERAPH_EINVAL, "null argument");
        m->model.set_params(params);
        return SERAPH_OK;
    });
}

int seraph_sched_loss_grad(seraph_sched_model* m, const float* x, const int32_t* k,
                           const float* prio, uint64_t n, int mem, float* loss, float* grad) {
    return guarded([&] {
        SR_CHECK(m && x && k && prio && n > 0, SERAPH_EINVAL, "null argument or n == 0");
        seraph::DevBuf<float> hx, hp, g(SERAPH_SCHED_PARAMS);
        seraph::DevBuf<int32_t> hk;
        const float* dx = dev_input(x, n * SERAPH_SCHED_FEATURES, mem, hx);
        const int32_t* dk = dev_input(k, n, mem, hk);
        const float* dp = dev_input(prio, n, mem, hp);
        const float l = m->model.loss_grad(dx, dk, dp, nullptr, n, g.p, nullptr);
        if (loss) *loss = l;
        if (grad) SR_CUDA(cudaMemcpy(grad, g.p, SERAPH_SCHED_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
        return SERAPH_OK;
    });
}

int seraph_sched_train(seraph_sched_model* m, const float* x, const int32_t* k, const float* prio,
                       uint64_t n, int mem, uint32_t epochs, uint32_t batch, float lr,
                       uint64_t seed, float* losses) {
    return guarded([&] {
        SR_CHECK(m && x && k && prio && n > 0 && batch > 0, SERAPH_EINVAL, "bad arguments");
        SR_CHECK(n < (1ull << 32), SERAPH_EINVAL, "too many samples");
        seraph::DevBuf<float> hx, hp, g(SERAPH_SCHED_PARAMS);
        seraph::DevBuf<int32_t> hk;
        const float* dx = dev_input(x, n * SERAPH_SCHED_FEATURES, mem, hx);
        const int32_t* dk = dev_input(k, n, mem, hk);
        const float* dp = dev_input(prio, n, mem, hp);
        std::vector<uint32_t> perm(n);
        seraph::DevBuf<uint32_t> didx(n);
        for (uint32_t e = 0; e < epochs; ++e) {
            for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
            for (uint64_t i = n - 1; i > 0; --i) {  // seeded Fisher-Yates shuffle
                const uint64_t j = mix64(seed, e * n + i) % (i + 1);
                std::swap(perm[i], perm[j]);
            }
            SR_CUDA(cudaMemcpy(didx.p, perm.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice));
            double sum = 0.0;
            uint64_t nb = 0;
            for (uint64_t off = 0; off < n; off += batch, ++nb) {
                const uint64_t cnt = std::min<uint64_t>(batch, n - off);
                sum += m->model.loss_grad(dx, dk, dp, didx.p + off, cnt, g.p, nullptr);
                m->model.adam(g.p, lr, nullptr);
            }
            if (losses) losses[e] = (float)(sum / (double)nb);
        }
        SR_CUDA(cudaDeviceSynchronize());
        return SERAPH_OK;
    });
}

int seraph_sched_infer(const seraph_sched_model* m, const float* x, uint64_t n, int mem,
                       int32_t* k_out, float* prio_out) {
    return guarded([&] {
        SR_CHECK(m && x && k_out && prio_out, SERAPH_EINVAL, "null argument");
        if (n == 0) return SERAPH_OK;
        seraph::DevBuf<float> hx, hp;
        seraph::DevBuf<int32_t> hk;
        const float* dx = dev_input(x, n * SERAPH_SCHED_FEATURES, mem, hx);
        int32_t* dk = k_out;
        float* dp = prio_out;
        if (mem != SERAPH_MEM_DEVICE) { hk.alloc(n); hp.alloc(n); dk = hk.p; dp = hp.p; }
        m->model.infer(dx, n, dk, dp, nullptr);
        if (mem != SERAPH_MEM_DEVICE) {
            SR_CUDA(cudaMemcpy(k_out, dk, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
            SR_CUDA(cudaMemcpy(prio_out, dp, n * sizeof(float), cudaMemcpyDeviceToHost));
        }
        SR_CUDA(cudaDeviceSynchronize());
        return SERAPH_OK;
    });
}

int seraph_sched_targets(const seraph_trace* t, float share, int32_t* k_out, float* prio_out) {
    return guarded([&] {
        SR_CHECK(t && k_out && prio_out, SERAPH_EINVAL, "null argument");
        SR_CHECK(share > 0.f && share <= 1.f, SERAPH_EINVAL, "share must be in (0, 1]");
        for (uint64_t r = 0; r < t->count; ++r) {
            const uint32_t* g = t->gains + r * SERAPH_SCHED_FEATURES;
            double total = 0.0;
            for (int j = 0; j < 16; ++j) total += g[j];
            int k = 1;
            double acc = g[0];
            while (k < 16 && acc < share * total) acc += g[k++];
            k_out[r] = k;
            prio_out[r] = (float)(std::log2(1.0 + g[0]) / 24.0);
        }
        return SERAPH_OK;
    });
}

void seraph_sched_free(seraph_sched_model* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    delete m;
}

}  // extern "C"

// ------------------------------------------------------- batched queries

extern "C" {

int seraph_bgraph_from_edges(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                             const uint32_t* w, int mem, void* stream, seraph_bgraph** out) {
    return guarded([&] {
        SR_CHECK(out != nullptr, SERAPH_EINVAL, "out must not be NULL");
        *out = nullptr;
        seraph::Stream s;
        s.use(stream);
        auto* g = new seraph_bgraph();
        try {
            seraph::bgraph_build(g, n, m, src, dst, w, mem, s.s);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
        return SERAPH_OK;
    });
}

void seraph_bgraph_free(seraph_bgraph* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    delete g;
}

int seraph_batch_params_default(seraph_batch_params* p) {
    return guarded([&] {
        SR_CHECK(p != nullptr, SERAPH_EINVAL, "null params");
        std::memset(p, 0, sizeof(*p));
        p->mapping = SERAPH_MAP_AUTO;
        p->tile = 0;
        p->use_graph = 1;
        p->replays = 1;
        p->timeout_ms = 60000;
        p->group = 1;
        return SERAPH_OK;
    });
}

int seraph_batch_run(seraph_bgraph* const* graphs, uint32_t ng, const seraph_query* queries,
                     uint32_t nq, int out_mem, const seraph_batch_params* p,
                     seraph_batch_stats* stats) {
    return guarded([&] { return seraph::batch_run(graphs, ng, queries, nq, out_mem, p, stats); });
}

int seraph_batch_plan_create(seraph_bgraph* const* graphs, uint32_t ng, const seraph_query* queries,
                             uint32_t nq, const seraph_batch_params* p, seraph_batch_plan** out) {
    return guarded([&] { return seraph::batch_plan_create(graphs, ng, queries, nq, p, out); });
}

int seraph_batch_plan_run(seraph_batch_plan* plan, const uint32_t* sources, seraph_batch_stats* stats) {
    return guarded([&] { return seraph::batch_plan_run(plan, sources, stats); });
}

void seraph_batch_plan_free(seraph_batch_plan* plan) {
    try {
        seraph::batch_plan_free(plan);
    } catch (...) {
    }
}

}  // extern "C"
