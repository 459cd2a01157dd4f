// Learned scheduler network: a 16 -> 64 -> 64 -> 17 MLP with GELU, BF16
// weights (FP32 master copy) and FP32 accumulation.  Outputs 0..15 are the
// logits of the number of local passes k = 1..16 for a pipeline step; output
// 16 is the chunk's streaming priority (its predicted first-pass gain).
//
// Training minimises mean over a batch of
//   CE(softmax(o[0..15]), k - 1) + (o[16] - priority)^2
// with Adam.  One CTA handles a tile of 32 samples: forward into shared
// memory, backward, and per-tile weight-gradient partials that a second
// kernel sums in a fixed order (deterministic).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.cuh"

namespace seraph {
namespace {

constexpr int IN = kSchedIn, HID = kSchedHidden, OUT = kSchedOut;
constexpr int TILE = 32;
constexpr int NT = 256;

struct Off {  // parameter offsets in the flat vector
    static constexpr int W1 = 0, B1 = W1 + HID * IN, W2 = B1 + HID, B2 = W2 + HID * HID,
                         W3 = B2 + HID, B3 = W3 + OUT * HID, N = B3 + OUT;
};
static_assert(Off::N == kSchedParams, "parameter count");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// Weights as used by the forward pass: the BF16 copy (or FP32 in debug mode).
template <bool FP32>
__device__ __forceinline__ void load_weights(const float* master, const __nv_bfloat16* w16, float* s_w) {
    for (int i = threadIdx.x; i < Off::N; i += blockDim.x)
        s_w[i] = FP32 ? master[i] : __bfloat162float(w16[i]);
}

// Forward for `cnt` samples of a tile into shared memory.
__device__ void tile_forward(const float* s_w, const float* s_x, int cnt, float* s_z1, float* s_h1,
                             float* s_z2, float* s_h2, float* s_o) {
    for (int i = threadIdx.x; i < cnt * HID; i += blockDim.x) {
        const int b = i / HID, j = i % HID;
        float acc = s_w[Off::B1 + j];
#pragma unroll
        for (int k = 0; k < IN; ++k) acc = fmaf(s_w[Off::W1 + j * IN + k], s_x[b * IN + k], acc);
        s_z1[i] = acc;
        s_h1[i] = gelu(acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * HID; i += blockDim.x) {
        const int b = i / HID, j = i % HID;
        float acc = s_w[Off::B2 + j];
        for (int k = 0; k < HID; ++k) acc = fmaf(s_w[Off::W2 + j * HID + k], s_h1[b * HID + k], acc);
        s_z2[i] = acc;
        s_h2[i] = gelu(acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * OUT; i += blockDim.x) {
        const int b = i / OUT, j = i % OUT;
        float acc = s_w[Off::B3 + j];
        for (int k = 0; k < HID; ++k) acc = fmaf(s_w[Off::W3 + j * HID + k], s_h2[b * HID + k], acc);
        s_o[i] = acc;
    }
    __syncthreads();
}

constexpr size_t kTileSmem =
    sizeof(float) * (Off::N + TILE * IN + 4 * TILE * HID + TILE * OUT + 2 * TILE * HID + TILE * OUT + TILE);

// Loss and weight-gradient partials of one tile (samples idx[tile*TILE ...]).
template <bool FP32>
__global__ void __launch_bounds__(NT) fwd_bwd_kernel(const float* __restrict__ master,
                                                     const __nv_bfloat16* __restrict__ w16,
                                                     const float* __restrict__ x,
                                                     const int32_t* __restrict__ ktgt,
                                                     const float* __restrict__ ptgt,
                                                     const uint32_t* __restrict__ idx, uint64_t n,
                                                     float inv_batch, float* __restrict__ part,
                                                     float* __restrict__ loss_part) {
    extern __shared__ float sm[];
    float* s_w = sm;
    float* s_x = s_w + Off::N;
    float* s_z1 = s_x + TILE * IN;
    float* s_h1 = s_z1 + TILE * HID;
    float* s_z2 = s_h1 + TILE * HID;
    float* s_h2 = s_z2 + TILE * HID;
    float* s_o = s_h2 + TILE * HID;
    float* s_d2 = s_o + TILE * OUT;   // dL/dz2
    float* s_d1 = s_d2 + TILE * HID;  // dL/dz1
    float* s_do = s_d1 + TILE * HID;  // dL/do
    float* s_loss = s_do + TILE * OUT;

    const uint64_t t0 = (uint64_t)blockIdx.x * TILE;
    const int cnt = (int)(n - t0 < (uint64_t)TILE ? n - t0 : (uint64_t)TILE);
    load_weights<FP32>(master, w16, s_w);
    for (int i = threadIdx.x; i < TILE * IN; i += blockDim.x) {
        const int b = i / IN;
        s_x[i] = b < cnt ? x[(uint64_t)(idx ? idx[t0 + b] : t0 + b) * IN + (i % IN)] : 0.f;
    }
    __syncthreads();
    tile_forward(s_w, s_x, cnt, s_z1, s_h1, s_z2, s_h2, s_o);

    // output gradient: softmax cross-entropy over 16 logits, squared error on o[16]
    if (threadIdx.x < cnt) {
        const int b = threadIdx.x;
        const uint64_t s = idx ? idx[t0 + b] : t0 + b;
        const float* o = s_o + b * OUT;
        float mx = o[0];
        for (int j = 1; j < 16; ++j) mx = fmaxf(mx, o[j]);
        float se = 0.f;
        for (int j = 0; j < 16; ++j) se += expf(o[j] - mx);
        const int k = min(max(ktgt[s], 1), 16) - 1;
        const float diff = o[16] - ptgt[s];
        s_loss[b] = (logf(se) + mx - o[k]) + diff * diff;
        for (int j = 0; j < 16; ++j) s_do[b * OUT + j] = (expf(o[j] - mx) / se - (j == k ? 1.f : 0.f)) * inv_batch;
        s_do[b * OUT + 16] = 2.f * diff * inv_batch;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * HID; i += blockDim.x) {  // dz2 = (W3^T do) * gelu'(z2)
        const int b = i / HID, j = i % HID;
        float acc = 0.f;
        for (int o = 0; o < OUT; ++o) acc = fmaf(s_w[Off::W3 + o * HID + j], s_do[b * OUT + o], acc);
        s_d2[i] = acc * gelu_grad(s_z2[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * HID; i += blockDim.x) {  // dz1 = (W2^T dz2) * gelu'(z1)
        const int b = i / HID, j = i % HID;
        float acc = 0.f;
        for (int o = 0; o < HID; ++o) acc = fmaf(s_w[Off::W2 + o * HID + j], s_d2[b * HID + o], acc);
        s_d1[i] = acc * gelu_grad(s_z1[i]);
    }
    __syncthreads();
    // weight-gradient partials of this tile (sum over its samples, fixed order)
    float* g = part + (uint64_t)blockIdx.x * Off::N;
    for (int p = threadIdx.x; p < Off::N; p += blockDim.x) {
        float acc = 0.f;
        if (p < Off::B1) {
            const int j = p / IN, k = p % IN;
            for (int b = 0; b < cnt; ++b) acc = fmaf(s_d1[b * HID + j], s_x[b * IN + k], acc);
        } else if (p < Off::W2) {
            for (int b = 0; b < cnt; ++b) acc += s_d1[b * HID + (p - Off::B1)];
        } else if (p < Off::B2) {
            const int q = p - Off::W2, j = q / HID, k = q % HID;
            for (int b = 0; b < cnt; ++b) acc = fmaf(s_d2[b * HID + j], s_h1[b * HID + k], acc);
        } else if (p < Off::W3) {
            for (int b = 0; b < cnt; ++b) acc += s_d2[b * HID + (p - Off::B2)];
        } else if (p < Off::B3) {
            const int q = p - Off::W3, j = q / HID, k = q % HID;
            for (int b = 0; b < cnt; ++b) acc = fmaf(s_do[b * OUT + j], s_h2[b * HID + k], acc);
        } else {
            for (int b = 0; b < cnt; ++b) acc += s_do[b * OUT + (p - Off::B3)];
        }
        g[p] = acc;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int b = 0; b < cnt; ++b) l += s_loss[b];
        loss_part[blockIdx.x] = l;
    }
}

// grad[p] = sum over tiles of part[tile][p] (fixed order); loss likewise.
__global__ void reduce_grad_kernel(const float* __restrict__ part, int tiles, float* __restrict__ grad,
                                   const float* __restrict__ loss_part, float* loss, float inv_batch) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < Off::N) {
        float acc = 0.f;
        for (int t = 0; t < tiles; ++t) acc += part[(uint64_t)t * Off::N + p];
        grad[p] = acc;
    }
    if (p == 0) {
        float l = 0.f;
        for (int t = 0; t < tiles; ++t) l += loss_part[t];
        *loss = l * inv_batch;
    }
}

__global__ void adam_kernel(float* __restrict__ master, __nv_bfloat16* __restrict__ w16,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Off::N) return;
    const float gp = grad[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float w = master[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
    master[p] = w;
    w16[p] = __float2bfloat16_rn(w);
}

__global__ void to_bf16_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ w16) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < Off::N) w16[p] = __float2bfloat16_rn(master[p]);
}

template <bool FP32>
__global__ void __launch_bounds__(NT) infer_kernel(const float* __restrict__ master,
                                                   const __nv_bfloat16* __restrict__ w16,
                                                   const float* __restrict__ x, uint64_t n,
                                                   int32_t* __restrict__ kout,
                                                   float* __restrict__ pout) {
    extern __shared__ float sm[];
    float* s_w = sm;
    float* s_x = s_w + Off::N;
    float* s_z1 = s_x + TILE * IN;
    float* s_h1 = s_z1 + TILE * HID;
    float* s_z2 = s_h1 + TILE * HID;
    float* s_h2 = s_z2 + TILE * HID;
    float* s_o = s_h2 + TILE * HID;
    const uint64_t t0 = (uint64_t)blockIdx.x * TILE;
    const int cnt = (int)(n - t0 < (uint64_t)TILE ? n - t0 : (uint64_t)TILE);
    load_weights<FP32>(master, w16, s_w);
    for (int i = threadIdx.x; i < TILE * IN; i += blockDim.x) {
        const int b = i / IN;
        s_x[i] = b < cnt ? x[(t0 + b) * IN + (i % IN)] : 0.f;
    }
    __syncthreads();
    tile_forward(s_w, s_x, cnt, s_z1, s_h1, s_z2, s_h2, s_o);
    if (threadIdx.x < cnt) {
        const float* o = s_o + threadIdx.x * OUT;
        int best = 0;
        for (int j = 1; j < 16; ++j)
            if (o[j] > o[best]) best = j;  // first maximum wins
        kout[t0 + threadIdx.x] = best + 1;
        pout[t0 + threadIdx.x] = o[16];
    }
}

// The 16 features of a chunk at a step (all scaled to about [0, 1]).
__device__ void chunk_features(const SchedArgs& a, uint32_t c, float* f) {
    const ChunkStatic st = a.cs[c];
    const ChunkDyn d = a.cd[c];
    const float nv = fmaxf(st.nv, 1.f);
    f[0] = a.is_pr;
    f[1] = log2f(1.f + st.nv) / 32.f;
    f[2] = log2f(1.f + st.ne) / 36.f;
    f[3] = fminf(st.ne / nv, 256.f) / 256.f;
    f[4] = log2f(1.f + st.maxdeg) / 32.f;
    f[5] = st.bytes_frac;
    f[6] = fminf((float)d.visits, 64.f) / 64.f;
    f[7] = fminf(a.sweep, 64.f) / 64.f;
    for (int k = 0; k < 4; ++k) f[8 + k] = fminf((float)d.gains[k] / nv, 1.f);
    f[12] = fminf((float)a.rs->prev_changed * a.inv_n, 1.f);
    f[13] = fminf((float)a.rs->cur.changed * a.inv_n, 1.f);
    f[14] = fminf((float)d.last_passes, 16.f) / 16.f;
    f[15] = a.predict;
}

__global__ void sched_step_kernel(SchedArgs a, RunState* rs, uint32_t chunk, float* feat_row,
                                  const float* __restrict__ master,
                                  const __nv_bfloat16* __restrict__ w16, int use_model, int fp32) {
    __shared__ float f[IN], h1[HID], h2[HID], o[OUT];
    if (threadIdx.x == 0) {
        chunk_features(a, chunk, f);
        if (feat_row)
            for (int k = 0; k < IN; ++k) feat_row[k] = f[k];
        rs->step_passes = 0;
    }
    __syncthreads();
    if (!use_model) return;
    auto W = [&](int i) { return fp32 ? master[i] : __bfloat162float(w16[i]); };
    const int j = threadIdx.x;  // 64 threads: one hidden unit each
    float acc = W(Off::B1 + j);
    for (int k = 0; k < IN; ++k) acc = fmaf(W(Off::W1 + j * IN + k), f[k], acc);
    h1[j] = gelu(acc);
    __syncthreads();
    acc = W(Off::B2 + j);
    for (int k = 0; k < HID; ++k) acc = fmaf(W(Off::W2 + j * HID + k), h1[k], acc);
    h2[j] = gelu(acc);
    __syncthreads();
    if (j < OUT) {
        acc = W(Off::B3 + j);
        for (int k = 0; k < HID; ++k) acc = fmaf(W(Off::W3 + j * HID + k), h2[k], acc);
        o[j] = acc;
    }
    __syncthreads();
    if (j == 0) {
        int best = 0;
        for (int q = 1; q < 16; ++q)
            if (o[q] > o[best]) best = q;
        rs->k_limit = (unsigned)(best + 1);
    }
}

__global__ void sched_features_kernel(SchedArgs a, uint32_t C, float* feats) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) chunk_features(a, c, feats + (uint64_t)c * IN);
}

uint64_t splitmix(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

SchedModel::SchedModel(uint64_t seed, bool fp32_) : fp32(fp32_) {
    master.alloc(Off::N);
    w16.alloc(Off::N);
    m.alloc(Off::N);
    v.alloc(Off::N);
    std::vector<float> h(Off::N, 0.f);
    // Glorot-uniform weights from a seeded splitmix64 stream, zero biases.
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) {
            const double u = (splitmix(seed, (uint64_t)(off + i)) >> 11) * (1.0 / 9007199254740992.0);
            h[off + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    fill(Off::W1, HID, IN);
    fill(Off::W2, HID, HID);
    fill(Off::W3, OUT, HID);
    set_params(h.data());
}

void SchedModel::set_params(const float* host) {
    SR_CUDA(cudaMemcpy(master.p, host, Off::N * sizeof(float), cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemset(m.p, 0, Off::N * sizeof(float)));
    SR_CUDA(cudaMemset(v.p, 0, Off::N * sizeof(float)));
    to_bf16_kernel<<<(Off::N + 255) / 256, 256>>>(master.p, (__nv_bfloat16*)w16.p);
    SR_LAUNCH();
    SR_CUDA(cudaDeviceSynchronize());
    adam_t = 0;
}

void SchedModel::get_params(float* host) const {
    SR_CUDA(cudaMemcpy(host, master.p, Off::N * sizeof(float), cudaMemcpyDeviceToHost));
}

void SchedModel::infer(const float* x, uint64_t n, int32_t* kout, float* pout, cudaStream_t s) const {
    if (n == 0) return;
    static bool attr = false;
    if (!attr) {
        SR_CUDA(cudaFuncSetAttribute(infer_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem));
        SR_CUDA(cudaFuncSetAttribute(infer_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem));
        attr = true;
    }
    const unsigned tiles = (unsigned)((n + TILE - 1) / TILE);
    if (fp32) infer_kernel<true><<<tiles, NT, kTileSmem, s>>>(master.p, (const __nv_bfloat16*)w16.p, x, n, kout, pout);
    else infer_kernel<false><<<tiles, NT, kTileSmem, s>>>(master.p, (const __nv_bfloat16*)w16.p, x, n, kout, pout);
    SR_LAUNCH();
}

float SchedModel::loss_grad(const float* x, const int32_t* k, const float* p, const uint32_t* idx,
                            uint64_t n, float* grad_dev, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        SR_CUDA(cudaFuncSetAttribute(fwd_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem));
        SR_CUDA(cudaFuncSetAttribute(fwd_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem));
        attr = true;
    }
    const int tiles = (int)((n + TILE - 1) / TILE);
    if ((uint64_t)tiles * Off::N > part.n) part.alloc((uint64_t)tiles * Off::N);
    if ((uint64_t)tiles > loss_part.n) loss_part.alloc(tiles);
    if (!loss_dev.p) loss_dev.alloc(1);
    const float inv = 1.f / (float)n;
    if (fp32)
        fwd_bwd_kernel<true><<<tiles, NT, kTileSmem, s>>>(master.p, (const __nv_bfloat16*)w16.p, x, k, p, idx, n, inv, part.p, loss_part.p);
    else
        fwd_bwd_kernel<false><<<tiles, NT, kTileSmem, s>>>(master.p, (const __nv_bfloat16*)w16.p, x, k, p, idx, n, inv, part.p, loss_part.p);
    reduce_grad_kernel<<<(Off::N + 255) / 256, 256, 0, s>>>(part.p, tiles, grad_dev, loss_part.p, loss_dev.p, inv);
    SR_LAUNCH();
    float loss = 0.f;
    SR_CUDA(cudaMemcpyAsync(&loss, loss_dev.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    SR_CUDA(cudaStreamSynchronize(s));
    return loss;
}

void launch_sched_step(const SchedArgs& a, RunState* rs, uint32_t chunk, float* feat_row,
                       const SchedModel* model, cudaStream_t s) {
    sched_step_kernel<<<1, HID, 0, s>>>(a, rs, chunk, feat_row, model ? model->master.p : nullptr,
                                        model ? (const __nv_bfloat16*)model->w16.p : nullptr,
                                        model ? 1 : 0, model && model->fp32 ? 1 : 0);
    SR_LAUNCH();
}

void launch_sched_features(const SchedArgs& a, uint32_t C, float* feats, cudaStream_t s) {
    sched_features_kernel<<<(C + 127) / 128, 128, 0, s>>>(a, C, feats);
    SR_LAUNCH();
}

void SchedModel::adam(const float* grad_dev, float lr, cudaStream_t s) {
    ++adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)adam_t), c2 = 1.f - std::pow(b2, (float)adam_t);
    adam_kernel<<<(Off::N + 255) / 256, 256, 0, s>>>(master.p, (__nv_bfloat16*)w16.p, m.p, v.p, grad_dev, lr, b1, b2, 1e-8f, c1, c2);
    SR_LAUNCH();
}

}  // namespace seraph
