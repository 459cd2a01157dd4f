// Learned-scheduler network (see mlp.cu).
#pragma once

#include "common.cuh"
#include "engine.cuh"

namespace seraph {

constexpr int kSchedIn = 16, kSchedHidden = 64, kSchedOut = 17;
constexpr int kSchedParams =
    kSchedHidden * kSchedIn + kSchedHidden + kSchedHidden * kSchedHidden + kSchedHidden +
    kSchedOut * kSchedHidden + kSchedOut;

struct SchedModel {
    bool fp32;                      // debug mode: forward with FP32 weights
    DevBuf<float> master, m, v;     // FP32 master weights and Adam moments
    DevBuf<uint16_t> w16;           // BF16 copy used by the forward pass
    DevBuf<float> part, loss_part, loss_dev;
    uint64_t adam_t = 0;

    SchedModel(uint64_t seed, bool fp32);
    void set_params(const float* host);
    void get_params(float* host) const;
    // x: n x 16 device features; outputs device arrays
    void infer(const float* x, uint64_t n, int32_t* kout, float* pout, cudaStream_t s) const;
    // mean loss over the n samples idx[0..n) (idx null: 0..n-1); gradient to grad_dev
    float loss_grad(const float* x, const int32_t* k, const float* p, const uint32_t* idx, uint64_t n,
                    float* grad_dev, cudaStream_t s);
    void adam(const float* grad_dev, float lr, cudaStream_t s);
};

// Inputs of the per-step and per-sweep scheduler kernels.
struct SchedArgs {
    const ChunkStatic* cs;
    const ChunkDyn* cd;
    const RunState* rs;
    float inv_n;      // 1 / vertices
    float is_pr;      // 1 for PageRank
    float predict;    // 1 if prediction is on in this sweep
    float sweep;      // sweep index
};

// Step start: the 16 features of `chunk` (into feat_row if not null) and, if
// `model` is not null, its predicted pass count into rs->k_limit; resets the
// step's pass counter.
void launch_sched_step(const SchedArgs& a, RunState* rs, uint32_t chunk, float* feat_row,
                       const SchedModel* model, cudaStream_t s);
// Features of chunks 0..C-1 into feats (C x 16).
void launch_sched_features(const SchedArgs& a, uint32_t C, float* feats, cudaStream_t s);

}  // namespace seraph

// The opaque handle of the C ABI.
struct seraph_sched_model {
    int device = 0;
    seraph::SchedModel model;
    seraph_sched_model(uint64_t seed, bool fp32) : model(seed, fp32) {}
};
