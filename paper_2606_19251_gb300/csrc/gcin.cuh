// GCIN coefficient network (Sec. 3.2, App. A.1): parameter layout and the
// batched graph container shared by inference and training.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "ctx.cuh"

namespace amg {

constexpr int kHidden = 64;
constexpr int kLayers = 4;
constexpr int kRo = 32;          // readout width per layer
constexpr int kEmb = kRo * kLayers;   // 128
constexpr int kNumParams = 55045;

// Offsets of each tensor in the flat parameter vector (App. A.1 layout).
struct ParamLayout {
    int convW[kLayers], convB[kLayers];
    int inG[kLayers], inB[kLayers];
    int roW[kLayers], roB[kLayers];
    int lnG, lnB;
    int h1W, h1B, h2W, h2B, h3W, h3B;
    int total;
};

constexpr ParamLayout make_layout() {
    ParamLayout p{};
    int o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int fin = (l == 0) ? 2 : kHidden;
        p.convW[l] = o; o += fin * kHidden;
        p.convB[l] = o; o += kHidden;
    }
    for (int l = 0; l < kLayers; ++l) {
        p.inG[l] = o; o += kHidden;
        p.inB[l] = o; o += kHidden;
    }
    for (int l = 0; l < kLayers; ++l) {
        p.roW[l] = o; o += 2 * kHidden * kRo;
        p.roB[l] = o; o += kRo;
    }
    p.lnG = o; o += kEmb;
    p.lnB = o; o += kEmb;
    p.h1W = o; o += kEmb * 128;
    p.h1B = o; o += 128;
    p.h2W = o; o += 128 * 64;
    p.h2B = o; o += 64;
    p.h3W = o; o += 64 * 5;
    p.h3B = o; o += 5;
    p.total = o;
    return p;
}
constexpr ParamLayout kPL = make_layout();
static_assert(kPL.total == kNumParams, "GCIN layout must have 55,045 parameters (App. A.1)");

// Batch graph (Algorithm 1 steps 1-5): disjoint union of level graphs with
// node ranges gptr[g] .. gptr[g+1] and edges = the concatenated CSR patterns.
// Nodes are cut into tiles of at most kTile consecutive nodes that never
// cross a graph boundary; every reduction over a graph is a fixed-order
// combination of per-tile partials (deterministic, no atomics).
constexpr int kTile = 64;
constexpr int kChunkTiles = 64;
constexpr int kGradChunks = 64;      // tile chunks of the weight-gradient reduction

struct GcinBatch {
    int G = 0, N = 0, NT = 0;            // graphs, nodes, tiles
    int bf16 = 0;                        // layers 2..4 on tensor cores (BF16 operands, FP32 accumulation)
    int *err = nullptr;                  // device error flag (tensor-core wait timeout)
    long long E = 0;
    int *rp = nullptr, *col = nullptr, *gptr = nullptr, *gid = nullptr;
    int *tstart = nullptr, *tgraph = nullptr, *gtile = nullptr;   // tile -> first node / graph; graph -> first tile
    // chunks of up to kChunkTiles tiles of one graph: the per-graph
    // reductions run tiles -> chunks -> graph, every stage in parallel
    int NC = 0;
    int *ctile = nullptr, *cnode = nullptr, *gchunk = nullptr;      // chunk -> first tile / node; graph -> first chunk
    float *cmean = nullptr, *cm2 = nullptr, *cmax = nullptr;        // NC x 64 chunk statistics
    double *csum = nullptr;                                         // NC x 64
    int *carg = nullptr;                                            // NC x 64
    float *w = nullptr;
    double *w64 = nullptr;
    // activations (kept for the backward pass)
    double *x0 = nullptr;                // N x 2 raw features [a_ii, deg] (FP64)
    float *h1 = nullptr;                 // N x 2      layer-1 aggregation
    float *h[kLayers] = {};              // N x 64     layers 2..4 aggregation (h[0] unused)
    float *y[kLayers] = {};              // N x 64     linear outputs
    float *x[kLayers] = {};              // N x 64     ReLU(IN(y))
    float *mu[kLayers] = {}, *rstd[kLayers] = {};   // G x 64
    float *tmean = nullptr, *tm2 = nullptr;          // NT x 64 tile statistics of y
    double *tsum = nullptr;                          // NT x 64 tile sums (pooling / backward)
    double *tsum2 = nullptr;                         // NT x 64 second tile sums (backward)
    float *tmax = nullptr;                           // NT x 64
    int *targ = nullptr;                             // NT x 64
    float *pooled = nullptr;             // G x 4 x 128 (mean | max per layer)
    int *argmax = nullptr;               // G x 4 x 64  node index of each max
    float *head = nullptr;               // G x head scratch
    float *c = nullptr;                  // G x 5
    // backward work
    float *dc = nullptr;                 // G x 5
    float *dhead = nullptr;              // G x (dz1 128 | dz2 64 | dzh 128 | dz 128)
    float *dpooled = nullptr;            // G x 4 x 128
    float *dx = nullptr, *dh = nullptr, *dy = nullptr;   // N x 64
    double *gS1 = nullptr, *gS2 = nullptr;               // G x 64 per-graph sums
    float *dWt = nullptr;                // NT x (64 x 64 + 64) per-tile weight/bias gradient partials
    double *dWc = nullptr;               // kGradChunks x (64 x 64 + 64) chunk sums of dWt
    char *arena = nullptr;
    size_t bytes = 0;
};

void gcin_batch_free(GcinBatch &b);
// Build the batch from every level of every context; allocates device memory
// (with the backward buffers when `backward` is set).
int gcin_batch_build(GcinBatch &b, int n_problems, amg_ctx *const *problems, cudaStream_t s, std::string &err,
                     bool backward);
// Forward pass on the batch with parameters theta (device, 55,045 floats).
void gcin_forward(GcinBatch &b, const float *theta, cudaStream_t s);
// Backward from b.dc (device, G x 5) into grad (device, 55,045 floats, overwritten).
void gcin_backward(GcinBatch &b, const float *theta, float *grad, cudaStream_t s);

// Per-graph head scratch floats (activations kept for backward).
constexpr int kHeadScratch = kEmb /*z*/ + kEmb /*zhat*/ + kEmb /*sig*/ + 128 /*a1*/ + 64 /*a2*/ + 4 /*mean,rstd*/;
constexpr int kHeadGrad = 128 /*dz1*/ + 64 /*dz2*/ + kEmb /*dzh*/ + kEmb /*dz*/;

struct GcinEngine {
    float *theta = nullptr;
    bool have_params = false;
    GcinBatch batch;
    long long batch_version = -1;   // hierarchy version the batch was built from
    // inference + smoother assembly captured once per batch and arithmetic
    // (the parameters are read from `theta` at replay)
    cudaGraphExec_t exec = nullptr;
    long long exec_version = -1;
    int exec_key = -1;
    long long exec_kernels = 0;
};

// Per-device kernel attributes of the GCIN forward (set before any capture).
void gcin_prepare_device();

}  // namespace amg
