// GCIN coefficient network (Sec. 3.2, App. A.1): parameter layout and the
// batched graph container shared by inference and training.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "ctx.cuh"

namespace amg {

constexpr int kHidden = 64;      // GCIN width of the App. A.1 network (the widest one built)
constexpr int kHidden32 = 32;    // the halved width of App. B.3 (structured meshes)
constexpr int kLayers = 4;
constexpr int kRo = 32;          // readout width per layer
constexpr int kEmb = kRo * kLayers;   // 128
constexpr int kNumParams = 55045;     // hidden 64
constexpr int kNumParams32 = 37189;   // hidden 32

// Offsets of each tensor in the flat parameter vector (App. A.1 layout; a
// width H replaces every GCIN width 64, the readout input being 2H).
struct ParamLayout {
    int convW[kLayers], convB[kLayers];
    int inG[kLayers], inB[kLayers];
    int roW[kLayers], roB[kLayers];
    int lnG, lnB;
    int h1W, h1B, h2W, h2B, h3W, h3B;
    int total;
};

constexpr ParamLayout make_layout(int H) {
    ParamLayout p{};
    int o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int fin = (l == 0) ? 2 : H;
        p.convW[l] = o; o += fin * H;
        p.convB[l] = o; o += H;
    }
    for (int l = 0; l < kLayers; ++l) {
        p.inG[l] = o; o += H;
        p.inB[l] = o; o += H;
    }
    for (int l = 0; l < kLayers; ++l) {
        p.roW[l] = o; o += 2 * H * kRo;
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
constexpr ParamLayout kPL = make_layout(kHidden);
constexpr ParamLayout kPL32 = make_layout(kHidden32);
static_assert(kPL.total == kNumParams, "GCIN layout must have 55,045 parameters (App. A.1)");
static_assert(kPL32.total == kNumParams32, "hidden-32 GCIN layout has 37,189 parameters");
inline const ParamLayout &host_layout(int H) { return H == kHidden32 ? kPL32 : kPL; }
// GCIN width of a parameter vector of n entries (0 if none matches)
inline int hidden_of(long long n) { return n == kNumParams ? kHidden : n == kNumParams32 ? kHidden32 : 0; }

// Batch graph (Algorithm 1 steps 1-5): disjoint union of level graphs with
// node ranges gptr[g] .. gptr[g+1] and edges = the concatenated CSR patterns.
// Nodes are cut into tiles of at most kTile consecutive nodes that never
// cross a graph boundary; every reduction over a graph is a fixed-order
// combination of per-tile partials (deterministic, no atomics).
constexpr int kTile = 64;
constexpr int kChunkTiles = 64;     // smallest chunk of the tile -> chunk -> graph reductions
constexpr int kGradChunks = 64;      // tile chunks of the weight-gradient reduction

// Per-node and per-tile buffers are sized for the widest network (64) and
// indexed with the width of the parameters in use (`hidden`).
struct GcinBatch {
    int G = 0, N = 0, NT = 0;            // graphs, nodes, tiles
    int hidden = kHidden;                // GCIN width H of the parameters (64 or 32)
    int bf16 = 0;                        // layers 2..4 on tensor cores (BF16 operands, FP32 accumulation)
    int infer = 0;                       // inference only: no h, x in bfloat16 with bf16 (nothing kept for a backward)
    unsigned char *wtile = nullptr;      // layers 2..4: round(W)^T as BF16 tensor-core B tiles (bf16 inference)
    int *err = nullptr;                  // device error flag (tensor-core wait timeout)
    long long E = 0;
    int *rp = nullptr, *col = nullptr, *gptr = nullptr, *gid = nullptr;
    int *tstart = nullptr, *tgraph = nullptr, *gtile = nullptr;   // tile -> first node / graph; graph -> first tile
    // chunks of up to kChunkTiles tiles of one graph: the per-graph
    // reductions run tiles -> chunks -> graph, every stage in parallel
    int NC = 0;
    int *ctile = nullptr, *cnode = nullptr, *gchunk = nullptr;      // chunk -> first tile / node; graph -> first chunk
    float *cmean = nullptr, *cm2 = nullptr, *cmax = nullptr;        // NC x H chunk statistics
    double *csum = nullptr;                                         // NC x H
    int *carg = nullptr;                                            // NC x H
    float *w = nullptr;
    double *w64 = nullptr;
    // activations (kept for the backward pass)
    double *x0 = nullptr;                // N x 2 raw features [a_ii, deg] (FP64)
    float *h1 = nullptr;                 // N x 2      layer-1 aggregation
    float *h[kLayers] = {};              // N x H      layers 2..4 aggregation (h[0] unused)
    float *y[kLayers] = {};              // N x H      linear outputs
    float *x[kLayers] = {};              // N x H      ReLU(IN(y))
    float *mu[kLayers] = {}, *rstd[kLayers] = {};   // G x H
    float *tmean = nullptr, *tm2 = nullptr;          // NT x H tile statistics of y
    double *tsum = nullptr;                          // NT x H tile sums (pooling / backward)
    double *tsum2 = nullptr;                         // NT x H second tile sums (backward)
    float *tmax = nullptr;                           // NT x H
    int *targ = nullptr;                             // NT x H
    float *pooled = nullptr;             // G x 4 x 2H (mean | max per layer)
    int *argmax = nullptr;               // G x 4 x H   node index of each max
    float *head = nullptr;               // G x head scratch
    float *c = nullptr;                  // G x 5
    // backward work
    float *dc = nullptr;                 // G x 5
    float *dhead = nullptr;              // G x (dz1 128 | dz2 64 | dzh 128 | dz 128)
    float *dpooled = nullptr;            // G x 4 x 2H
    float *dx = nullptr, *dh = nullptr, *dy = nullptr;   // N x H
    double *gS1 = nullptr, *gS2 = nullptr;               // G x H per-graph sums
    float *dWt = nullptr;                // NT x (H x H + H) per-tile weight/bias gradient partials
    double *dWc = nullptr;               // kGradChunks x (H x H + H) chunk sums of dWt
    char *arena = nullptr;
    size_t bytes = 0;
};

void gcin_batch_free(GcinBatch &b);
// Build the batch from every level of every context; allocates device memory
// (with the backward buffers when `backward` is set).
int gcin_batch_build(GcinBatch &b, int n_problems, amg_ctx *const *problems, cudaStream_t s, std::string &err,
                     bool backward);
// Forward pass on the batch with parameters theta (device; 55,045 floats for
// b.hidden = 64, 37,189 for 32).
void gcin_forward(GcinBatch &b, const float *theta, cudaStream_t s);
// Backward from b.dc (device, G x 5) into grad (device, one float per
// parameter of width b.hidden, overwritten).
void gcin_backward(GcinBatch &b, const float *theta, float *grad, cudaStream_t s);

// Per-graph head scratch floats (activations kept for backward).
constexpr int kHeadScratch = kEmb /*z*/ + kEmb /*zhat*/ + kEmb /*sig*/ + 128 /*a1*/ + 64 /*a2*/ + 4 /*mean,rstd*/;
constexpr int kHeadGrad = 128 /*dz1*/ + 64 /*dz2*/ + kEmb /*dzh*/ + kEmb /*dz*/;

struct GcinEngine {
    float *theta = nullptr;              // room for the widest network
    bool have_params = false;
    int hidden = kHidden;                // width of the loaded parameters
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
