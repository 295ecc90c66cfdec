// GCIN coefficient network, forward pass (Sec. 3.2, App. A.1; Algorithm 1
// steps 1-6) on sm_103a.
//
// The batch is the disjoint union of every level graph (Algorithm 1 step 5):
// one concatenated CSR whose entries are the edges (weight a_ij; the
// diagonal entry is the self-loop of A_hat with weight a_ii) plus the node
// range of every graph.  Per layer:
//   aggregation  h_i = sum_j w_ij x_j         warp per node, lanes own 2 features
//   linear       y = h Theta + b              fused into the aggregation kernel
//   statistics   per graph mean/rstd of y     block per graph, FP64 sums
//   normalise    x = ReLU((y - mu) rstd gamma + beta)
//   pooling      per graph mean / max (+argmax) of x
// Head (block per graph): 4 readout linears 128->32, LayerNorm(128),
// sigmoid, Linear 128->128 + ReLU, Linear 128->64 + ReLU, Linear 64->5.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gcin.cuh"

namespace amg {

constexpr float kEps = 1e-5f;
__constant__ ParamLayout kPLd = make_layout();   // device copy of the parameter offsets

// ---------------------------------------------------------------------------
// batch construction
// ---------------------------------------------------------------------------
__global__ void k_cat_graph(int n, int nnz, const int *__restrict__ rp, const int *__restrict__ col,
                            const double *__restrict__ v, int node_off, int edge_off, int g,
                            int *__restrict__ rp_out, int *__restrict__ col_out, float *__restrict__ w_out,
                            double *__restrict__ w64_out, int *__restrict__ gid) {
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t < n) {
        rp_out[node_off + t] = rp[t] + edge_off;
        gid[node_off + t] = g;
    }
    if (t < nnz) {
        col_out[edge_off + t] = col[t] + node_off;
        w_out[edge_off + t] = static_cast<float>(v[t]);
        w64_out[edge_off + t] = v[t];
    }
}

__global__ void k_set_int(int *p, int v) { *p = v; }

void gcin_batch_free(GcinBatch &b) {
    if (b.arena) cudaFree(b.arena);
    b = GcinBatch{};
}

static void batch_layout(GcinBatch &b, Planner &pl) {
    const size_t N = b.N, G = b.G, E = std::max<long long>(1, b.E);
    b.rp = pl.take<int>(N + 1);
    b.col = pl.take<int>(E);
    b.w = pl.take<float>(E);
    b.w64 = pl.take<double>(E);
    b.gptr = pl.take<int>(G + 1);
    b.gid = pl.take<int>(N);
    b.x0 = pl.take<double>(N * 2);
    b.h1 = pl.take<float>(N * 2);
    for (int l = 0; l < kLayers; ++l) {
        b.h[l] = (l == 0) ? nullptr : pl.take<float>(N * kHidden);
        b.y[l] = pl.take<float>(N * kHidden);
        b.x[l] = pl.take<float>(N * kHidden);
        b.mu[l] = pl.take<float>(G * kHidden);
        b.rstd[l] = pl.take<float>(G * kHidden);
    }
    b.pooled = pl.take<float>(G * kLayers * 2 * kHidden);
    b.argmax = pl.take<int>(G * kLayers * kHidden);
    b.head = pl.take<float>(G * kHeadScratch);
    b.c = pl.take<float>(G * 5);
}

int gcin_batch_build(GcinBatch &b, int n_problems, amg_ctx *const *problems, cudaStream_t s, std::string &err) {
    gcin_batch_free(b);
    std::vector<int> gptr(1, 0);
    long long E = 0;
    for (int m = 0; m < n_problems; ++m) {
        const amg_ctx *c = problems[m];
        if (!c || c->lev.empty()) {
            err = "problem " + std::to_string(m) + " has no hierarchy";
            return AMG_ERR_STATE;
        }
        for (const auto &L : c->lev) {
            gptr.push_back(gptr.back() + L.n);
            E += L.A.nnz;
        }
    }
    if (E > 2000000000LL || gptr.back() <= 0) {
        err = "batch graph too large or empty";
        return AMG_ERR_ARG;
    }
    b.G = static_cast<int>(gptr.size()) - 1;
    b.N = gptr.back();
    b.E = E;
    Planner pl;
    batch_layout(b, pl);
    cudaError_t e = cudaMalloc(&b.arena, pl.off);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc batch: ") + cudaGetErrorString(e);
        b.arena = nullptr;
        return AMG_ERR_CUDA;
    }
    b.bytes = pl.off;
    pl = Planner{};
    pl.base = b.arena;
    batch_layout(b, pl);
    cudaMemcpyAsync(b.gptr, gptr.data(), sizeof(int) * gptr.size(), cudaMemcpyHostToDevice, s);
    int g = 0;
    long long eoff = 0;
    for (int m = 0; m < n_problems; ++m) {
        for (const auto &L : problems[m]->lev) {
            const int work = std::max(L.n, L.A.nnz);
            k_cat_graph<<<grid_for(work), kBlock, 0, s>>>(L.n, L.A.nnz, L.A.rp, L.A.col, L.A.v64, gptr[g],
                                                          static_cast<int>(eoff), g, b.rp, b.col, b.w, b.w64,
                                                          b.gid); AMG_COUNT();
            eoff += L.A.nnz;
            ++g;
        }
    }
    k_set_int<<<1, 1, 0, s>>>(b.rp + b.N, static_cast<int>(E)); AMG_COUNT();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("batch build: ") + cudaGetErrorString(e);
        return AMG_ERR_CUDA;
    }
    return AMG_OK;
}

// ---------------------------------------------------------------------------
// forward kernels
// ---------------------------------------------------------------------------
// x0_i = [a_ii, deg_i] (Algorithm 1 step 3; deg = off-diagonal pattern entries)
__global__ void k_feat0(int N, const int *__restrict__ rp, const int *__restrict__ col,
                        const double *__restrict__ w64, double *__restrict__ x0) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= N) return;
    double d = 0.0;
    int deg = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        if (col[p] == i) d += w64[p];
        else ++deg;
    }
    x0[2 * i] = d;
    x0[2 * i + 1] = static_cast<double>(deg);
}

// Layer 1: h = A_hat x0 (2 features, FP64 sums of the raw features), y = h W + b.
__global__ void __launch_bounds__(kBlock) k_layer1(int N, const int *__restrict__ rp, const int *__restrict__ col,
                                                   const double *__restrict__ w64, const double *__restrict__ x0,
                                                   const float *__restrict__ W, const float *__restrict__ bias,
                                                   float *__restrict__ h1, float *__restrict__ y) {
    const int warp = (blockIdx.x * kBlock + threadIdx.x) / 32, lane = threadIdx.x % 32;
    const int i = warp;
    double a0 = 0.0, a1 = 0.0;
    if (i < N) {
        for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const double wv = w64[p];
            const int j = col[p];
            a0 += wv * x0[2 * j];
            a1 += wv * x0[2 * j + 1];
        }
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (i >= N) return;
    if (lane == 0) {
        h1[2 * i] = static_cast<float>(a0);
        h1[2 * i + 1] = static_cast<float>(a1);
    }
    const int k = 2 * lane;
    const double y0 = a0 * W[k] + a1 * W[kHidden + k] + bias[k];
    const double y1 = a0 * W[k + 1] + a1 * W[kHidden + k + 1] + bias[k + 1];
    reinterpret_cast<float2 *>(y)[static_cast<size_t>(i) * 32 + lane] =
        make_float2(static_cast<float>(y0), static_cast<float>(y1));
}

// Layers 2..4: h = A_hat x (64 features, lanes own feature pairs), y = h W + b.
__global__ void __launch_bounds__(kBlock) k_agg_lin(int N, const int *__restrict__ rp, const int *__restrict__ col,
                                                    const float *__restrict__ w, const float *__restrict__ x,
                                                    const float *__restrict__ W, const float *__restrict__ bias,
                                                    float *__restrict__ hout, float *__restrict__ y) {
    __shared__ float2 sW[kHidden * 32];   // W[m][2 lane .. 2 lane + 1]
    for (int t = threadIdx.x; t < kHidden * 32; t += kBlock)
        sW[t] = reinterpret_cast<const float2 *>(W)[t];
    __syncthreads();
    const int i = (blockIdx.x * kBlock + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (i >= N) return;
    const float2 *x2 = reinterpret_cast<const float2 *>(x);
    float hx = 0.f, hy = 0.f;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const float wv = w[p];
        const float2 v = x2[static_cast<size_t>(col[p]) * 32 + lane];
        hx = fmaf(wv, v.x, hx);
        hy = fmaf(wv, v.y, hy);
    }
    reinterpret_cast<float2 *>(hout)[static_cast<size_t>(i) * 32 + lane] = make_float2(hx, hy);
    float y0 = bias[2 * lane], y1 = bias[2 * lane + 1];
#pragma unroll 8
    for (int m = 0; m < kHidden; ++m) {
        const float hm = __shfl_sync(0xffffffffu, (m & 1) ? hy : hx, m >> 1);
        const float2 wm = sW[m * 32 + lane];
        y0 = fmaf(hm, wm.x, y0);
        y1 = fmaf(hm, wm.y, y1);
    }
    reinterpret_cast<float2 *>(y)[static_cast<size_t>(i) * 32 + lane] = make_float2(y0, y1);
}

// Per-graph instance-norm statistics (biased variance, two passes, FP64 sums).
__global__ void __launch_bounds__(kBlock) k_graph_stats(const int *__restrict__ gptr, const float *__restrict__ y,
                                                        float *__restrict__ mu, float *__restrict__ rstd) {
    __shared__ double red[kBlock];
    __shared__ double smean[kHidden];
    const int g = blockIdx.x;
    const int f = threadIdx.x % kHidden, q = threadIdx.x / kHidden;   // 4 node lanes
    const int a = gptr[g], e = gptr[g + 1];
    const int n = e - a;
    double s = 0.0;
    for (int i = a + q; i < e; i += kBlock / kHidden) s += y[static_cast<size_t>(i) * kHidden + f];
    red[threadIdx.x] = s;
    __syncthreads();
    if (q == 0) {
        double t = 0.0;
        for (int k = 0; k < kBlock / kHidden; ++k) t += red[k * kHidden + f];
        smean[f] = t / n;
    }
    __syncthreads();
    const double m = smean[f];
    double v = 0.0;
    for (int i = a + q; i < e; i += kBlock / kHidden) {
        const double d = y[static_cast<size_t>(i) * kHidden + f] - m;
        v += d * d;
    }
    __syncthreads();
    red[threadIdx.x] = v;
    __syncthreads();
    if (q == 0) {
        double t = 0.0;
        for (int k = 0; k < kBlock / kHidden; ++k) t += red[k * kHidden + f];
        mu[g * kHidden + f] = static_cast<float>(m);
        rstd[g * kHidden + f] = static_cast<float>(1.0 / sqrt(t / n + static_cast<double>(kEps)));
    }
}

// x = ReLU((y - mu) rstd gamma + beta)
__global__ void k_norm_relu(int N, const int *__restrict__ gid, const float *__restrict__ y,
                            const float *__restrict__ mu, const float *__restrict__ rstd,
                            const float *__restrict__ gamma, const float *__restrict__ beta, float *__restrict__ x) {
    const long long t = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (t >= static_cast<long long>(N) * kHidden) return;
    const int i = static_cast<int>(t / kHidden), f = static_cast<int>(t % kHidden);
    const int g = gid[i];
    const float z = (y[t] - mu[g * kHidden + f]) * rstd[g * kHidden + f] * gamma[f] + beta[f];
    x[t] = fmaxf(z, 0.f);
}

// Per-graph mean and max (first index of the max kept) of x.
__global__ void __launch_bounds__(kBlock) k_pool(const int *__restrict__ gptr, const float *__restrict__ x,
                                                 float *__restrict__ pooled, int *__restrict__ argmax, int layer) {
    __shared__ double rs[kBlock];
    __shared__ float rm[kBlock];
    __shared__ int ri[kBlock];
    const int g = blockIdx.x;
    const int f = threadIdx.x % kHidden, q = threadIdx.x / kHidden;
    const int a = gptr[g], e = gptr[g + 1];
    double s = 0.0;
    float mx = -INFINITY;
    int mi = a;
    for (int i = a + q; i < e; i += kBlock / kHidden) {
        const float v = x[static_cast<size_t>(i) * kHidden + f];
        s += v;
        if (v > mx) { mx = v; mi = i; }
    }
    rs[threadIdx.x] = s;
    rm[threadIdx.x] = mx;
    ri[threadIdx.x] = mi;
    __syncthreads();
    if (q == 0) {
        double t = 0.0;
        float bm = -INFINITY;
        int bi = a;
        for (int k = 0; k < kBlock / kHidden; ++k) {
            const int idx = k * kHidden + f;
            t += rs[idx];
            if (rm[idx] > bm || (rm[idx] == bm && ri[idx] < bi)) { bm = rm[idx]; bi = ri[idx]; }
        }
        float *P = pooled + (static_cast<size_t>(g) * kLayers + layer) * 2 * kHidden;
        P[f] = static_cast<float>(t / (e - a));
        P[kHidden + f] = bm;
        argmax[(static_cast<size_t>(g) * kLayers + layer) * kHidden + f] = bi;
    }
}

__device__ __forceinline__ float block128_sum(float v, float *red) {
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    float t = red[0] + red[1] + red[2] + red[3];
    __syncthreads();
    return t;
}

// Readout + head for one graph (128 threads).
__global__ void __launch_bounds__(128) k_head(const float *__restrict__ pooled, const float *__restrict__ th,
                                              float *__restrict__ scratch, float *__restrict__ c) {
    __shared__ float sp[kLayers * 2 * kHidden];
    __shared__ float ss[kEmb], sa1[128], sa2[64];
    __shared__ float red[4];
    const int g = blockIdx.x, t = threadIdx.x;
    for (int k = t; k < kLayers * 2 * kHidden; k += 128) sp[k] = pooled[static_cast<size_t>(g) * kLayers * 2 * kHidden + k];
    __syncthreads();
    float *S = scratch + static_cast<size_t>(g) * kHeadScratch;
    // readout linears: z[32 l + k] = [mean_l, max_l] . W_l[:, k] + b_l[k]
    const int l = t / kRo, k = t % kRo;
    const float *W = th + kPLd.roW[l];
    float z = th[kPLd.roB[l] + k];
    for (int m = 0; m < 2 * kHidden; ++m) z = fmaf(sp[l * 2 * kHidden + m], W[m * kRo + k], z);
    // layer norm over the 128-vector
    const float mean = block128_sum(z, red) / kEmb;
    const float d = z - mean;
    const float var = block128_sum(d * d, red) / kEmb;
    const float rs = rsqrtf(var + kEps);
    const float zh = d * rs * th[kPLd.lnG + t] + th[kPLd.lnB + t];
    const float sg = 1.f / (1.f + expf(-zh));
    S[t] = z;
    S[kEmb + t] = zh;
    S[2 * kEmb + t] = sg;
    if (t == 0) {
        S[3 * kEmb + 128 + 64] = mean;
        S[3 * kEmb + 128 + 64 + 1] = rs;
    }
    ss[t] = sg;
    __syncthreads();
    float a1 = th[kPLd.h1B + t];
    for (int m = 0; m < kEmb; ++m) a1 = fmaf(ss[m], th[kPLd.h1W + m * 128 + t], a1);
    a1 = fmaxf(a1, 0.f);
    sa1[t] = a1;
    S[3 * kEmb + t] = a1;
    __syncthreads();
    if (t < 64) {
        float a2 = th[kPLd.h2B + t];
        for (int m = 0; m < 128; ++m) a2 = fmaf(sa1[m], th[kPLd.h2W + m * 64 + t], a2);
        a2 = fmaxf(a2, 0.f);
        sa2[t] = a2;
        S[3 * kEmb + 128 + t] = a2;
    }
    __syncthreads();
    if (t < 5) {
        float o = th[kPLd.h3B + t];
        for (int m = 0; m < 64; ++m) o = fmaf(sa2[m], th[kPLd.h3W + m * 5 + t], o);
        c[g * 5 + t] = o;
    }
}

void gcin_forward(GcinBatch &b, const float *th, cudaStream_t s) {
    const int N = b.N, G = b.G;
    k_feat0<<<grid_for(N), kBlock, 0, s>>>(N, b.rp, b.col, b.w64, b.x0); AMG_COUNT();
    const int warp_grid = grid_for(static_cast<long long>(N) * 32);
    const int elem_grid = grid_for(static_cast<long long>(N) * kHidden);
    for (int l = 0; l < kLayers; ++l) {
        if (l == 0) {
            k_layer1<<<warp_grid, kBlock, 0, s>>>(N, b.rp, b.col, b.w64, b.x0, th + kPL.convW[0], th + kPL.convB[0],
                                                  b.h1, b.y[0]); AMG_COUNT();
        } else {
            k_agg_lin<<<warp_grid, kBlock, 0, s>>>(N, b.rp, b.col, b.w, b.x[l - 1], th + kPL.convW[l],
                                                   th + kPL.convB[l], b.h[l], b.y[l]); AMG_COUNT();
        }
        k_graph_stats<<<G, kBlock, 0, s>>>(b.gptr, b.y[l], b.mu[l], b.rstd[l]); AMG_COUNT();
        k_norm_relu<<<elem_grid, kBlock, 0, s>>>(N, b.gid, b.y[l], b.mu[l], b.rstd[l], th + kPL.inG[l],
                                                 th + kPL.inB[l], b.x[l]); AMG_COUNT();
        k_pool<<<G, kBlock, 0, s>>>(b.gptr, b.x[l], b.pooled, b.argmax, l); AMG_COUNT();
    }
    k_head<<<G, 128, 0, s>>>(b.pooled, th, b.head, b.c); AMG_COUNT();
}

void gcin_engine_free(GcinEngine *e) {
    if (!e) return;
    gcin_batch_free(e->batch);
    if (e->theta) cudaFree(e->theta);
    delete e;
}

}  // namespace amg

using namespace amg;

extern "C" {

int gnn_load_params(amg_ctx *c, const float *theta, long long n) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!theta || n != kNumParams) return ctx_fail(c, "expected 55045 parameters"), AMG_ERR_ARG;
    cudaError_t e = cudaSetDevice(c->opt.device);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "cudaSetDevice");
    if (!c->gnn) {
        c->gnn = new GcinEngine();
        e = cudaMalloc(&c->gnn->theta, sizeof(float) * kNumParams);
        if (e != cudaSuccess) {
            delete c->gnn;
            c->gnn = nullptr;
            return ctx_cuda_check(c, e, "cudaMalloc params");
        }
    }
    e = cudaMemcpyAsync(c->gnn->theta, theta, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "upload params");
    c->gnn->have_params = true;
    return AMG_OK;
}

int gnn_predict_coeffs(amg_ctx *c, double *c_out) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!c->gnn || !c->gnn->have_params) return ctx_fail(c, "no GCIN parameters loaded"), AMG_ERR_STATE;
    cudaError_t e = cudaSetDevice(c->opt.device);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "cudaSetDevice");
    GcinEngine *g = c->gnn;
    cudaStream_t s = c->stream;
    if (g->batch_version != c->hier_version || g->batch.G != static_cast<int>(c->lev.size())) {
        std::string err;
        amg_ctx *one[1] = {c};
        int rc = gcin_batch_build(g->batch, 1, one, s, err);
        if (rc) return ctx_fail(c, err), rc;
        g->batch_version = c->hier_version;
    }
    gcin_forward(g->batch, g->theta, s);
    const int G = g->batch.G;
    std::vector<float> cf(static_cast<size_t>(G) * 5);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cf.data(), g->batch.c, sizeof(float) * cf.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "GCIN forward");
    std::vector<double> cd(cf.begin(), cf.end());
    if (c_out) std::copy(cd.begin(), cd.end(), c_out);
    int rc = set_coeffs_device(c, cd.data(), G, s);
    if (rc) return rc;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "assemble smoother");
    return AMG_OK;
}

}  // extern "C"
