// GCIN coefficient network (Sec. 3.2, App. A.1; Algorithm 1 steps 1-6 and
// the network half of step 13) on sm_103a: forward, backward and Adam.
//
// The batch is the disjoint union of every level graph (Algorithm 1 step 5):
// one concatenated CSR whose entries are the edges (weight a_ij; the
// diagonal entry is the self-loop of A_hat with weight a_ii).  Nodes are cut
// into tiles of <= 64 consecutive nodes inside one graph; one block owns a
// tile.  Per layer (forward):
//   aggregation + linear   h_i = sum_j w_ij x_j, y = h Theta + b   (warp per
//                          node, lanes own feature pairs) and, in the same
//                          kernel, the tile's mean / M2 of y per feature
//   statistics             per graph: Chan combination of tile partials
//   normalise + pool       x = ReLU((y - mu) rstd gamma + beta) and the
//                          tile's sum / max / argmax of x
//   pooling                per graph: combination of tile partials
// Head (block per graph): 4 readout linears 128->32, LayerNorm(128),
// sigmoid, Linear 128->128 + ReLU, Linear 128->64 + ReLU, Linear 64->5.
// Backward mirrors these steps; every parameter gradient is a fixed-order
// sum of per-tile or per-graph partials, so gradients are bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <mutex>
#include <vector>

#include "gcin.cuh"

namespace amg {

constexpr float kEps = 1e-5f;
__constant__ ParamLayout kPLd[2] = {make_layout(kHidden), make_layout(kHidden32)};   // device copies of the offsets
template <int H>
__device__ __forceinline__ const ParamLayout &PL() { return kPLd[H == kHidden ? 0 : 1]; }
template <int H>
__host__ __device__ constexpr int num_params() { return make_layout(H).total; }

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

static void batch_layout(GcinBatch &b, Planner &pl, bool backward) {
    const size_t N = b.N, G = b.G, NT = b.NT, E = std::max<long long>(1, b.E);
    b.rp = pl.take<int>(N + 1);
    b.col = pl.take<int>(E);
    b.w = pl.take<float>(E);
    b.w64 = pl.take<double>(E);
    b.gptr = pl.take<int>(G + 1);
    b.gid = pl.take<int>(N);
    b.tstart = pl.take<int>(NT + 1);
    b.tgraph = pl.take<int>(NT);
    b.gtile = pl.take<int>(G + 1);
    const size_t NC = b.NC;
    b.ctile = pl.take<int>(NC + 1);
    b.cnode = pl.take<int>(NC + 1);
    b.gchunk = pl.take<int>(G + 1);
    b.cmean = pl.take<float>(NC * kHidden);
    b.cm2 = pl.take<float>(NC * kHidden);
    b.cmax = pl.take<float>(NC * kHidden);
    b.csum = pl.take<double>(NC * kHidden);
    b.carg = pl.take<int>(NC * kHidden);
    b.x0 = pl.take<double>(N * 2);
    b.h1 = pl.take<float>(N * 2);
    for (int l = 0; l < kLayers; ++l) {
        b.h[l] = (l == 0) ? nullptr : pl.take<float>(N * kHidden);
        b.y[l] = pl.take<float>(N * kHidden);
        b.x[l] = pl.take<float>(N * kHidden);
        b.mu[l] = pl.take<float>(G * kHidden);
        b.rstd[l] = pl.take<float>(G * kHidden);
    }
    b.tmean = pl.take<float>(NT * kHidden);
    b.tm2 = pl.take<float>(NT * kHidden);
    b.tsum = pl.take<double>(NT * kHidden);
    b.tsum2 = pl.take<double>(NT * kHidden);
    b.tmax = pl.take<float>(NT * kHidden);
    b.targ = pl.take<int>(NT * kHidden);
    b.pooled = pl.take<float>(G * kLayers * 2 * kHidden);
    b.argmax = pl.take<int>(G * kLayers * kHidden);
    b.head = pl.take<float>(G * kHeadScratch);
    b.c = pl.take<float>(G * 5);
    b.err = pl.take<int>(4);
    b.wtile = pl.take<unsigned char>(static_cast<size_t>(kLayers - 1) * kHidden * kHidden * 2);
    if (backward) {
        b.dc = pl.take<float>(G * 5);
        b.dhead = pl.take<float>(G * kHeadGrad);
        b.dpooled = pl.take<float>(G * kLayers * 2 * kHidden);
        b.dx = pl.take<float>(N * kHidden);
        b.dh = pl.take<float>(N * kHidden);
        b.dy = pl.take<float>(N * kHidden);
        b.gS1 = pl.take<double>(G * kHidden);
        b.gS2 = pl.take<double>(G * kHidden);
        b.dWt = pl.take<float>(NT * (kHidden * kHidden + kHidden));
        b.dWc = pl.take<double>(static_cast<size_t>(kGradChunks) * (kHidden * kHidden + kHidden));
    }
}

int gcin_batch_build(GcinBatch &b, int n_problems, amg_ctx *const *problems, cudaStream_t s, std::string &err,
                     bool backward) {
    gcin_batch_free(b);
    std::vector<int> gptr(1, 0), tstart, tgraph, gtile;
    long long E = 0;
    for (int m = 0; m < n_problems; ++m) {
        const amg_ctx *c = problems[m];
        if (!c || c->lev.empty()) {
            err = "problem " + std::to_string(m) + " has no hierarchy";
            return AMG_ERR_STATE;
        }
        for (const auto &L : c->lev) {
            const int g = static_cast<int>(gptr.size()) - 1;
            gtile.push_back(static_cast<int>(tstart.size()));
            for (int a = gptr.back(); a < gptr.back() + L.n; a += kTile) {
                tstart.push_back(a);
                tgraph.push_back(g);
            }
            gptr.push_back(gptr.back() + L.n);
            E += L.A.nnz;
        }
    }
    if (E > 2000000000LL || gptr.back() <= 0 || gptr.back() > 200000000) {
        err = "batch graph too large or empty";
        return AMG_ERR_ARG;
    }
    b.G = static_cast<int>(gptr.size()) - 1;
    b.N = gptr.back();
    b.NT = static_cast<int>(tstart.size());
    b.E = E;
    tstart.push_back(b.N);
    gtile.push_back(b.NT);
    std::vector<int> ctile, cnode, gchunk;
    for (int g = 0; g < b.G; ++g) {
        gchunk.push_back(static_cast<int>(ctile.size()));
        // about sqrt(tiles) tiles per chunk: both reduction stages then loop
        // over about as many parts per lane (at least kChunkTiles per chunk)
        const int nt_g = gtile[g + 1] - gtile[g];
        const int ct = std::max(kChunkTiles, static_cast<int>(std::ceil(std::sqrt(static_cast<double>(nt_g)))));
        for (int t = gtile[g]; t < gtile[g + 1]; t += ct) {
            ctile.push_back(t);
            cnode.push_back(tstart[t]);
        }
    }
    b.NC = static_cast<int>(ctile.size());
    ctile.push_back(b.NT);
    cnode.push_back(b.N);
    gchunk.push_back(b.NC);
    Planner pl;
    batch_layout(b, pl, backward);
    cudaError_t e = cudaMalloc(&b.arena, pl.off);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc batch: ") + cudaGetErrorString(e);
        b.arena = nullptr;
        return AMG_ERR_CUDA;
    }
    b.bytes = pl.off;
    pl = Planner{};
    pl.base = b.arena;
    batch_layout(b, pl, backward);
    cudaMemcpyAsync(b.gptr, gptr.data(), sizeof(int) * gptr.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.tstart, tstart.data(), sizeof(int) * tstart.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.tgraph, tgraph.data(), sizeof(int) * tgraph.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.gtile, gtile.data(), sizeof(int) * gtile.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.ctile, ctile.data(), sizeof(int) * ctile.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.cnode, cnode.data(), sizeof(int) * cnode.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.gchunk, gchunk.data(), sizeof(int) * gchunk.size(), cudaMemcpyHostToDevice, s);
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
    cudaMemsetAsync(b.err, 0, sizeof(int) * 4, s);
    e = cudaStreamSynchronize(s);   // host vectors above must outlive the async copies
    if (e == cudaSuccess) e = cudaGetLastError();
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

// mean and M2 (sum of squared deviations) per feature of the tile's y rows;
// the block's threads form kBlock / H groups of H (one thread per feature)
template <int H>
__device__ __forceinline__ void tile_stats(const float (*sY)[H + 1], int nn, float *tmean, float *tm2) {
    constexpr int Q = kBlock / H;
    __shared__ float red[Q][H];
    __shared__ float smean[H];
    const int f = threadIdx.x % H, q = threadIdx.x / H;
    float s = 0.f;
    for (int k = q; k < nn; k += Q) s += sY[k][f];
    red[q][f] = s;
    __syncthreads();
    if (q == 0) {
        float t = red[0][f];
#pragma unroll
        for (int j = 1; j < Q; ++j) t += red[j][f];
        smean[f] = t / nn;
    }
    __syncthreads();
    const float m = smean[f];
    float v = 0.f;
    for (int k = q; k < nn; k += Q) {
        const float d = sY[k][f] - m;
        v = fmaf(d, d, v);
    }
    __syncthreads();
    red[q][f] = v;
    __syncthreads();
    if (q == 0) {
        float t = red[0][f];
#pragma unroll
        for (int j = 1; j < Q; ++j) t += red[j][f];
        tmean[f] = m;
        tm2[f] = t;
    }
}

// Layer 1: h = A_hat x0 (FP64 sums of the raw features, four threads per
// node), y = h W + b (K = 2: FMA units); tile stats.
// bfloat16 copy of four FP32 values (round to nearest even), as 8 bytes
__device__ __forceinline__ uint2 bf16x4(float a, float b, float c, float d) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<unsigned *>(&lo), *reinterpret_cast<unsigned *>(&hi));
}

// YB (BF16 inference): y only feeds the tile statistics (FP32); h1 is stored
// and the normalisation pass recomputes y from it.
template <int H, bool YB = false>
__global__ void __launch_bounds__(kBlock) k_layer1_tile(const int *__restrict__ rp, const int *__restrict__ col,
                                                        const double *__restrict__ w64, const double *__restrict__ x0,
                                                        const float *__restrict__ W, const float *__restrict__ bias,
                                                        const int *__restrict__ tstart, float *__restrict__ h1,
                                                        float *__restrict__ y, float *__restrict__ tmean,
                                                        float *__restrict__ tm2) {
    __shared__ float sY[kTile][H + 1];
    __shared__ float sH[kTile][2];
    const int t = blockIdx.x, a = tstart[t], nn = tstart[t + 1] - a;
    {
        static_assert(kTile * 4 == kBlock, "four threads per node of a tile");
        // four threads per node (kTile * 4 = kBlock), entries p0 + q, p0 + q + 4,
        // ...; the four partial sums are added pairwise, the same in each lane
        const int k = threadIdx.x >> 2, q = threadIdx.x & 3;
        double a0 = 0.0, a1 = 0.0;
        if (k < nn) {
            const int i = a + k;
            for (int p = rp[i] + q; p < rp[i + 1]; p += 4) {
                const double wv = w64[p];
                const double2 xj = reinterpret_cast<const double2 *>(x0)[col[p]];
                a0 += wv * xj.x;
                a1 += wv * xj.y;
            }
        }
        a0 += __shfl_xor_sync(0xffffffffu, a0, 1);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
        a0 += __shfl_xor_sync(0xffffffffu, a0, 2);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
        if (k < nn && q == 0) {
            const float h0 = static_cast<float>(a0), hv1 = static_cast<float>(a1);
            reinterpret_cast<float2 *>(h1)[a + k] = make_float2(h0, hv1);
            sH[k][0] = h0;
            sH[k][1] = hv1;
        }
    }
    __syncthreads();
    // 64 nodes x H features: thread -> node k = tid / 4, features FT (tid % 4) .. + FT - 1
    constexpr int FT = H / 4;
    const int k = threadIdx.x / 4, f0 = FT * (threadIdx.x % 4);
    if (k < nn) {
        const float h0 = sH[k][0], hv1 = sH[k][1];
        float out[FT];
#pragma unroll
        for (int q = 0; q < FT; ++q) {
            const int f = f0 + q;
            out[q] = fmaf(h0, W[f], fmaf(hv1, W[H + f], bias[f]));
            sY[k][f] = out[q];
        }
        // BF16 inference stores no y: the normalisation pass forms it again
        // from h1 (8 bytes per node instead of 128)
        if (!YB) {
            float4 *yo = reinterpret_cast<float4 *>(y + static_cast<size_t>(a + k) * H + f0);
#pragma unroll
            for (int q = 0; q < FT / 4; ++q) yo[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
        }
    }
    __syncthreads();
    tile_stats<H>(sY, nn, tmean + static_cast<size_t>(t) * H, tm2 + static_cast<size_t>(t) * H);
}

// h_i = sum_p w_p x_{col p} with L = H / 4 lanes per row and 32 / L rows per
// warp (two rows for H = 64, four for H = 32): lane j of a row's group owns
// features 4 j .. 4 j + 3, and entries are added in row order.  Up to L
// (col, w) pairs per row come in with one coalesced load and are broadcast by
// shuffles; each lane keeps four 16-byte gathers in flight, so a warp has
// eight H = 64 (or sixteen H = 32) feature rows in flight.  Called by a whole
// warp (the loop runs to the longest row of the warp, shorter rows predicated
// off).
template <int H, class XR = const float4 *>
__device__ __forceinline__ float4 agg_rows(int p0, int p1, const int *__restrict__ col, const float *__restrict__ w,
                                           const XR &x4, int hl) {
    constexpr int L = H / 4;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
    const int deg = p1 - p0;
    int maxdeg = deg;
#pragma unroll
    for (int o = L; o < 32; o <<= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xffffffffu, maxdeg, o));
    for (int base = 0; base < maxdeg; base += L) {
        int cj = 0;
        float wj = 0.f;
        if (base + hl < deg) {
            cj = col[p0 + base + hl];
            wj = w[p0 + base + hl];
        }
        const int cnt = deg - base;                  // entries of this row in the chunk (may be <= 0)
        const int cmax = min(L, maxdeg - base);
        int k = 0;
        for (; k + 4 <= cmax; k += 4) {
            int c[4];
            float wk[4];
            float4 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                c[j] = __shfl_sync(0xffffffffu, cj, k + j, L);
                wk[j] = __shfl_sync(0xffffffffu, wj, k + j, L);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                v[j] = (k + j < cnt) ? x4[static_cast<size_t>(c[j]) * L + hl] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k + j < cnt) {
                    h.x = fmaf(wk[j], v[j].x, h.x);
                    h.y = fmaf(wk[j], v[j].y, h.y);
                    h.z = fmaf(wk[j], v[j].z, h.z);
                    h.w = fmaf(wk[j], v[j].w, h.w);
                }
            }
        }
        for (; k < cmax; ++k) {
            const int c = __shfl_sync(0xffffffffu, cj, k, L);
            const float wk = __shfl_sync(0xffffffffu, wj, k, L);
            if (k < cnt) {
                const float4 v = x4[static_cast<size_t>(c) * L + hl];
                h.x = fmaf(wk, v.x, h.x);
                h.y = fmaf(wk, v.y, h.y);
                h.z = fmaf(wk, v.z, h.z);
                h.w = fmaf(wk, v.w, h.w);
            }
        }
    }
    return h;
}

// Layers 2..4: h = A_hat x (H features), y = h W + b; tile stats.
template <int H>
__global__ void __launch_bounds__(kBlock) k_agg_lin_tile(const int *__restrict__ rp, const int *__restrict__ col,
                                                         const float *__restrict__ w, const float *__restrict__ x,
                                                         const float *__restrict__ W, const float *__restrict__ bias,
                                                         const int *__restrict__ tstart, float *__restrict__ hout,
                                                         float *__restrict__ y, float *__restrict__ tmean,
                                                         float *__restrict__ tm2) {
    constexpr int L = H / 4, R = 32 / L;   // lanes per row, rows per warp
    __shared__ float4 sW[H * L];   // W[m][4 j .. 4 j + 3]
    __shared__ float sY[kTile][H + 1];
    for (int t2 = threadIdx.x; t2 < H * L; t2 += kBlock) sW[t2] = reinterpret_cast<const float4 *>(W)[t2];
    __syncthreads();
    const int t = blockIdx.x, a = tstart[t], nn = tstart[t + 1] - a;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, grp = lane / L, hl = lane % L;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 b4 = reinterpret_cast<const float4 *>(bias)[hl];
    for (int k0 = R * warp; k0 < nn; k0 += R * (kBlock / 32)) {
        const int k = k0 + grp;
        const bool live = k < nn;                    // the last rows of the last group may be absent
        const int i = a + (live ? k : k0);
        const int p0 = rp[i], p1 = live ? rp[i + 1] : p0;
        const float4 hv = agg_rows<H>(p0, p1, col, w, x4, hl);
        if (live && hout) reinterpret_cast<float4 *>(hout)[static_cast<size_t>(i) * L + hl] = hv;
        float4 yv = b4;
#pragma unroll 4
        for (int m = 0; m < H; ++m) {
            const float hsrc = (m & 3) == 0 ? hv.x : (m & 3) == 1 ? hv.y : (m & 3) == 2 ? hv.z : hv.w;
            const float hm = __shfl_sync(0xffffffffu, hsrc, m >> 2, L);
            const float4 wm = sW[m * L + hl];
            yv.x = fmaf(hm, wm.x, yv.x);
            yv.y = fmaf(hm, wm.y, yv.y);
            yv.z = fmaf(hm, wm.z, yv.z);
            yv.w = fmaf(hm, wm.w, yv.w);
        }
        if (live) {
            reinterpret_cast<float4 *>(y)[static_cast<size_t>(i) * L + hl] = yv;
            sY[k][4 * hl] = yv.x;
            sY[k][4 * hl + 1] = yv.y;
            sY[k][4 * hl + 2] = yv.z;
            sY[k][4 * hl + 3] = yv.w;
        }
    }
    __syncthreads();
    tile_stats<H>(sY, nn, tmean + static_cast<size_t>(t) * H, tm2 + static_cast<size_t>(t) * H);
}

// Fixed-order sum over the 16 tile lanes of one feature (16 H-thread blocks:
// f = tid % H, lane = tid / H); every thread receives the total.
constexpr int kLanes = 16;
template <int H>
constexpr int combine_threads() { return kLanes * H; }
template <int H>
__device__ __forceinline__ double lanes_sum(double v, double (*red)[H]) {
    const int f = threadIdx.x % H, q = threadIdx.x / H;
    red[q][f] = v;
    __syncthreads();
    for (int w = kLanes / 2; w > 0; w >>= 1) {
        if (q < w) red[q][f] += red[q + w][f];
        __syncthreads();
    }
    const double t = red[0][f];
    __syncthreads();
    return t;
}

// Group statistics from part statistics (biased variance):
// mean = sum_t n_t mean_t / n, M2 = sum_t [M2_t + n_t (mean_t - mean)^2].
// Parts t of group g are gtile[g] .. gtile[g+1] with node ranges
// tstart[t] .. tstart[t+1].  Run twice: tiles -> chunks (final = 0: writes
// the chunk mean and M2 into mu / rstd) and chunks -> graphs (final = 1:
// writes the instance-norm mean and 1/sqrt(var + eps)).  16 lanes of parts
// per feature; one FP64 add per part, the rest in FP32.
template <int H>
__global__ void __launch_bounds__(kLanes * H) k_stats_combine(const int *__restrict__ gtile, const int *__restrict__ gptr,
                                                            const int *__restrict__ tstart,
                                                            const float *__restrict__ tmean,
                                                            const float *__restrict__ tm2, float *__restrict__ mu,
                                                            float *__restrict__ rstd, int final) {
    __shared__ double red[kLanes][H];
    const int g = blockIdx.x, f = threadIdx.x % H, q = threadIdx.x / H;
    const double n = gptr[g + 1] - gptr[g];
    double s = 0.0;
    for (int t = gtile[g] + q; t < gtile[g + 1]; t += kLanes)
        s += static_cast<double>(static_cast<float>(tstart[t + 1] - tstart[t]) * tmean[static_cast<size_t>(t) * H + f]);
    const double mean = lanes_sum<H>(s, red) / n;
    const float mf = static_cast<float>(mean);
    double v = 0.0;
    for (int t = gtile[g] + q; t < gtile[g + 1]; t += kLanes) {
        const float d = tmean[static_cast<size_t>(t) * H + f] - mf;
        v += static_cast<double>(fmaf(static_cast<float>(tstart[t + 1] - tstart[t]) * d, d,
                                      tm2[static_cast<size_t>(t) * H + f]));
    }
    const double m2 = lanes_sum<H>(v, red);
    if (q == 0) {
        mu[static_cast<size_t>(g) * H + f] = mf;
        rstd[static_cast<size_t>(g) * H + f] =
            final ? static_cast<float>(1.0 / sqrt(m2 / n + static_cast<double>(kEps))) : static_cast<float>(m2);
    }
}

// x = ReLU((y - mu) rstd gamma + beta); tile sum / max / argmax of x
// (groups of H / 4 threads, four features per thread, kBlock / (H / 4) rows
// at a time).  x is stored in
// FP32 (x), in bfloat16 (xb: BF16 inference) or not at all (both null: the
// last layer in inference); the pooling always reads the FP32 value.
// YM: 0 FP32 y; 1 bfloat16 y (BF16 inference); 2 layer 1 in BF16 inference:
// y = h1 W1 + b1 recomputed from the stored h1 with the same FMAs as
// k_layer1_tile, rounded to bfloat16 as a stored y would be.
template <int H, int YM = 0>
__global__ void __launch_bounds__(kBlock, 6) k_norm_relu_pool_tile(const int *__restrict__ tstart,
                                                                const int *__restrict__ tgraph,
                                                                const float *__restrict__ y,
                                                                const float *__restrict__ mu,
                                                                const float *__restrict__ rstd,
                                                                const float *__restrict__ gamma,
                                                                const float *__restrict__ beta, float *__restrict__ x,
                                                                __nv_bfloat16 *__restrict__ xb,
                                                                double *__restrict__ tsum, float *__restrict__ tmax,
                                                                int *__restrict__ targ,
                                                                const float *__restrict__ h1 = nullptr,
                                                                const float *__restrict__ W1 = nullptr,
                                                                const float *__restrict__ b1 = nullptr) {
    constexpr int F = H / 4, Q = kBlock / F;   // threads per row (4 features each), rows at a time
    __shared__ double rs[Q][H];
    __shared__ float rm[Q][H];
    __shared__ int ri[Q][H];
    const int t = blockIdx.x, a = tstart[t], e = tstart[t + 1], g = tgraph[t];
    const int f = 4 * (threadIdx.x % F), q = threadIdx.x / F;
    const float4 m = *reinterpret_cast<const float4 *>(mu + g * H + f);
    const float4 r = *reinterpret_cast<const float4 *>(rstd + g * H + f);
    const float4 ga = *reinterpret_cast<const float4 *>(gamma + f);
    const float4 be = *reinterpret_cast<const float4 *>(beta + f);
    // FP32 partial sums of at most kTile / Q values per thread (GB300's FP64
    // pipe is narrow); the tile and graph sums are taken in FP64
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    float mx[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int mi[4] = {a, a, a, a};
    static_assert(kTile % Q == 0, "rows per thread");
#pragma unroll
    // every row's load first (predicated), so a thread's kTile / Q loads are in flight together
    float4 yr[kTile / Q];
#pragma unroll
    for (int r4 = 0; r4 < kTile / Q; ++r4) {
        const int i = a + q + r4 * Q;
        const size_t o = static_cast<size_t>(i < e ? i : a) * H + f;
        if (YM == 1) {   // bfloat16 y (BF16 inference), widened exactly
            const uint2 u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(y) + o);
            yr[r4] = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                                 __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
        } else if (YM == 2) {
            const float2 hh = reinterpret_cast<const float2 *>(h1)[i < e ? i : a];
            float yv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                yv[j] = __bfloat162float(__float2bfloat16_rn(fmaf(hh.x, W1[f + j], fmaf(hh.y, W1[H + f + j], b1[f + j]))));
            yr[r4] = make_float4(yv[0], yv[1], yv[2], yv[3]);
        } else {
            yr[r4] = *reinterpret_cast<const float4 *>(y + o);
        }
    }
#pragma unroll
    for (int r4 = 0; r4 < kTile / Q; ++r4) {
        const int i = a + q + r4 * Q;
        if (i >= e) break;
        const size_t o = static_cast<size_t>(i) * H + f;
        const float4 yv = yr[r4];
        float v[4];
        v[0] = fmaxf((yv.x - m.x) * r.x * ga.x + be.x, 0.f);
        v[1] = fmaxf((yv.y - m.y) * r.y * ga.y + be.y, 0.f);
        v[2] = fmaxf((yv.z - m.z) * r.z * ga.z + be.z, 0.f);
        v[3] = fmaxf((yv.w - m.w) * r.w * ga.w + be.w, 0.f);
        if (xb) {   // inference: the next aggregation's BF16 input
            *reinterpret_cast<uint2 *>(xb + o) = bf16x4(v[0], v[1], v[2], v[3]);
        } else if (x) {
            *reinterpret_cast<float4 *>(x + o) = make_float4(v[0], v[1], v[2], v[3]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s[j] += v[j];
            if (v[j] > mx[j]) { mx[j] = v[j]; mi[j] = i; }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rs[q][f + j] = static_cast<double>(s[j]);
        rm[q][f + j] = mx[j];
        ri[q][f + j] = mi[j];
    }
    __syncthreads();
    if (threadIdx.x < H) {
        const int ff = threadIdx.x;
        double ts = 0.0;
        float bm = -INFINITY;
        int bi = a;
        for (int k = 0; k < Q; ++k) {
            ts += rs[k][ff];
            if (rm[k][ff] > bm || (rm[k][ff] == bm && ri[k][ff] < bi)) { bm = rm[k][ff]; bi = ri[k][ff]; }
        }
        tsum[static_cast<size_t>(t) * H + ff] = ts;
        tmax[static_cast<size_t>(t) * H + ff] = bm;
        targ[static_cast<size_t>(t) * H + ff] = bi;
    }
}

// Group sum and max (first index of the max kept) from part partials; as
// for the statistics, tiles -> chunks (csum != nullptr: writes the chunk sum,
// max and argmax) and chunks -> graphs (writes the pooled mean and max).
template <int H>
__global__ void __launch_bounds__(kLanes * H) k_pool_combine(const int *__restrict__ gtile, const int *__restrict__ gptr,
                                                           const double *__restrict__ tsum,
                                                           const float *__restrict__ tmax,
                                                           const int *__restrict__ targ, float *__restrict__ pooled,
                                                           int *__restrict__ argmax, int layer,
                                                           double *__restrict__ csum, float *__restrict__ cmax,
                                                           int *__restrict__ carg) {
    __shared__ double red[kLanes][H];
    __shared__ float rm[kLanes][H];
    __shared__ int ri[kLanes][H];
    const int g = blockIdx.x, f = threadIdx.x % H, q = threadIdx.x / H;
    double s = 0.0;
    float bm = -INFINITY;
    int bi = gptr[g];
    for (int t = gtile[g] + q; t < gtile[g + 1]; t += kLanes) {
        const size_t o = static_cast<size_t>(t) * H + f;
        s += tsum[o];
        if (tmax[o] > bm) { bm = tmax[o]; bi = targ[o]; }   // tiles ascend, so the first max wins
    }
    rm[q][f] = bm;
    ri[q][f] = bi;
    const double total = lanes_sum<H>(s, red);
    if (q == 0) {
        for (int k = 1; k < kLanes; ++k)
            if (rm[k][f] > bm || (rm[k][f] == bm && ri[k][f] < bi)) { bm = rm[k][f]; bi = ri[k][f]; }
        if (csum) {
            const size_t o = static_cast<size_t>(g) * H + f;
            csum[o] = total;
            cmax[o] = bm;
            carg[o] = bi;
            return;
        }
        float *P = pooled + (static_cast<size_t>(g) * kLayers + layer) * 2 * H;
        P[f] = static_cast<float>(total / (gptr[g + 1] - gptr[g]));
        P[H + f] = bm;
        argmax[(static_cast<size_t>(g) * kLayers + layer) * H + f] = bi;
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

// Head scratch layout per graph: z[128] | zh[128] | sig[128] | a1[128] | a2[64] | mean | rstd
constexpr int kSz = 0, kSzh = kEmb, kSsg = 2 * kEmb, kSa1 = 3 * kEmb, kSa2 = 3 * kEmb + 128,
              kSmean = 3 * kEmb + 192, kSrs = 3 * kEmb + 193;
// Head gradient layout per graph: dz1[128] | dz2[64] | dzh[128] | dz[128]
constexpr int kGdz1 = 0, kGdz2 = 128, kGdzh = 192, kGdz = 192 + kEmb;

// Readout + head for one graph (128 threads).
template <int H>
__global__ void __launch_bounds__(128) k_head(const float *__restrict__ pooled, const float *__restrict__ th,
                                              float *__restrict__ scratch, float *__restrict__ c) {
    __shared__ float sp[kLayers * 2 * H];
    __shared__ float ss[kEmb], sa1[128], sa2[64];
    __shared__ float red[4];
    const int g = blockIdx.x, t = threadIdx.x;
    for (int k = t; k < kLayers * 2 * H; k += 128) sp[k] = pooled[static_cast<size_t>(g) * kLayers * 2 * H + k];
    __syncthreads();
    float *S = scratch + static_cast<size_t>(g) * kHeadScratch;
    // readout linears: z[32 l + k] = [mean_l, max_l] . W_l[:, k] + b_l[k]
    const int l = t / kRo, k = t % kRo;
    const float *W = th + PL<H>().roW[l];
    float z = th[PL<H>().roB[l] + k];
#pragma unroll 8
    for (int m = 0; m < 2 * H; ++m) z = fmaf(sp[l * 2 * H + m], W[m * kRo + k], z);
    // layer norm over the 128-vector
    const float mean = block128_sum(z, red) / kEmb;
    const float d = z - mean;
    const float var = block128_sum(d * d, red) / kEmb;
    const float rs = rsqrtf(var + kEps);
    const float zh = d * rs * th[PL<H>().lnG + t] + th[PL<H>().lnB + t];
    const float sg = 1.f / (1.f + expf(-zh));
    S[kSz + t] = z;
    S[kSzh + t] = zh;
    S[kSsg + t] = sg;
    if (t == 0) {
        S[kSmean] = mean;
        S[kSrs] = rs;
    }
    ss[t] = sg;
    __syncthreads();
    float a1 = th[PL<H>().h1B + t];
#pragma unroll 8
    for (int m = 0; m < kEmb; ++m) a1 = fmaf(ss[m], th[PL<H>().h1W + m * 128 + t], a1);
    a1 = fmaxf(a1, 0.f);
    sa1[t] = a1;
    S[kSa1 + t] = a1;
    __syncthreads();
    if (t < 64) {
        float a2 = th[PL<H>().h2B + t];
#pragma unroll 8
        for (int m = 0; m < 128; ++m) a2 = fmaf(sa1[m], th[PL<H>().h2W + m * 64 + t], a2);
        a2 = fmaxf(a2, 0.f);
        sa2[t] = a2;
        S[kSa2 + t] = a2;
    }
    __syncthreads();
    if (t < 5) {
        float o = th[PL<H>().h3B + t];
#pragma unroll 8
        for (int m = 0; m < 64; ++m) o = fmaf(sa2[m], th[PL<H>().h3W + m * 5 + t], o);
        c[g * 5 + t] = o;
    }
}

}  // namespace amg
#include "gcin_tc.cuh"
namespace amg {

void gcin_prepare_device() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaFuncSetAttribute(k_agg_lin_tc<kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<kHidden>());
    cudaFuncSetAttribute(k_agg_lin_tc<kHidden32>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<kHidden32>());
    cudaFuncSetAttribute(k_agg_lin_tc<kHidden, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<kHidden>());
    cudaFuncSetAttribute(k_agg_lin_tc<kHidden32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc_smem<kHidden32>());
    cudaFuncSetAttribute(k_bwd_lin_tc<kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcb_smem<kHidden>());
    cudaFuncSetAttribute(k_bwd_lin_tc<kHidden32>, cudaFuncAttributeMaxDynamicSharedMemorySize, tcb_smem<kHidden32>());
    done[dev] = true;
}

template <int H>
static void forward_impl(GcinBatch &b, const float *th, cudaStream_t s) {
    const ParamLayout &pl = host_layout(H);
    const int N = b.N, G = b.G, NT = b.NT;
    constexpr int CT = combine_threads<H>();
    const bool xb16 = b.bf16 && b.infer;   // BF16 inference on the tensor cores
    const bool xbf = xb16 && kInferBF16Acts;   // ... with y and x stored in bfloat16
    if (xb16) {
        k_pack_wtile<H><<<kLayers - 1, kBlock, 0, s>>>(th + pl.convW[1], th + pl.convW[2], th + pl.convW[3],
                                                      b.wtile); AMG_COUNT();
    }
    k_feat0<<<grid_for(N), kBlock, 0, s>>>(N, b.rp, b.col, b.w64, b.x0); AMG_COUNT();
    for (int l = 0; l < kLayers; ++l) {
        if (l == 0 && xbf) {
            k_layer1_tile<H, true><<<NT, kBlock, 0, s>>>(b.rp, b.col, b.w64, b.x0, th + pl.convW[0],
                                                         th + pl.convB[0], b.tstart, b.h1, b.y[0], b.tmean,
                                                         b.tm2); AMG_COUNT();
        } else if (l == 0) {
            k_layer1_tile<H><<<NT, kBlock, 0, s>>>(b.rp, b.col, b.w64, b.x0, th + pl.convW[0], th + pl.convB[0],
                                                   b.tstart, b.h1, b.y[0], b.tmean, b.tm2); AMG_COUNT();
        } else if (xb16) {
            k_agg_lin_tc<H, true><<<(NT + 1) / 2, kBlock, tc_smem<H>(), s>>>(
                b.rp, b.col, b.w, b.x[l - 1], nullptr, b.wtile + static_cast<size_t>(l - 1) * tc_b_bytes<H>(),
                th + pl.convB[l], b.tstart, NT, nullptr, b.y[l], b.tmean, b.tm2, b.err, 0); AMG_COUNT();
        } else if (b.bf16) {
            k_agg_lin_tc<H><<<(NT + 1) / 2, kBlock, tc_smem<H>(), s>>>(b.rp, b.col, b.w, b.x[l - 1],
                                                                     th + pl.convW[l], nullptr, th + pl.convB[l],
                                                                     b.tstart, NT, b.infer ? nullptr : b.h[l], b.y[l],
                                                                     b.tmean, b.tm2, b.err, 0); AMG_COUNT();
        } else {
            k_agg_lin_tile<H><<<NT, kBlock, 0, s>>>(b.rp, b.col, b.w, b.x[l - 1], th + pl.convW[l],
                                                    th + pl.convB[l], b.tstart, b.infer ? nullptr : b.h[l], b.y[l],
                                                    b.tmean, b.tm2); AMG_COUNT();
        }
        k_stats_combine<H><<<b.NC, CT, 0, s>>>(b.ctile, b.cnode, b.tstart, b.tmean, b.tm2, b.cmean, b.cm2, 0); AMG_COUNT();
        k_stats_combine<H><<<G, CT, 0, s>>>(b.gchunk, b.gptr, b.cnode, b.cmean, b.cm2, b.mu[l], b.rstd[l], 1); AMG_COUNT();
        // inference keeps only what the next aggregation reads (bfloat16 with
        // the tensor-core linears, nothing after the last layer)
        const bool last = l == kLayers - 1;
        float *xo = (b.infer && (xbf || last)) ? nullptr : b.x[l];
        __nv_bfloat16 *xbo = (xbf && !last) ? reinterpret_cast<__nv_bfloat16 *>(b.x[l]) : nullptr;
        if (xbf && l == 0) {
            k_norm_relu_pool_tile<H, 2><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.y[l], b.mu[l], b.rstd[l],
                                                              th + pl.inG[l], th + pl.inB[l], xo, xbo, b.tsum,
                                                              b.tmax, b.targ, b.h1, th + pl.convW[0],
                                                              th + pl.convB[0]); AMG_COUNT();
        } else if (xbf) {
            k_norm_relu_pool_tile<H, 1><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.y[l], b.mu[l], b.rstd[l],
                                                              th + pl.inG[l], th + pl.inB[l], xo, xbo, b.tsum,
                                                              b.tmax, b.targ); AMG_COUNT();
        } else {
            k_norm_relu_pool_tile<H><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.y[l], b.mu[l], b.rstd[l],
                                                           th + pl.inG[l], th + pl.inB[l], xo, xbo, b.tsum, b.tmax,
                                                           b.targ); AMG_COUNT();
        }
        k_pool_combine<H><<<b.NC, CT, 0, s>>>(b.ctile, b.cnode, b.tsum, b.tmax, b.targ, nullptr, nullptr, l,
                                              b.csum, b.cmax, b.carg); AMG_COUNT();
        k_pool_combine<H><<<G, CT, 0, s>>>(b.gchunk, b.gptr, b.csum, b.cmax, b.carg, b.pooled, b.argmax, l,
                                           nullptr, nullptr, nullptr); AMG_COUNT();
    }
    k_head<H><<<G, 128, 0, s>>>(b.pooled, th, b.head, b.c); AMG_COUNT();
}

void gcin_forward(GcinBatch &b, const float *th, cudaStream_t s) {
    gcin_prepare_device();
    // the tensor-core kernel's wait-timeout flag belongs to this forward pass
    // only: clear it first (a captured inference graph replays this too), so
    // one timed-out pass does not fail every later one
    cudaMemsetAsync(b.err, 0, sizeof(int) * 4, s);
    if (b.hidden == kHidden32) forward_impl<kHidden32>(b, th, s);
    else forward_impl<kHidden>(b, th, s);
}

// ---------------------------------------------------------------------------
// backward kernels
// ---------------------------------------------------------------------------
// Head backward for one graph: dc -> dz2, dz1, dzh, dz (readout outputs) and
// the pooled-feature gradient dpooled.
template <int H>
__global__ void __launch_bounds__(128) k_head_bwd(const float *__restrict__ scratch, const float *__restrict__ th,
                                                  const float *__restrict__ dc, float *__restrict__ dhead,
                                                  float *__restrict__ dpooled) {
    __shared__ float sdc[5], sdz2[64], sdz1[128], sdz[kEmb];
    __shared__ float red[4];
    const int g = blockIdx.x, t = threadIdx.x;
    const float *S = scratch + static_cast<size_t>(g) * kHeadScratch;
    float *D = dhead + static_cast<size_t>(g) * kHeadGrad;
    if (t < 5) sdc[t] = dc[g * 5 + t];
    __syncthreads();
    if (t < 64) {
        float da2 = 0.f;
        for (int k = 0; k < 5; ++k) da2 = fmaf(sdc[k], th[PL<H>().h3W + t * 5 + k], da2);
        const float dz2 = S[kSa2 + t] > 0.f ? da2 : 0.f;
        sdz2[t] = dz2;
        D[kGdz2 + t] = dz2;
    }
    __syncthreads();
    float da1 = 0.f;
    for (int k = 0; k < 64; ++k) da1 = fmaf(sdz2[k], th[PL<H>().h2W + t * 64 + k], da1);
    const float dz1 = S[kSa1 + t] > 0.f ? da1 : 0.f;
    sdz1[t] = dz1;
    D[kGdz1 + t] = dz1;
    __syncthreads();
    float ds = 0.f;
    for (int k = 0; k < 128; ++k) ds = fmaf(sdz1[k], th[PL<H>().h1W + t * 128 + k], ds);
    const float sg = S[kSsg + t];
    const float dzh = ds * sg * (1.f - sg);
    D[kGdzh + t] = dzh;
    // layer norm backward
    const float rs = S[kSrs], mean = S[kSmean];
    const float zn = (S[kSz + t] - mean) * rs;
    const float dzn = dzh * th[PL<H>().lnG + t];
    const float m1 = block128_sum(dzn, red) / kEmb;
    const float m2 = block128_sum(dzn * zn, red) / kEmb;
    const float dz = rs * (dzn - m1 - zn * m2);
    sdz[t] = dz;
    D[kGdz + t] = dz;
    __syncthreads();
    // readout linears: dpooled_l[m] = sum_k dz[32 l + k] W_l[m][k]
    for (int j = t; j < kLayers * 2 * H; j += 128) {
        const int l = j / (2 * H), m = j % (2 * H);
        const float *W = th + PL<H>().roW[l] + m * kRo;
        float acc = 0.f;
        for (int k = 0; k < kRo; ++k) acc = fmaf(sdz[l * kRo + k], W[k], acc);
        dpooled[static_cast<size_t>(g) * kLayers * 2 * H + j] = acc;
    }
}

// Gradients of the readout / layer-norm / head parameters: one thread per
// parameter, sum over graphs in graph order.
template <int H>
__global__ void k_head_param_grad(int G, const float *__restrict__ pooled, const float *__restrict__ scratch,
                                  const float *__restrict__ dhead, const float *__restrict__ dc,
                                  float *__restrict__ grad) {
    const int p = PL<H>().roW[0] + blockIdx.x * kBlock + threadIdx.x;
    if (p >= num_params<H>()) return;
    double acc = 0.0;
    int l = -1;
    for (int k = 0; k < kLayers; ++k)
        if (p >= PL<H>().roW[k] && p < PL<H>().roB[k] + kRo) l = k;
    for (int g = 0; g < G; ++g) {
        const float *S = scratch + static_cast<size_t>(g) * kHeadScratch;
        const float *D = dhead + static_cast<size_t>(g) * kHeadGrad;
        double v;
        if (l >= 0) {
            if (p < PL<H>().roB[l]) {
                const int o = p - PL<H>().roW[l], m = o / kRo, k = o % kRo;
                v = static_cast<double>(pooled[(static_cast<size_t>(g) * kLayers + l) * 2 * H + m]) *
                    D[kGdz + l * kRo + k];
            } else {
                v = D[kGdz + l * kRo + (p - PL<H>().roB[l])];
            }
        } else if (p < PL<H>().lnB) {
            const int k = p - PL<H>().lnG;
            v = static_cast<double>(D[kGdzh + k]) * ((S[kSz + k] - S[kSmean]) * S[kSrs]);
        } else if (p < PL<H>().h1W) {
            v = D[kGdzh + (p - PL<H>().lnB)];
        } else if (p < PL<H>().h1B) {
            const int o = p - PL<H>().h1W, m = o / 128, k = o % 128;
            v = static_cast<double>(S[kSsg + m]) * D[kGdz1 + k];
        } else if (p < PL<H>().h2W) {
            v = D[kGdz1 + (p - PL<H>().h1B)];
        } else if (p < PL<H>().h2B) {
            const int o = p - PL<H>().h2W, m = o / 64, k = o % 64;
            v = static_cast<double>(S[kSa1 + m]) * D[kGdz2 + k];
        } else if (p < PL<H>().h3W) {
            v = D[kGdz2 + (p - PL<H>().h2B)];
        } else if (p < PL<H>().h3B) {
            const int o = p - PL<H>().h3W, m = o / 5, k = o % 5;
            v = static_cast<double>(S[kSa2 + m]) * dc[g * 5 + k];
        } else {
            v = dc[g * 5 + (p - PL<H>().h3B)];
        }
        acc += v;
    }
    grad[p] = static_cast<float>(acc);
}

// Layer backward, part 1 (per tile): dX = dx_next + pooling routes; the
// ReLU mask gives d(yn); tile sums S1 = sum d(yn), S2 = sum d(yn) * yhat.
template <int H>
__global__ void __launch_bounds__(kBlock) k_bwd_relu_tile(const int *__restrict__ tstart,
                                                          const int *__restrict__ tgraph, const int *__restrict__ gptr,
                                                          const float *__restrict__ x, const float *__restrict__ y,
                                                          const float *__restrict__ mu, const float *__restrict__ rstd,
                                                          const float *__restrict__ dx, const float *__restrict__ dpooled,
                                                          const int *__restrict__ argmax, int layer,
                                                          float *__restrict__ dyn, double *__restrict__ tsum,
                                                          double *__restrict__ tsum2) {
    constexpr int Q = kBlock / H;
    __shared__ double r1[Q][H], r2[Q][H];
    const int t = blockIdx.x, a = tstart[t], e = tstart[t + 1], g = tgraph[t];
    const int f = threadIdx.x % H, q = threadIdx.x / H;
    const float *dp = dpooled + (static_cast<size_t>(g) * kLayers + layer) * 2 * H;
    const float dmean = dp[f] / (gptr[g + 1] - gptr[g]), dmax = dp[H + f];
    const int am = argmax[(static_cast<size_t>(g) * kLayers + layer) * H + f];
    const float m = mu[g * H + f], r = rstd[g * H + f];
    float s1 = 0.f, s2 = 0.f;                 // FP32 per thread, FP64 from the tile sum on
    for (int i = a + q; i < e; i += Q) {
        const size_t o = static_cast<size_t>(i) * H + f;
        float dX = dmean + (i == am ? dmax : 0.f);
        if (dx) dX += dx[o];
        const float d = x[o] > 0.f ? dX : 0.f;
        dyn[o] = d;
        s1 += d;
        s2 = fmaf(d, (y[o] - m) * r, s2);
    }
    r1[q][f] = static_cast<double>(s1);
    r2[q][f] = static_cast<double>(s2);
    __syncthreads();
    if (q == 0) {
        double t1 = r1[0][f], t2 = r2[0][f];
        for (int k = 1; k < Q; ++k) {
            t1 += r1[k][f];
            t2 += r2[k][f];
        }
        tsum[static_cast<size_t>(t) * H + f] = t1;
        tsum2[static_cast<size_t>(t) * H + f] = t2;
    }
}

template <int H>
__global__ void __launch_bounds__(kLanes * H) k_bwd_combine(const int *__restrict__ gtile,
                                                            const double *__restrict__ tsum,
                                                            const double *__restrict__ tsum2,
                                                            double *__restrict__ gS1, double *__restrict__ gS2) {
    __shared__ double red[kLanes][H];
    const int g = blockIdx.x, f = threadIdx.x % H, q = threadIdx.x / H;
    double s1 = 0.0, s2 = 0.0;
    for (int t = gtile[g] + q; t < gtile[g + 1]; t += kLanes) {
        s1 += tsum[static_cast<size_t>(t) * H + f];
        s2 += tsum2[static_cast<size_t>(t) * H + f];
    }
    const double t1 = lanes_sum<H>(s1, red);
    const double t2 = lanes_sum<H>(s2, red);
    if (q == 0) {
        gS1[g * H + f] = t1;
        gS2[g * H + f] = t2;
    }
}

// FPL = H / 32 consecutive floats of row i owned by lane `lane` (float2 for H = 64)
template <int FPL>
__device__ __forceinline__ void lane_load(const float *__restrict__ p, size_t i, int lane, float (&v)[FPL]) {
    if constexpr (FPL == 2) {
        const float2 t = reinterpret_cast<const float2 *>(p)[i * 32 + lane];
        v[0] = t.x;
        v[1] = t.y;
    } else {
        v[0] = p[i * 32 + lane];
    }
}

template <int FPL>
__device__ __forceinline__ void lane_store(float *__restrict__ p, size_t i, int lane, const float (&v)[FPL]) {
    if constexpr (FPL == 2) reinterpret_cast<float2 *>(p)[i * 32 + lane] = make_float2(v[0], v[1]);
    else p[i * 32 + lane] = v[0];
}

// Layer backward, part 2 (per tile): instance-norm backward
//   dy = rstd (gamma d(yn) - gamma S1/n - yhat gamma S2/n),
// then dh = dy W^T (layers 2..4) and the tile's partial weight and bias
// gradients sum_i h_i^T dy_i, sum_i dy_i.  A warp takes one node; lane j owns
// features FPL j .. FPL j + FPL - 1 (FPL = H / 32).
template <int FIN, int H>
__global__ void __launch_bounds__(kBlock) k_bwd_in_lin_tile(const int *__restrict__ tstart,
                                                            const int *__restrict__ tgraph,
                                                            const int *__restrict__ gptr, const float *__restrict__ y,
                                                            const float *__restrict__ mu,
                                                            const float *__restrict__ rstd,
                                                            const float *__restrict__ gamma,
                                                            const double *__restrict__ gS1,
                                                            const double *__restrict__ gS2,
                                                            const float *__restrict__ W, const float *__restrict__ hin,
                                                            const float *__restrict__ dyn, float *__restrict__ dh,
                                                            float *__restrict__ dWt, int round_w) {
    constexpr int FPL = H / 32;
    // sWT[k][FPL lane + j] = W[FPL lane + j][k]
    __shared__ __align__(8) float sWT[FIN == H ? H * H : 1];
    __shared__ float sH[kTile][FIN + 1];
    __shared__ float sD[kTile][H + 1];
    if (FIN == H) {
        for (int e = threadIdx.x; e < H * H; e += kBlock) {
            const int k = e / H, n = e % H;
            float wv = W[n * H + k];
            if (round_w) wv = __bfloat162float(__float2bfloat16_rn(wv));   // the forward multiplied by the BF16-rounded weights
            sWT[e] = wv;
        }
    }
    const int t = blockIdx.x, a = tstart[t], nn = tstart[t + 1] - a, g = tgraph[t];
    const float inv_n = 1.f / (gptr[g + 1] - gptr[g]);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    float ga[FPL], m[FPL], r[FPL], c1[FPL], c2[FPL];
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
        const int f = FPL * lane + j;
        ga[j] = gamma[f];
        m[j] = mu[g * H + f];
        r[j] = rstd[g * H + f];
        c1[j] = ga[j] * static_cast<float>(gS1[g * H + f]) * inv_n;
        c2[j] = ga[j] * static_cast<float>(gS2[g * H + f]) * inv_n;
    }
    __syncthreads();
    for (int k = warp; k < nn; k += kBlock / 32) {
        const int i = a + k;
        float d[FPL], yv[FPL], dy[FPL];
        lane_load<FPL>(dyn, i, lane, d);
        lane_load<FPL>(y, i, lane, yv);
#pragma unroll
        for (int j = 0; j < FPL; ++j) {
            const float yh = (yv[j] - m[j]) * r[j];
            dy[j] = r[j] * (ga[j] * d[j] - c1[j] - yh * c2[j]);
            sD[k][FPL * lane + j] = dy[j];
        }
        if (FIN == H) {
            float hv[FPL];
            lane_load<FPL>(hin, i, lane, hv);
#pragma unroll
            for (int j = 0; j < FPL; ++j) sH[k][FPL * lane + j] = hv[j];
            float acc[FPL] = {};
#pragma unroll 8
            for (int kk = 0; kk < H; ++kk) {
                const float dk = __shfl_sync(0xffffffffu, dy[kk % FPL], kk / FPL);
                if constexpr (FPL == 2) {
                    const float2 wk = reinterpret_cast<const float2 *>(sWT)[kk * 32 + lane];
                    acc[0] = fmaf(dk, wk.x, acc[0]);
                    acc[1] = fmaf(dk, wk.y, acc[1]);
                } else {
                    acc[0] = fmaf(dk, sWT[kk * H + lane], acc[0]);
                }
            }
            lane_store<FPL>(dh, i, lane, acc);
        } else {
            if (lane < FIN) sH[k][lane] = hin[static_cast<size_t>(i) * FIN + lane];
        }
    }
    __syncthreads();
    float *out = dWt + static_cast<size_t>(t) * (H * H + H);
    for (int e = threadIdx.x; e < FIN * H; e += kBlock) {
        const int mm = e / H, kk = e % H;
        float acc = 0.f;
        for (int j = 0; j < nn; ++j) acc = fmaf(sH[j][mm], sD[j][kk], acc);
        out[e] = acc;
    }
    if (threadIdx.x < H) {
        float acc = 0.f;
        for (int j = 0; j < nn; ++j) acc += sD[j][threadIdx.x];
        out[H * H + threadIdx.x] = acc;
    }
}

// dx = A_hat dh (A_hat symmetric), H features, 32 / (H / 4) nodes per warp.
template <int H>
__global__ void __launch_bounds__(kBlock) k_agg_plain(int N, const int *__restrict__ rp, const int *__restrict__ col,
                                                      const float *__restrict__ w, const float *__restrict__ v,
                                                      float *__restrict__ out) {
    constexpr int L = H / 4, R = 32 / L;
    const int wid = (blockIdx.x * kBlock + threadIdx.x) / 32, lane = threadIdx.x % 32, hl = lane % L;
    const int i0 = R * wid;
    if (i0 >= N) return;                         // warp-uniform
    const int i = i0 + lane / L;
    const bool live = i < N;
    const int p0 = rp[live ? i : i0], p1 = live ? rp[i + 1] : p0;
    const float4 h = agg_rows<H>(p0, p1, col, w, reinterpret_cast<const float4 *>(v), hl);
    if (live) reinterpret_cast<float4 *>(out)[static_cast<size_t>(i) * L + hl] = h;
}

// Conv weight/bias gradient: tile partials summed per chunk of tiles (FP64,
// tile order), then the chunks in order; instance-norm affine gradients are
// the per-graph sums added in graph order.
template <int H>
constexpr int grad_stride() { return H * H + H; }
template <int H>
__global__ void k_layer_param_partial(int NT, int fin, const float *__restrict__ dWt, double *__restrict__ chunk) {
    const int e = blockIdx.x * kBlock + threadIdx.x, c = blockIdx.y;
    const int nW = fin * H;
    if (e >= nW + H) return;
    const int src = (e < nW) ? e : H * H + (e - nW);
    const int t0 = static_cast<int>(static_cast<long long>(NT) * c / kGradChunks);
    const int t1 = static_cast<int>(static_cast<long long>(NT) * (c + 1) / kGradChunks);
    double acc = 0.0;
    for (int t = t0; t < t1; ++t) acc += dWt[static_cast<size_t>(t) * grad_stride<H>() + src];
    chunk[static_cast<size_t>(c) * grad_stride<H>() + e] = acc;
}

template <int H>
__global__ void k_layer_param_final(int G, int fin, const double *__restrict__ chunk, const double *__restrict__ gS1,
                                    const double *__restrict__ gS2, float *__restrict__ gW, float *__restrict__ gB,
                                    float *__restrict__ gG, float *__restrict__ gBeta) {
    const int e = blockIdx.x * kBlock + threadIdx.x;
    const int nW = fin * H;
    if (e < nW + H) {
        double acc = 0.0;
        for (int c = 0; c < kGradChunks; ++c) acc += chunk[static_cast<size_t>(c) * grad_stride<H>() + e];
        if (e < nW) gW[e] = static_cast<float>(acc);
        else gB[e - nW] = static_cast<float>(acc);
    } else if (e < nW + 2 * H) {
        const int f = e - nW - H;
        double s1 = 0.0, s2 = 0.0;
        for (int g = 0; g < G; ++g) {
            s1 += gS1[g * H + f];
            s2 += gS2[g * H + f];
        }
        gG[f] = static_cast<float>(s2);
        gBeta[f] = static_cast<float>(s1);
    }
}

template <int H>
static void backward_impl(GcinBatch &b, const float *th, float *grad, cudaStream_t s) {
    const ParamLayout &pl = host_layout(H);
    const int N = b.N, G = b.G, NT = b.NT;
    k_head_bwd<H><<<G, 128, 0, s>>>(b.head, th, b.dc, b.dhead, b.dpooled); AMG_COUNT();
    const int nhead = pl.total - pl.roW[0];
    k_head_param_grad<H><<<grid_for(nhead), kBlock, 0, s>>>(G, b.pooled, b.head, b.dhead, b.dc, grad); AMG_COUNT();
    constexpr int R = 32 / (H / 4);                                          // nodes per warp
    const int warp_grid = grid_for((static_cast<long long>(N) + R - 1) / R * 32);
    for (int l = kLayers - 1; l >= 0; --l) {
        k_bwd_relu_tile<H><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.gptr, b.x[l], b.y[l], b.mu[l], b.rstd[l],
                                                 l == kLayers - 1 ? nullptr : b.dx, b.dpooled, b.argmax, l, b.dy,
                                                 b.tsum, b.tsum2); AMG_COUNT();
        k_bwd_combine<H><<<G, combine_threads<H>(), 0, s>>>(b.gtile, b.tsum, b.tsum2, b.gS1, b.gS2); AMG_COUNT();
        if (l > 0 && b.bf16) {
            // the forward's node linear ran on the tensor cores: so does its backward
            k_bwd_lin_tc<H><<<(NT + 1) / 2, kBlock, tcb_smem<H>(), s>>>(b.tstart, b.tgraph, b.gptr, NT, b.y[l], b.mu[l],
                                                                      b.rstd[l], th + pl.inG[l], b.gS1, b.gS2,
                                                                      th + pl.convW[l], b.h[l], b.dy, b.dh, b.dWt,
                                                                      b.err); AMG_COUNT();
            k_agg_plain<H><<<warp_grid, kBlock, 0, s>>>(N, b.rp, b.col, b.w, b.dh, b.dx); AMG_COUNT();
        } else if (l > 0) {
            k_bwd_in_lin_tile<H, H><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.gptr, b.y[l], b.mu[l], b.rstd[l],
                                                          th + pl.inG[l], b.gS1, b.gS2, th + pl.convW[l], b.h[l],
                                                          b.dy, b.dh, b.dWt, b.bf16); AMG_COUNT();
            k_agg_plain<H><<<warp_grid, kBlock, 0, s>>>(N, b.rp, b.col, b.w, b.dh, b.dx); AMG_COUNT();
        } else {
            k_bwd_in_lin_tile<2, H><<<NT, kBlock, 0, s>>>(b.tstart, b.tgraph, b.gptr, b.y[l], b.mu[l], b.rstd[l],
                                                          th + pl.inG[l], b.gS1, b.gS2, th + pl.convW[l], b.h1,
                                                          b.dy, nullptr, b.dWt, 0); AMG_COUNT();
        }
        const int fin = (l == 0) ? 2 : H;
        k_layer_param_partial<H><<<dim3(grid_for(fin * H + H), kGradChunks), kBlock, 0, s>>>(NT, fin, b.dWt,
                                                                                          b.dWc); AMG_COUNT();
        k_layer_param_final<H><<<grid_for(fin * H + 2 * H), kBlock, 0, s>>>(
            G, fin, b.dWc, b.gS1, b.gS2, grad + pl.convW[l], grad + pl.convB[l], grad + pl.inG[l],
            grad + pl.inB[l]); AMG_COUNT();
    }
}

void gcin_backward(GcinBatch &b, const float *th, float *grad, cudaStream_t s) {
    if (b.hidden == kHidden32) backward_impl<kHidden32>(b, th, grad, s);
    else backward_impl<kHidden>(b, th, grad, s);
}

// ---------------------------------------------------------------------------
// optimiser: global-norm clipping + Adam (Table train_hyper)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_sq_partial_f(int n, const float *__restrict__ v, double *__restrict__ part) {
    __shared__ double red[kBlock / 32];
    double s = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) s += static_cast<double>(v[i]) * v[i];
    s = warp_sum(s);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) t += red[k];
        part[blockIdx.x] = t;
    }
}

__global__ void k_norm_from_partials(int np, const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    *out = sqrt(s);
}

// clip to max_norm (scale = min(1, max_norm / (||g|| + 1e-6))), then Adam
__global__ void k_adam(int n, float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, const double *__restrict__ gnorm, double max_norm, double lr,
                       double b1, double b2, double eps, double bc1, double bc2) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const double scale = fmin(1.0, max_norm / (*gnorm + 1e-6));
    const double gi = g[i] * scale;
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = static_cast<float>(mi);
    v[i] = static_cast<float>(vi);
    theta[i] = static_cast<float>(theta[i] - lr * (mi / bc1) / (sqrt(vi / bc2) + eps));
}

void gcin_engine_free(GcinEngine *e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    gcin_batch_free(e->batch);
    if (e->theta) cudaFree(e->theta);
    delete e;
}

}  // namespace amg

using namespace amg;

struct gcin_trainer {
    int device = 0;
    int bf16 = 0;
    int hidden = kHidden;            // GCIN width of the parameters
    int n = kNumParams;              // parameter count
    std::string err;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    double *part = nullptr;          // norm partials + the norm
    long long step = 0;
    GcinBatch batch;
    std::vector<const amg_ctx *> key;
    std::vector<long long> versions;
    bool have_forward = false;
};

static int tr_fail(gcin_trainer *t, int rc, const std::string &msg) {
    if (t) t->err = msg;
    return rc;
}

static int tr_cuda(gcin_trainer *t, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return AMG_OK;
    return tr_fail(t, AMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kNormBlocks = 64;

extern "C" {

int gnn_load_params(amg_ctx *c, const float *theta, long long n) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    const int H = hidden_of(n);
    if (!theta || !H) return ctx_fail(c, "expected 55045 (hidden 64) or 37189 (hidden 32) parameters"), AMG_ERR_ARG;
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
    e = cudaMemcpyAsync(c->gnn->theta, theta, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "upload params");
    c->gnn->have_params = true;
    c->gnn->hidden = H;
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
        int rc = gcin_batch_build(g->batch, 1, one, s, err, false);
        if (rc) return ctx_fail(c, err), rc;
        g->batch_version = c->hier_version;
    }
    g->batch.bf16 = (c->opt.gnn_precision == AMG_GNN_BF16) ? 1 : 0;
    g->batch.infer = 1;
    g->batch.hidden = g->hidden;
    // forward + smoother assembly (straight from the device coefficients) run
    // as one CUDA graph, captured once per batch and arithmetic: ~40 small
    // kernels whose host launch cost would otherwise exceed their run time
    const int key = g->batch.bf16 + 2 * c->opt.precision + 4 * (g->hidden == kHidden32 ? 1 : 0);
    if (!g->exec || g->exec_version != g->batch_version || g->exec_key != key) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        gcin_prepare_device();
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return ctx_cuda_check(c, e, "GCIN capture begin");
        const long long before = g_launches.load();
        gcin_forward(g->batch, g->theta, s);
        const int rc0 = enqueue_coeff_assembly(c, g->batch.c, s);
        g->exec_kernels = g_launches.load() - before;
        g_launches.fetch_sub(g->exec_kernels);
        e = cudaStreamEndCapture(s, &graph);
        if (rc0) {
            if (graph) cudaGraphDestroy(graph);
            return rc0;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g->exec = nullptr;
            return ctx_cuda_check(c, e, "GCIN graph");
        }
        g->exec_version = g->batch_version;
        g->exec_key = key;
    }
    e = cudaGraphLaunch(g->exec, s);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "GCIN graph launch");
    g_launches.fetch_add(g->exec_kernels);
    c->have_q = true;
    c->q_nodes = false;
    c->q64_stale = c->opt.precision != AMG_FP64;   // the graph assembled the FP32 values only
    c->smoother = AMG_SMOOTHER_GNN;
    int dflag = 0;
    const int G = g->batch.G;
    std::vector<float> cf(static_cast<size_t>(G) * 5);
    e = cudaMemcpyAsync(cf.data(), g->batch.c, sizeof(float) * cf.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dflag, g->batch.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "GCIN forward and smoother assembly");
    bool finite = true;
    for (size_t k = 0; k < static_cast<size_t>(G - 1) * 5; ++k) finite = finite && std::isfinite(cf[k]);   // smoothed levels
    if (dflag || !finite) {
        c->have_q = false;
        c->smoother = AMG_SMOOTHER_JACOBI;
        if (dflag) return ctx_fail(c, "tensor-core GCIN kernel timed out waiting for its MMAs"), AMG_ERR_DEVICE_FLAG;
        return ctx_fail(c, "non-finite coefficient"), AMG_ERR_ARG;
    }
    if (c_out) std::copy(cf.begin(), cf.end(), c_out);
    return AMG_OK;
}

int gcin_tc_selftest(int device, int no_commit, const float *x, const float *W, const float *bias, float *y,
                     float *h, int *flag) {
    if (!x || !W || !bias || !y || !h || !flag) return AMG_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return AMG_ERR_CUDA;
    gcin_prepare_device();
    constexpr int n = kTcRows;
    // identity graph (h = x), two 64-node tiles
    std::vector<int> rp(n + 1), col(n), tstart = {0, kTile, 2 * kTile};
    std::vector<float> w(n, 1.0f);
    for (int i = 0; i <= n; ++i) rp[i] = i;
    for (int i = 0; i < n; ++i) col[i] = i;
    char *mem = nullptr;
    Planner pl;
    auto lay = [&](Planner &P) {
        struct L { int *rp, *col, *ts, *err; float *w, *x, *W, *b, *h, *y, *tm, *t2; } l{};
        l.rp = P.take<int>(n + 1); l.col = P.take<int>(n); l.ts = P.take<int>(3); l.err = P.take<int>(4);
        l.w = P.take<float>(n); l.x = P.take<float>(n * kHidden); l.W = P.take<float>(kHidden * kHidden);
        l.b = P.take<float>(kHidden); l.h = P.take<float>(n * kHidden); l.y = P.take<float>(n * kHidden);
        l.tm = P.take<float>(2 * kHidden); l.t2 = P.take<float>(2 * kHidden);
        return l;
    };
    lay(pl);
    if (cudaMalloc(&mem, pl.off) != cudaSuccess) return AMG_ERR_CUDA;
    Planner p2;
    p2.base = mem;
    auto L = lay(p2);
    cudaError_t e = cudaMemset(mem, 0, p2.off);
    if (e == cudaSuccess) e = cudaMemcpy(L.rp, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.ts, tstart.data(), sizeof(int) * 3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.w, w.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.x, x, sizeof(float) * n * kHidden, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.W, W, sizeof(float) * kHidden * kHidden, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L.b, bias, sizeof(float) * kHidden, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_agg_lin_tc<kHidden><<<1, kBlock, tc_smem<kHidden>()>>>(L.rp, L.col, L.w, L.x, L.W, nullptr, L.b, L.ts, 2, L.h, L.y, L.tm, L.t2, L.err,
                                             no_commit ? 1 : 0); AMG_COUNT();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(y, L.y, sizeof(float) * n * kHidden, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h, L.h, sizeof(float) * n * kHidden, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(flag, L.err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    return e == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
}

int gcin_trainer_create(gcin_trainer **out, int device, int precision, const float *theta0, long long n_params) {
    if (!out || !theta0 || (precision != AMG_GNN_FP32 && precision != AMG_GNN_BF16) || !hidden_of(n_params))
        return AMG_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return AMG_ERR_CUDA;
    gcin_trainer *t = new gcin_trainer();
    t->device = device;
    t->bf16 = (precision == AMG_GNN_BF16) ? 1 : 0;
    t->hidden = hidden_of(n_params);
    t->n = static_cast<int>(n_params);
    cudaError_t e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
    const size_t P = t->n;
    const size_t fbytes = ((sizeof(float) * 4 * P + 255) / 256) * 256;
    if (e == cudaSuccess) e = cudaMalloc(&t->theta, fbytes + sizeof(double) * (kNormBlocks + 1));
    if (e != cudaSuccess) {
        if (t->stream) cudaStreamDestroy(t->stream);
        delete t;
        return AMG_ERR_CUDA;
    }
    t->grad = t->theta + P;
    t->m = t->grad + P;
    t->v = t->m + P;
    t->part = reinterpret_cast<double *>(reinterpret_cast<char *>(t->theta) + fbytes);
    e = cudaMemcpyAsync(t->theta, theta0, sizeof(float) * P, cudaMemcpyHostToDevice, t->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->grad, 0, sizeof(float) * 3 * P, t->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
    if (e != cudaSuccess) {
        gcin_trainer_destroy(t);
        return AMG_ERR_CUDA;
    }
    *out = t;
    return AMG_OK;
}

void gcin_trainer_destroy(gcin_trainer *t) {
    if (!t) return;
    cudaSetDevice(t->device);
    if (t->stream) cudaStreamSynchronize(t->stream);
    gcin_batch_free(t->batch);
    if (t->theta) cudaFree(t->theta);
    if (t->stream) cudaStreamDestroy(t->stream);
    delete t;
}

const char *gcin_trainer_last_error(const gcin_trainer *t) { return t ? t->err.c_str() : "trainer is NULL"; }

int gcin_trainer_get_params(const gcin_trainer *tc, float *theta_out) {
    gcin_trainer *t = const_cast<gcin_trainer *>(tc);
    if (!t || !theta_out) return AMG_ERR_ARG;
    int rc = tr_cuda(t, cudaSetDevice(t->device), "cudaSetDevice");
    if (rc) return rc;
    rc = tr_cuda(t, cudaMemcpyAsync(theta_out, t->theta, sizeof(float) * t->n, cudaMemcpyDeviceToHost, t->stream),
                 "params download");
    if (rc) return rc;
    return tr_cuda(t, cudaStreamSynchronize(t->stream), "sync");
}

int gcin_trainer_set_params(gcin_trainer *t, const float *theta, long long n) {
    if (!t) return AMG_ERR_ARG;
    t->err.clear();
    if (!theta || n != t->n) return tr_fail(t, AMG_ERR_ARG, "parameter count differs from the trainer's");
    int rc = tr_cuda(t, cudaSetDevice(t->device), "cudaSetDevice");
    if (rc) return rc;
    rc = tr_cuda(t, cudaMemcpyAsync(t->theta, theta, sizeof(float) * n, cudaMemcpyHostToDevice, t->stream),
                 "params upload");
    if (rc) return rc;
    t->have_forward = false;
    return tr_cuda(t, cudaStreamSynchronize(t->stream), "sync");
}

int gcin_trainer_forward(gcin_trainer *t, int n_problems, amg_ctx *const *problems, double *c_out) {
    if (!t) return AMG_ERR_ARG;
    t->err.clear();
    if (n_problems < 1 || !problems || !c_out) return tr_fail(t, AMG_ERR_ARG, "need at least one problem and c_out");
    int rc = tr_cuda(t, cudaSetDevice(t->device), "cudaSetDevice");
    if (rc) return rc;
    std::vector<const amg_ctx *> key(problems, problems + n_problems);
    std::vector<long long> versions;
    for (int m = 0; m < n_problems; ++m) {
        if (!problems[m]) return tr_fail(t, AMG_ERR_ARG, "NULL problem");
        versions.push_back(problems[m]->hier_version);
    }
    if (key != t->key || versions != t->versions || !t->batch.arena) {
        std::string err;
        rc = gcin_batch_build(t->batch, n_problems, problems, t->stream, err, true);
        if (rc) return tr_fail(t, rc, err);
        t->key = key;
        t->versions = versions;
    }
    t->batch.bf16 = t->bf16;
    t->batch.hidden = t->hidden;
    gcin_forward(t->batch, t->theta, t->stream);
    std::vector<float> cf(static_cast<size_t>(t->batch.G) * 5);
    int dflag = 0;
    rc = tr_cuda(t, cudaGetLastError(), "GCIN forward");
    if (!rc) rc = tr_cuda(t, cudaMemcpyAsync(cf.data(), t->batch.c, sizeof(float) * cf.size(), cudaMemcpyDeviceToHost,
                                             t->stream), "coefficients download");
    if (!rc) rc = tr_cuda(t, cudaMemcpyAsync(&dflag, t->batch.err, sizeof(int), cudaMemcpyDeviceToHost, t->stream),
                          "flag download");
    if (!rc) rc = tr_cuda(t, cudaStreamSynchronize(t->stream), "sync");
    if (rc) return rc;
    if (dflag) return tr_fail(t, AMG_ERR_DEVICE_FLAG, "tensor-core GCIN kernel timed out waiting for its MMAs");
    std::copy(cf.begin(), cf.end(), c_out);
    t->have_forward = true;
    return AMG_OK;
}

int gcin_trainer_backward(gcin_trainer *t, const double *dc, double *dtheta_out) {
    if (!t) return AMG_ERR_ARG;
    t->err.clear();
    if (!dc) return tr_fail(t, AMG_ERR_ARG, "dc is NULL");
    if (!t->have_forward) return tr_fail(t, AMG_ERR_STATE, "backward without a forward");
    int rc = tr_cuda(t, cudaSetDevice(t->device), "cudaSetDevice");
    if (rc) return rc;
    std::vector<float> df(dc, dc + static_cast<size_t>(t->batch.G) * 5);
    rc = tr_cuda(t, cudaMemcpyAsync(t->batch.dc, df.data(), sizeof(float) * df.size(), cudaMemcpyHostToDevice,
                                    t->stream), "dc upload");
    if (rc) return rc;
    gcin_backward(t->batch, t->theta, t->grad, t->stream);
    rc = tr_cuda(t, cudaGetLastError(), "GCIN backward");
    if (rc) return rc;
    std::vector<float> g(t->n);
    if (dtheta_out) {
        rc = tr_cuda(t, cudaMemcpyAsync(g.data(), t->grad, sizeof(float) * t->n, cudaMemcpyDeviceToHost,
                                        t->stream), "gradient download");
        if (rc) return rc;
    }
    int dflag = 0;   // the tensor-core backward's bounded MMA wait
    rc = tr_cuda(t, cudaMemcpyAsync(&dflag, t->batch.err, sizeof(int), cudaMemcpyDeviceToHost, t->stream),
                 "flag download");
    if (rc) return rc;
    rc = tr_cuda(t, cudaStreamSynchronize(t->stream), "sync");
    if (rc) return rc;
    if (dflag) return tr_fail(t, AMG_ERR_DEVICE_FLAG, "tensor-core GCIN kernel timed out waiting for its MMAs");
    if (dtheta_out) std::copy(g.begin(), g.end(), dtheta_out);
    return AMG_OK;
}

int gcin_trainer_adam_step(gcin_trainer *t, double lr, double max_norm) {
    if (!t) return AMG_ERR_ARG;
    t->err.clear();
    if (!(lr >= 0.0) || !(max_norm > 0.0)) return tr_fail(t, AMG_ERR_ARG, "bad lr or max_norm");
    int rc = tr_cuda(t, cudaSetDevice(t->device), "cudaSetDevice");
    if (rc) return rc;
    t->step += 1;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const double bc1 = 1.0 - std::pow(b1, static_cast<double>(t->step));
    const double bc2 = 1.0 - std::pow(b2, static_cast<double>(t->step));
    k_sq_partial_f<<<kNormBlocks, kBlock, 0, t->stream>>>(t->n, t->grad, t->part); AMG_COUNT();
    k_norm_from_partials<<<1, 32, 0, t->stream>>>(kNormBlocks, t->part, t->part + kNormBlocks); AMG_COUNT();
    k_adam<<<grid_for(t->n), kBlock, 0, t->stream>>>(t->n, t->theta, t->grad, t->m, t->v,
                                                           t->part + kNormBlocks, max_norm, lr, b1, b2, eps, bc1,
                                                           bc2); AMG_COUNT();
    rc = tr_cuda(t, cudaGetLastError(), "adam");
    if (rc) return rc;
    return tr_cuda(t, cudaStreamSynchronize(t->stream), "sync");
}

}  // extern "C"
