// AMG setup on the GB300 (Sec. 2.2; Algorithm 1 step 2) with a parallel
// C/F split.  Per level, all in CUDA kernels:
//   strength     j in S_i iff j != i and -a_ij >= theta max_{k != i}(-a_ik)
//                (that maximum > 0); S as CSR, S^T by counting + scatter
//   block RS     (AMG_SPLIT_RS_BLOCKS) the classical RS first pass on each
//                block of up to 4096 consecutive rows, one CTA per block with
//                the block's strength subgraph in shared memory, then every
//                F point left without a strong C point becomes C
//   PMIS split   (otherwise; De Sterck, Yang & Heys 2006) lambda_i = |S_i^T| + r_i in
//                FP64, r_i from splitmix64 (seed + level); points with
//                |S_i^T| = 0 start as F; rounds of "undecided i beats every
//                undecided j in S_i u S_i^T (ties: lower index) -> C, then
//                undecided points with a strong dependency on a new C -> F"
//                until nothing is undecided; the host reads the count of
//                undecided points after each round (at least the global
//                maximum is decided per round, so rounds <= n)
//   second pass  (optional) rounds in which the F points j with strong F
//                partners i (j in S_i, S_i n S_j n C empty) count their
//                violating pairs v_j, and candidates beating every candidate
//                of S_j u S_j^T (v + r, ties to the lower index) become C,
//                until no pair violates (the top candidate is promoted each
//                round, so rounds <= n)
//   direct interpolation, one thread per row in the row's entry order
//   R = P^T      counting transpose, rows sorted by column
//   Galerkin     A_c = R (A P): two row-wise products, a warp per row: the
//                row's columns hashed into its own open-addressing table
//                (load <= 2/3), compacted and rank-sorted; each entry then
//                summed over the row in ascending order (the Gustavson order)
// Offsets come from a three-phase exclusive scan.  The same stopping rules as
// the host setup; the finished levels stay on the device (their row pointers
// are copied to the host).
//
// Also here: the products the latency-optimised (small) levels use, for
// hierarchies from either setup: the pattern of A A (that of M A, M = Q^-1 on
// A's pattern) with the pair list assembling M A, and R A.
#include "setup_device.h"

#include <algorithm>
#include <cstdint>

#include "amg_gnn.h"
#include "common.cuh"

namespace amg {
namespace {

constexpr int8_t kF = 0, kC = 1, kU = -1;

struct DevCSR {
    int n_rows = 0, n_cols = 0;
    long long nnz = 0;
    int *rp = nullptr, *col = nullptr;
    double *val = nullptr;
};

// device allocations of one setup call: 256-byte aligned pieces cut from
// chunks of at least 64 MB (a few cudaMalloc calls instead of hundreds),
// freed together
struct Pool {
    static constexpr size_t kChunk = size_t(64) << 20;
    std::vector<void *> chunks;
    char *cur = nullptr;
    size_t left = 0;
    cudaError_t err = cudaSuccess;
    template <class T>
    T *get(long long n) {
        if (err != cudaSuccess) return nullptr;
        const size_t bytes = (static_cast<size_t>(std::max<long long>(1, n)) * sizeof(T) + 255) & ~size_t(255);
        if (bytes > left) {
            const size_t cb = std::max(bytes, kChunk);
            void *p = nullptr;
            err = cudaMalloc(&p, cb);
            if (err != cudaSuccess) return nullptr;
            chunks.push_back(p);
            cur = static_cast<char *>(p);
            left = cb;
        }
        T *r = reinterpret_cast<T *>(cur);
        cur += bytes;
        left -= bytes;
        return r;
    }
    ~Pool() {
        for (void *p : chunks) cudaFree(p);
    }
};

// ---------------------------------------------------------------------------
// exclusive scan (out may alias in)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256, kScanItems = 4, kScanTile = kScanBlock * kScanItems;

template <class T>
__global__ void __launch_bounds__(kScanBlock) k_scan_tile(const T *in, T *out, T *__restrict__ tile_sum, long long n) {
    __shared__ T warp_tot[kScanBlock / 32];
    const long long base = static_cast<long long>(blockIdx.x) * kScanTile + static_cast<long long>(threadIdx.x) * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? in[base + j] : T(0);
        s += v[j];
    }
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    T inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    T woff = 0;
    for (int k = 0; k < w; ++k) woff += warp_tot[k];
    T run = woff + inc - s;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == kScanBlock - 1) tile_sum[blockIdx.x] = woff + inc;
}

template <class T>
__global__ void k_scan_add(T *out, const T *__restrict__ tile_off, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (i < n) out[i] += tile_off[i / kScanTile];
}

template <class T>
cudaError_t exclusive_scan(const T *in, T *out, long long n, Pool &pool, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long nt = (n + kScanTile - 1) / kScanTile;
    T *sums = pool.get<T>(nt);
    if (!sums) return pool.err;
    k_scan_tile<T><<<static_cast<unsigned>(nt), kScanBlock, 0, s>>>(in, out, sums, n); AMG_COUNT();
    if (nt > 1) {
        const cudaError_t e = exclusive_scan<T>(sums, sums, nt, pool, s);
        if (e != cudaSuccess) return e;
        k_scan_add<T><<<grid_for(n), kBlock, 0, s>>>(out, sums, n); AMG_COUNT();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// strength graph
// ---------------------------------------------------------------------------
__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const double *__restrict__ val, double theta, uint8_t *__restrict__ strong,
                           int *__restrict__ scnt) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    bool has_off = false;
    double m = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        if (col[p] == i) continue;
        const double neg = -val[p];
        if (!has_off || neg > m) m = neg;
        has_off = true;
    }
    int cnt = 0;
    if (has_off && m > 0.0) {
        const double thr = theta * m;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const uint8_t st = (col[p] != i && -val[p] >= thr) ? 1 : 0;
            strong[p] = st;
            cnt += st;
        }
    } else {
        for (int p = rp[i]; p < rp[i + 1]; ++p) strong[p] = 0;
    }
    scnt[i] = cnt;
}

__global__ void k_fill_strong(int n, const int *__restrict__ rp, const int *__restrict__ col,
                              const uint8_t *__restrict__ strong, const int *__restrict__ S_rp,
                              int *__restrict__ S_col) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    int o = S_rp[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (strong[p]) S_col[o++] = col[p];
}

__global__ void k_count_cols(int n, const int *__restrict__ rp, const int *__restrict__ col, int *__restrict__ cnt) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) atomicAdd(cnt + col[p], 1);
}

// scatter of a transpose (entries of a row land in arbitrary order)
__global__ void k_scatter_transpose(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                    const double *__restrict__ val, int *__restrict__ cursor, int *__restrict__ T_col,
                                    double *__restrict__ T_val) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int at = atomicAdd(cursor + col[p], 1);
        T_col[at] = i;
        if (T_val) T_val[at] = val[p];
    }
}

template <class V>
__device__ void heap_sort(int *K, V *W, int u);

// sort each row by column (values carried along)
__global__ void k_sort_rows(int n, const int *__restrict__ rp, int *__restrict__ col, double *__restrict__ val) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const int p0 = rp[i];
    heap_sort(col + p0, val + p0, rp[i + 1] - p0);
}

// ---------------------------------------------------------------------------
// PMIS
// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood 2014): output k of the sequence started at
// `seed`, mapped to [0, 1) by its top 53 bits
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return static_cast<double>(z >> 11) * 0x1.0p-53;
}

__global__ void k_pmis_init(int n, const int *__restrict__ T_rp, unsigned long long seed, double *__restrict__ lam,
                            int8_t *__restrict__ state) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const int d = T_rp[i + 1] - T_rp[i];
    lam[i] = static_cast<double>(d) + splitmix_uniform(seed, static_cast<unsigned long long>(i) + 1ull);
    state[i] = d == 0 ? kF : kU;
}

__device__ __forceinline__ bool beats(double li, int i, double lj, int j) { return li > lj || (li == lj && i < j); }

__global__ void k_pmis_select(int n, const int *__restrict__ S_rp, const int *__restrict__ S_col,
                              const int *__restrict__ T_rp, const int *__restrict__ T_col,
                              const double *__restrict__ lam, const int8_t *__restrict__ state,
                              int8_t *__restrict__ newc) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    int8_t win = 0;
    if (state[i] == kU) {
        win = 1;
        const double li = lam[i];
        for (int p = S_rp[i]; p < S_rp[i + 1] && win; ++p) {
            const int j = S_col[p];
            if (state[j] == kU && !beats(li, i, lam[j], j)) win = 0;
        }
        for (int p = T_rp[i]; p < T_rp[i + 1] && win; ++p) {
            const int j = T_col[p];
            if (state[j] == kU && !beats(li, i, lam[j], j)) win = 0;
        }
    }
    newc[i] = win;
}

__global__ void k_pmis_update(int n, const int *__restrict__ S_rp, const int *__restrict__ S_col,
                              const int8_t *__restrict__ newc, int8_t *__restrict__ state, int *__restrict__ remaining) {
    __shared__ int red[kBlock / 32];
    const int i = blockIdx.x * kBlock + threadIdx.x;
    int still = 0;
    if (i < n && state[i] == kU) {
        if (newc[i]) {
            state[i] = kC;
        } else {
            bool f = false;
            for (int p = S_rp[i]; p < S_rp[i + 1] && !f; ++p) f = newc[S_col[p]] != 0;
            if (f) state[i] = kF;
            else still = 1;
        }
    }
    still = warp_sum(still);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = still;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < kBlock / 32; ++k) t += red[k];
        if (t) atomicAdd(remaining, t);
    }
}

// v_j += 1 for every F point i with j in S_i an F point and no common strong
// C point (S rows are sorted: a merge of the two rows)
__global__ void k_h1_violations(int n, const int *__restrict__ S_rp, const int *__restrict__ S_col,
                                const int8_t *__restrict__ state, int *__restrict__ v, int *__restrict__ total) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n || state[i] != kF) return;
    int mine = 0;
    const int pe = S_rp[i + 1];
    for (int p0 = S_rp[i]; p0 < pe; ++p0) {
        const int j = S_col[p0];
        if (state[j] != kF) continue;
        bool share = false;
        int p = S_rp[i], q = S_rp[j];
        const int qe = S_rp[j + 1];
        while (p < pe && q < qe && !share) {
            const int a = S_col[p], b = S_col[q];
            if (a == b) {
                share = state[a] == kC;
                ++p;
                ++q;
            } else if (a < b) {
                ++p;
            } else {
                ++q;
            }
        }
        if (!share) {
            atomicAdd(v + j, 1);
            ++mine;
        }
    }
    if (mine) atomicAdd(total, mine);
}

// candidates (v_j > 0) that beat every candidate of S_j u S_j^T become C
__global__ void k_h1_promote(int n, const int *__restrict__ S_rp, const int *__restrict__ S_col,
                             const int *__restrict__ T_rp, const int *__restrict__ T_col, const int *__restrict__ v,
                             unsigned long long seed, int8_t *__restrict__ state) {
    const int j = blockIdx.x * kBlock + threadIdx.x;
    if (j >= n || v[j] == 0) return;
    const double wj = static_cast<double>(v[j]) + splitmix_uniform(seed, static_cast<unsigned long long>(j) + 1ull);
    bool win = true;
    for (int p = S_rp[j]; p < S_rp[j + 1] && win; ++p) {
        const int k = S_col[p];
        if (v[k] && !beats(wj, j, static_cast<double>(v[k]) + splitmix_uniform(seed, static_cast<unsigned long long>(k) + 1ull), k))
            win = false;
    }
    for (int p = T_rp[j]; p < T_rp[j + 1] && win; ++p) {
        const int k = T_col[p];
        if (v[k] && !beats(wj, j, static_cast<double>(v[k]) + splitmix_uniform(seed, static_cast<unsigned long long>(k) + 1ull), k))
            win = false;
    }
    if (win) state[j] = kC;
}

__global__ void k_cflag(int n, const int8_t *__restrict__ state, int *__restrict__ cflag) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) cflag[i] = state[i] == kC ? 1 : 0;
}

// ---------------------------------------------------------------------------
// block-local Ruge-Stueben split
// ---------------------------------------------------------------------------
// Consecutive blocks of B rows each run the classical first pass on their
// induced strength subgraph (pairs with both points in the block).  B is the
// largest of 4096, 2048, ..., 128 for which no block holds more than
// kRsMaxPairs strong pairs, so a block's two restricted adjacency lists fit
// one CTA's shared memory (128 always fits: 128 * 127 < kRsMaxPairs).
constexpr int kRsMaxPairs = 32768;
constexpr int kRsMaxBlock = 4096;
constexpr int kRsSizes = 5;          // B = 256 << k, k = 0 .. 4 counted; 128 always fits
constexpr int kRsThreads = 128;

// Strong pairs inside the row's block for B = 256 << k, summed per 256-row
// CTA: part[kRsSizes c + k].
__global__ void __launch_bounds__(kBlock) k_rs_pairs(int n, const int *__restrict__ S_rp,
                                                     const int *__restrict__ S_col, int *__restrict__ part) {
    __shared__ int red[kRsSizes][kBlock / 32];
    const int i = blockIdx.x * kBlock + threadIdx.x;
    int c[kRsSizes] = {};
    if (i < n) {
        for (int p = S_rp[i]; p < S_rp[i + 1]; ++p) {
            const int j = S_col[p];
#pragma unroll
            for (int k = 0; k < kRsSizes; ++k) c[k] += (j >> (8 + k)) == (i >> (8 + k));
        }
    }
#pragma unroll
    for (int k = 0; k < kRsSizes; ++k) {
        const int v = warp_sum(c[k]);
        if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRsSizes) {
        int t = 0;
        for (int w = 0; w < kBlock / 32; ++w) t += red[threadIdx.x][w];
        part[kRsSizes * blockIdx.x + threadIdx.x] = t;
    }
}

// worst[k] = the largest block sum of part for B = 256 << k: groups of 2^k
// consecutive CTAs (one CTA)
__global__ void __launch_bounds__(kBlock) k_rs_pairs_max(int nparts, const int *__restrict__ part,
                                                         int *__restrict__ worst) {
    __shared__ int red[kRsSizes][kBlock / 32];
    int m[kRsSizes] = {};
    for (int g = threadIdx.x; g < nparts; g += kBlock) {
#pragma unroll
        for (int k = 0; k < kRsSizes; ++k) {
            if (g % (1 << k)) continue;
            int t = 0;
            for (int q = g; q < min(g + (1 << k), nparts); ++q) t += part[kRsSizes * q + k];
            m[k] = max(m[k], t);
        }
    }
#pragma unroll
    for (int k = 0; k < kRsSizes; ++k) {
        int v = m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRsSizes) {
        int t = 0;
        for (int w = 0; w < kBlock / 32; ++w) t = max(t, red[threadIdx.x][w]);
        worst[threadIdx.x] = t;
    }
}

// exclusive scan of cnt[0 .. m) into ptr[0 .. m] by warp 0 (m <= 1024)
__device__ void rs_warp_scan(const int *cnt, int *ptr, int m) {
    const int lane = threadIdx.x % 32;
    const int per = (m + 31) / 32, a = min(m, lane * per), e = min(m, a + per);
    int tot = 0;
    for (int k = a; k < e; ++k) tot += cnt[k];
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    int run = inc - tot;
    for (int k = a; k < e; ++k) {
        ptr[k] = run;
        run += cnt[k];
    }
    if (lane == 31) ptr[m] = inc;
}

// One CTA per block of B rows.  Shared memory: the block's S and S^T rows
// restricted to the block (local indices), lambda, the states and a list of
// the points made F by the current selection.  Each step of the first pass
// takes the undecided point of largest (lambda, -index) as C (the CTA-wide
// maximum of (lambda + 1) << 16 | (65535 - k)); warp 0 then makes its
// undecided block dependents F, raises lambda_k for every undecided k that a
// new F point strongly depends on and lowers it for every undecided k the new
// C point strongly depends on.  Those updates commute (the increments reach
// only points that stay undecided), so lanes apply them in any order with
// shared-memory atomics and the result is that of the sequential pass.  Each
// step decides at least one point: at most B steps.
__global__ void __launch_bounds__(kRsThreads) k_rs_block(int n, int B, int max_pairs, const int *__restrict__ S_rp,
                                                         const int *__restrict__ S_col, const int *__restrict__ T_rp,
                                                         const int *__restrict__ T_col, int8_t *__restrict__ state) {
    extern __shared__ __align__(16) unsigned char rs_buf[];
    int *sp = reinterpret_cast<int *>(rs_buf);          // B + 1
    int *tp = sp + (B + 1);                              // B + 1
    int *lam = tp + (B + 1);                             // B (first the S counts)
    int *tcnt = lam + B;                                 // B
    unsigned short *sc = reinterpret_cast<unsigned short *>(tcnt + B);   // max_pairs
    unsigned short *tc = sc + max_pairs;                                  // max_pairs
    unsigned short *newf = tc + max_pairs;                                // B
    int8_t *st = reinterpret_cast<int8_t *>(newf + B);                    // B
    const int b0 = blockIdx.x * B, m = min(B, n - b0), b1 = b0 + m;
    const int lane = threadIdx.x % 32;
    // restricted row lengths
    for (int k = threadIdx.x; k < m; k += kRsThreads) {
        const int i = b0 + k;
        int cs = 0, ct = 0;
        for (int p = S_rp[i]; p < S_rp[i + 1]; ++p) cs += (S_col[p] >= b0 && S_col[p] < b1);
        for (int p = T_rp[i]; p < T_rp[i + 1]; ++p) ct += (T_col[p] >= b0 && T_col[p] < b1);
        lam[k] = cs;
        tcnt[k] = ct;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        rs_warp_scan(lam, sp, m);
        rs_warp_scan(tcnt, tp, m);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += kRsThreads) {
        const int i = b0 + k;
        int q = sp[k];
        for (int p = S_rp[i]; p < S_rp[i + 1]; ++p) {
            const int j = S_col[p];
            if (j >= b0 && j < b1) sc[q++] = static_cast<unsigned short>(j - b0);
        }
        q = tp[k];
        for (int p = T_rp[i]; p < T_rp[i + 1]; ++p) {
            const int j = T_col[p];
            if (j >= b0 && j < b1) tc[q++] = static_cast<unsigned short>(j - b0);
        }
        const int ns = sp[k + 1] - sp[k], nt = tp[k + 1] - tp[k];
        lam[k] = nt;
        st[k] = (ns == 0 && nt == 0) ? kF : kU;
    }
    __syncthreads();
    __shared__ unsigned red[kRsThreads / 32];
    for (int step = 0; step <= m; ++step) {
        unsigned best = 0;
        for (int k = threadIdx.x; k < m; k += kRsThreads)
            if (st[k] == kU) best = max(best, (static_cast<unsigned>(lam[k] + 1) << 16) | (65535u - k));
        best = __reduce_max_sync(0xffffffffu, best);
        if (lane == 0) red[threadIdx.x / 32] = best;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w) best = max(best, red[w]);
        if (best == 0) break;                                   // the same value in every thread
        if (threadIdx.x < 32) {
            const int i = 65535 - static_cast<int>(best & 0xFFFFu);
            if (lane == 0) st[i] = kC;
            __syncwarp();
            // undecided block dependents of i become F
            int nf = 0;
            for (int q0 = tp[i]; q0 < tp[i + 1]; q0 += 32) {
                const int q = q0 + lane;
                const int j = q < tp[i + 1] ? tc[q] : 0;
                const bool fresh = q < tp[i + 1] && st[j] == kU;
                const unsigned mask = __ballot_sync(0xffffffffu, fresh);
                if (fresh) {
                    newf[nf + __popc(mask & ((1u << lane) - 1u))] = static_cast<unsigned short>(j);
                    st[j] = kF;
                }
                nf += __popc(mask);
            }
            __syncwarp();
            for (int e = lane; e < nf; e += 32) {
                const int j = newf[e];
                for (int q = sp[j]; q < sp[j + 1]; ++q)
                    if (st[sc[q]] == kU) atomicAdd(lam + sc[q], 1);
            }
            for (int q = sp[i] + lane; q < sp[i + 1]; q += 32)
                if (st[sc[q]] == kU) atomicSub(lam + sc[q], 1);
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < m; k += kRsThreads) state[b0 + k] = st[k] == kC ? kC : kF;
}

inline int rs_smem(int B, int max_pairs) {
    return ((2 * (B + 1) + 2 * B) * 4 + 2 * max_pairs * 2 + B * 2 + B + 15) / 16 * 16;
}

// Repair after the block split: an F point with strong dependencies but none
// on a C point (its strong couplings all leave its block) becomes C, all
// decided from the split as it stands (mark, then apply).
__global__ void k_rs_repair_mark(int n, const int *__restrict__ S_rp, const int *__restrict__ S_col,
                                 const int8_t *__restrict__ state, int8_t *__restrict__ mark) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    bool m = state[i] == kF && S_rp[i + 1] > S_rp[i];
    for (int p = S_rp[i]; p < S_rp[i + 1] && m; ++p) m = state[S_col[p]] != kC;
    mark[i] = m ? 1 : 0;
}

__global__ void k_rs_repair_apply(int n, const int8_t *__restrict__ mark, int8_t *__restrict__ state) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n && mark[i]) state[i] = kC;
}

// ---------------------------------------------------------------------------
// direct interpolation (one thread per row, the row's entry order)
// ---------------------------------------------------------------------------
__global__ void k_interp_count(int n, const int *__restrict__ rp, const int *__restrict__ col,
                               const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                               int *__restrict__ pcnt) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    if (state[i] == kC) {
        pcnt[i] = 1;
        return;
    }
    int c = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) c += (strong[p] && state[col[p]] == kC) ? 1 : 0;
    pcnt[i] = c;
}

// C rows: identity onto the coarse numbering.  F row i with strong C
// neighbours C_i: w_ij = -alpha_i a_ij / d_i, alpha_i = (sum of the negative
// off-diagonal a_ik) / (sum over C_i of a_ik), d_i = a_ii + (sum of the
// positive off-diagonal a_ik); sums taken in the row's entry order.
__global__ void k_interp_fill(int n, const int *__restrict__ rp, const int *__restrict__ col,
                              const double *__restrict__ val, const uint8_t *__restrict__ strong,
                              const int8_t *__restrict__ state, const int *__restrict__ cidx,
                              const int *__restrict__ P_rp, int *__restrict__ P_col, double *__restrict__ P_val) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    int o = P_rp[i];
    if (state[i] == kC) {
        P_col[o] = cidx[i];
        P_val[o] = 1.0;
        return;
    }
    if (P_rp[i + 1] == o) return;    // no strong C neighbour: empty row
    double a_ii = 0.0, neg_all = 0.0, pos_all = 0.0, neg_c = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = col[p];
        const double a = val[p];
        if (j == i) {
            a_ii += a;
        } else if (a < 0.0) {
            neg_all += a;
            if (strong[p] && state[j] == kC) neg_c += a;
        } else if (a > 0.0) {
            pos_all += a;
        }
    }
    const double d = a_ii + pos_all;
    const double alpha = neg_all / neg_c;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = col[p];
        if (j != i && strong[p] && state[j] == kC) {
            P_col[o] = cidx[j];
            P_val[o] = (-alpha * val[p]) / d;
            ++o;
        }
    }
}

// ---------------------------------------------------------------------------
// row-wise sparse product Z = X Y
// ---------------------------------------------------------------------------
// In-place heapsort of u (key, value) pairs by key (keys distinct): a
// thread's own row, O(u log u) where the rows of dense coarse levels hold
// hundreds of entries.
template <class V>
__device__ void heap_sift(int *K, V *W, int root, int end) {
    while (true) {
        int child = 2 * root + 1;
        if (child >= end) return;
        if (child + 1 < end && K[child + 1] > K[child]) ++child;
        if (K[root] >= K[child]) return;
        const int tk = K[root];
        K[root] = K[child];
        K[child] = tk;
        const V tv = W[root];
        W[root] = W[child];
        W[child] = tv;
        root = child;
    }
}

template <class V>
__device__ void heap_sort(int *K, V *W, int u) {
    for (int r = u / 2 - 1; r >= 0; --r) heap_sift(K, W, r, u);
    for (int end = u - 1; end > 0; --end) {
        const int tk = K[0];
        K[0] = K[end];
        K[end] = tk;
        const V tv = W[0];
        W[0] = W[end];
        W[end] = tv;
        heap_sift(K, W, 0, end);
    }
}

__global__ void k_spgemm_size(int nX, const int *__restrict__ X_rp, const int *__restrict__ X_col,
                              const int *__restrict__ Y_rp, long long *__restrict__ hsz) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= nX) return;
    long long ub = 0;
    for (int p = X_rp[i]; p < X_rp[i + 1]; ++p) {
        const int k = X_col[p];
        ub += Y_rp[k + 1] - Y_rp[k];
    }
    long long h = 0;
    if (ub > 0) {
        h = 1;
        while (h < ub + ub / 2 + 1) h <<= 1;
    }
    hsz[i] = h;
}

// The products below take one warp per output row i.  Symbolic pass: the
// lanes insert every column j of Y_k, k in X_i, into the row's own
// open-addressing table (atomicCAS on the key), compact the distinct columns
// to the front of the table in slot order (ballot prefix), rank each column
// by the number of smaller ones and write them sorted to skeys; cnt[i] = the
// number of columns.  Numeric pass: lane t owns output entries t, t + 32, ...
// and sums x_ik y_kj over k in X_i in ascending order, finding j in the
// sorted row Y_k by binary search: the row-by-row (Gustavson) summation order
// of each entry, deterministic and without atomics on values.
__device__ __forceinline__ int find_sorted(const int *__restrict__ col, int lo, int hi, int j) {
    // index of j in col[lo, hi) (ascending), or -1
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int c = col[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

__global__ void k_sym_warp(int nX, const int *__restrict__ X_rp, const int *__restrict__ X_col,
                           const int *__restrict__ Y_rp, const int *__restrict__ Y_col,
                           const long long *__restrict__ hoff, int *__restrict__ table, int *__restrict__ skeys,
                           int *__restrict__ cnt) {
    const long long wid = (static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (wid >= nX) return;                       // warp-uniform
    const int i = static_cast<int>(wid);
    const long long o = hoff[i], size = hoff[i + 1] - o;
    if (size == 0) {
        if (lane == 0) cnt[i] = 0;
        return;
    }
    int *T = table + o;
    const unsigned long long mask = static_cast<unsigned long long>(size) - 1ull;
    for (long long t = lane; t < size; t += 32) T[t] = -1;
    __syncwarp();
    for (int p = X_rp[i]; p < X_rp[i + 1]; ++p) {
        const int k = X_col[p];
        for (int q = Y_rp[k] + lane; q < Y_rp[k + 1]; q += 32) {
            const int j = Y_col[q];
            unsigned long long h = (static_cast<unsigned long long>(static_cast<unsigned>(j)) * 0x9E3779B1ull) & mask;
            while (true) {
                const int prev = atomicCAS(T + h, -1, j);
                if (prev == -1 || prev == j) break;
                h = (h + 1ull) & mask;
            }
        }
    }
    __syncwarp();
    int u = 0;                                   // distinct columns so far (warp-uniform)
    for (long long base = 0; base < size; base += 32) {
        const long long t = base + lane;
        const int key = t < size ? T[t] : -1;
        const unsigned occ = __ballot_sync(0xffffffffu, key != -1);
        __syncwarp();                            // every lane has read its slot before any write
        if (key != -1) T[u + __popc(occ & ((1u << lane) - 1u))] = key;
        u += __popc(occ);
        __syncwarp();
    }
    for (int a = lane; a < u; a += 32) {
        const int key = T[a];
        int rank = 0;
        for (int b2 = 0; b2 < u; ++b2) rank += T[b2] < key ? 1 : 0;
        skeys[o + rank] = key;
    }
    if (lane == 0) cnt[i] = u;
}

__global__ void k_num_warp(int nX, const int *__restrict__ X_rp, const int *__restrict__ X_col,
                           const double *__restrict__ X_val, const int *__restrict__ Y_rp,
                           const int *__restrict__ Y_col, const double *__restrict__ Y_val,
                           const long long *__restrict__ hoff, const int *__restrict__ skeys,
                           const int *__restrict__ Z_rp, int *__restrict__ Z_col, double *__restrict__ Z_val) {
    const long long wid = (static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (wid >= nX) return;
    const int i = static_cast<int>(wid);
    const long long o = hoff[i];
    const int w = Z_rp[i], u = Z_rp[i + 1] - w;
    for (int t = lane; t < u; t += 32) {
        const int j = skeys[o + t];
        double acc = 0.0;
        for (int p = X_rp[i]; p < X_rp[i + 1]; ++p) {
            const int k = X_col[p];
            const int q = find_sorted(Y_col, Y_rp[k], Y_rp[k + 1], j);
            if (q >= 0) acc += X_val[p] * Y_val[q];
        }
        Z_col[w + t] = j;
        Z_val[w + t] = acc;
    }
}

// Pattern of A A (sorted columns) with the number of pairs (p, q) of each entry.
__global__ void k_pat_count_warp(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                 const long long *__restrict__ hoff, const int *__restrict__ skeys,
                                 const int *__restrict__ Z_rp, int *__restrict__ Z_col, int *__restrict__ entry_cnt) {
    const long long wid = (static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (wid >= n) return;
    const int i = static_cast<int>(wid);
    const long long o = hoff[i];
    const int w = Z_rp[i], u = Z_rp[i + 1] - w;
    for (int t = lane; t < u; t += 32) {
        const int j = skeys[o + t];
        int c = 0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int k = col[p];
            c += find_sorted(col, rp[k], rp[k + 1], j) >= 0 ? 1 : 0;
        }
        Z_col[w + t] = j;
        entry_cnt[w + t] = c;
    }
}

// Pair list of M A: entry e's pairs (p, q) from pair_ptr[e], in ascending p
// (the host planner's order).
__global__ void k_pairs_warp(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const int *__restrict__ Z_rp, const int *__restrict__ Z_col,
                             const int *__restrict__ pair_ptr, int *__restrict__ pair_p, int *__restrict__ pair_q) {
    const long long wid = (static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (wid >= n) return;
    const int i = static_cast<int>(wid);
    for (int e = Z_rp[i] + lane; e < Z_rp[i + 1]; e += 32) {
        const int j = Z_col[e];
        int at = pair_ptr[e];
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int k = col[p];
            const int q = find_sorted(col, rp[k], rp[k + 1], j);
            if (q >= 0) {
                pair_p[at] = p;
                pair_q[at] = q;
                ++at;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct Fail {
    std::string msg;
};

void check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw Fail{std::string(what) + ": " + cudaGetErrorString(e)};
}

template <class T>
T read_one(const T *d, cudaStream_t s) {
    T v{};
    check(cudaMemcpyAsync(&v, d, sizeof(T), cudaMemcpyDeviceToHost, s), "read back");
    check(cudaStreamSynchronize(s), "synchronise");
    return v;
}

template <class T>
T *need(Pool &pool, long long n) {
    T *p = pool.get<T>(n);
    if (!p) check(pool.err, "cudaMalloc");
    return p;
}

// counts[0..n) filled by the caller's kernel; counts[n] = 0; scanned in place
template <class T>
T scan_counts(T *counts, long long n, Pool &pool, cudaStream_t s) {
    check(exclusive_scan<T>(counts, counts, n + 1, pool, s), "scan");
    return read_one(counts + n, s);
}

DevCSR transpose_sorted(const DevCSR &M, Pool &pool, cudaStream_t s) {
    DevCSR T;
    T.n_rows = M.n_cols;
    T.n_cols = M.n_rows;
    T.nnz = M.nnz;
    T.rp = need<int>(pool, T.n_rows + 1);
    check(cudaMemsetAsync(T.rp, 0, sizeof(int) * (T.n_rows + 1), s), "memset");
    k_count_cols<<<grid_for(M.n_rows), kBlock, 0, s>>>(M.n_rows, M.rp, M.col, T.rp); AMG_COUNT();
    scan_counts<int>(T.rp, T.n_rows, pool, s);
    int *cursor = need<int>(pool, T.n_rows);
    check(cudaMemcpyAsync(cursor, T.rp, sizeof(int) * T.n_rows, cudaMemcpyDeviceToDevice, s), "copy");
    T.col = need<int>(pool, T.nnz);
    T.val = need<double>(pool, T.nnz);
    k_scatter_transpose<<<grid_for(M.n_rows), kBlock, 0, s>>>(M.n_rows, M.rp, M.col, M.val, cursor, T.col, T.val); AMG_COUNT();
    k_sort_rows<<<grid_for(T.n_rows), kBlock, 0, s>>>(T.n_rows, T.rp, T.col, T.val); AMG_COUNT();
    return T;
}

DevCSR spgemm(const DevCSR &X, const DevCSR &Y, Pool &pool, cudaStream_t s) {
    const int n = X.n_rows;
    long long *hoff = need<long long>(pool, n + 1);
    check(cudaMemsetAsync(hoff + n, 0, sizeof(long long), s), "memset");
    k_spgemm_size<<<grid_for(n), kBlock, 0, s>>>(n, X.rp, X.col, Y.rp, hoff); AMG_COUNT();
    const long long total = scan_counts<long long>(hoff, n, pool, s);
    if (total > 2000000000LL) throw Fail{"sparse product too large for 32-bit offsets"};
    int *table = need<int>(pool, total), *skeys = need<int>(pool, total);
    DevCSR Z;
    Z.n_rows = n;
    Z.n_cols = Y.n_cols;
    Z.rp = need<int>(pool, n + 1);
    check(cudaMemsetAsync(Z.rp + n, 0, sizeof(int), s), "memset");
    const int wg = grid_for(static_cast<long long>(n) * 32);
    k_sym_warp<<<wg, kBlock, 0, s>>>(n, X.rp, X.col, Y.rp, Y.col, hoff, table, skeys, Z.rp); AMG_COUNT();
    Z.nnz = scan_counts<int>(Z.rp, n, pool, s);
    Z.col = need<int>(pool, Z.nnz);
    Z.val = need<double>(pool, Z.nnz);
    k_num_warp<<<wg, kBlock, 0, s>>>(n, X.rp, X.col, X.val, Y.rp, Y.col, Y.val, hoff, skeys, Z.rp, Z.col, Z.val); AMG_COUNT();
    check(cudaGetLastError(), "sparse product");
    return Z;
}

void download(const DevCSR &M, HostCSR &h, cudaStream_t s) {
    h.n_rows = M.n_rows;
    h.n_cols = M.n_cols;
    h.rp.resize(M.n_rows + 1);
    h.col.resize(M.nnz);
    h.val.resize(M.nnz);
    check(cudaMemcpyAsync(h.rp.data(), M.rp, sizeof(int) * (M.n_rows + 1), cudaMemcpyDeviceToHost, s), "download");
    if (M.nnz) {
        check(cudaMemcpyAsync(h.col.data(), M.col, sizeof(int) * M.nnz, cudaMemcpyDeviceToHost, s), "download");
        check(cudaMemcpyAsync(h.val.data(), M.val, sizeof(double) * M.nnz, cudaMemcpyDeviceToHost, s), "download");
    }
}

// a level described on the device (row pointers copied to the host too)
void describe(const DevCSR &M, HostCSR &h, cudaStream_t s) {
    h.n_rows = M.n_rows;
    h.n_cols = M.n_cols;
    h.rp.resize(M.n_rows + 1);
    h.col.clear();
    h.val.clear();
    check(cudaMemcpyAsync(h.rp.data(), M.rp, sizeof(int) * (M.n_rows + 1), cudaMemcpyDeviceToHost, s), "download");
    h.drp = M.rp;
    h.dcol = M.col;
    h.dval = M.val;
}

DevCSR upload_csr(const HostCSR &h, Pool &pool, cudaStream_t s) {
    DevCSR M;
    M.n_rows = h.n_rows;
    M.n_cols = h.n_cols;
    M.nnz = h.nnz();
    if (h.on_device()) {   // already there
        M.rp = const_cast<int *>(h.drp);
        M.col = const_cast<int *>(h.dcol);
        M.val = const_cast<double *>(h.dval);
        return M;
    }
    M.rp = need<int>(pool, M.n_rows + 1);
    M.col = need<int>(pool, M.nnz);
    M.val = need<double>(pool, M.nnz);
    check(cudaMemcpyAsync(M.rp, h.rp.data(), sizeof(int) * (M.n_rows + 1), cudaMemcpyHostToDevice, s), "upload");
    if (M.nnz) {
        check(cudaMemcpyAsync(M.col, h.col.data(), sizeof(int) * M.nnz, cudaMemcpyHostToDevice, s), "upload");
        check(cudaMemcpyAsync(M.val, h.val.data(), sizeof(double) * M.nnz, cudaMemcpyHostToDevice, s), "upload");
    }
    return M;
}

void plan_products(HostLevel &H, Pool &pool, cudaStream_t s) {
    const DevCSR A = upload_csr(H.A, pool, s);
    const DevCSR R = upload_csr(H.R, pool, s);
    const int n = A.n_rows;
    // pattern of A A with per-entry pair counts
    long long *hoff = need<long long>(pool, n + 1);
    check(cudaMemsetAsync(hoff + n, 0, sizeof(long long), s), "memset");
    k_spgemm_size<<<grid_for(n), kBlock, 0, s>>>(n, A.rp, A.col, A.rp, hoff); AMG_COUNT();
    const long long total = scan_counts<long long>(hoff, n, pool, s);
    if (total > 2000000000LL) throw Fail{"product pattern too large for 32-bit offsets"};
    int *table = need<int>(pool, total), *skeys = need<int>(pool, total);
    int *Z_rp = need<int>(pool, n + 1);
    check(cudaMemsetAsync(Z_rp + n, 0, sizeof(int), s), "memset");
    const int wg = grid_for(static_cast<long long>(n) * 32);
    k_sym_warp<<<wg, kBlock, 0, s>>>(n, A.rp, A.col, A.rp, A.col, hoff, table, skeys, Z_rp); AMG_COUNT();
    const int nz = scan_counts<int>(Z_rp, n, pool, s);
    int *Z_col = need<int>(pool, nz);
    int *pp = need<int>(pool, static_cast<long long>(nz) + 1);
    check(cudaMemsetAsync(pp + nz, 0, sizeof(int), s), "memset");
    k_pat_count_warp<<<wg, kBlock, 0, s>>>(n, A.rp, A.col, hoff, skeys, Z_rp, Z_col, pp); AMG_COUNT();
    const int npairs = scan_counts<int>(pp, nz, pool, s);
    int *pair_p = need<int>(pool, npairs), *pair_q = need<int>(pool, npairs);
    k_pairs_warp<<<wg, kBlock, 0, s>>>(n, A.rp, A.col, Z_rp, Z_col, pp, pair_p, pair_q); AMG_COUNT();
    const DevCSR RA = spgemm(R, A, pool, s);
    // back to the host level
    H.MA = HostCSR{};
    H.MA.n_rows = n;
    H.MA.n_cols = A.n_cols;
    H.MA.rp.resize(n + 1);
    H.MA.col.resize(nz);
    H.MA.val.assign(nz, 0.0);
    H.pair_ptr.resize(static_cast<size_t>(nz) + 1);
    H.pair_p.resize(npairs);
    H.pair_q.resize(npairs);
    check(cudaMemcpyAsync(H.MA.rp.data(), Z_rp, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s), "download");
    check(cudaMemcpyAsync(H.MA.col.data(), Z_col, sizeof(int) * nz, cudaMemcpyDeviceToHost, s), "download");
    check(cudaMemcpyAsync(H.pair_ptr.data(), pp, sizeof(int) * (static_cast<size_t>(nz) + 1), cudaMemcpyDeviceToHost, s),
          "download");
    if (npairs) {
        check(cudaMemcpyAsync(H.pair_p.data(), pair_p, sizeof(int) * npairs, cudaMemcpyDeviceToHost, s), "download");
        check(cudaMemcpyAsync(H.pair_q.data(), pair_q, sizeof(int) * npairs, cudaMemcpyDeviceToHost, s), "download");
    }
    download(RA, H.RA, s);
    check(cudaStreamSynchronize(s), "products");
    check(cudaGetLastError(), "product kernels");
}

void build(const HostCSR &A0, double theta, int max_levels, int max_coarse, unsigned long long seed,
           int split_mode, cudaStream_t s, std::vector<HostLevel> &levels, Pool &pool) {
    const bool second = (split_mode & AMG_SPLIT_SECOND_PASS) != 0;
    const bool rs_blocks = (split_mode & AMG_SPLIT_RS_BLOCKS) != 0;
    if (rs_blocks)
        check(cudaFuncSetAttribute(k_rs_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   rs_smem(kRsMaxBlock, kRsMaxPairs)),
              "block split shared memory");
    DevCSR A;
    A.n_rows = A.n_cols = A0.n_rows;
    A.nnz = A0.nnz();
    A.rp = need<int>(pool, A.n_rows + 1);
    A.col = need<int>(pool, A.nnz);
    A.val = need<double>(pool, A.nnz);
    check(cudaMemcpyAsync(A.rp, A0.rp.data(), sizeof(int) * (A.n_rows + 1), cudaMemcpyHostToDevice, s), "upload");
    check(cudaMemcpyAsync(A.col, A0.col.data(), sizeof(int) * A.nnz, cudaMemcpyHostToDevice, s), "upload");
    check(cudaMemcpyAsync(A.val, A0.val.data(), sizeof(double) * A.nnz, cudaMemcpyHostToDevice, s), "upload");
    std::vector<DevCSR> dA{A}, dP, dR;
    while (static_cast<int>(dA.size()) < max_levels && dA.back().n_rows > max_coarse) {
        const DevCSR L = dA.back();
        const int n = L.n_rows;
        const unsigned long long seed_l = seed + static_cast<unsigned long long>(dA.size() - 1);
        const int g = grid_for(n);
        // strength graph and its transpose
        uint8_t *strong = need<uint8_t>(pool, L.nnz);
        int *S_rp = need<int>(pool, n + 1);
        check(cudaMemsetAsync(S_rp + n, 0, sizeof(int), s), "memset");
        k_strength<<<g, kBlock, 0, s>>>(n, L.rp, L.col, L.val, theta, strong, S_rp); AMG_COUNT();
        const int nS = scan_counts<int>(S_rp, n, pool, s);
        int *S_col = need<int>(pool, nS);
        k_fill_strong<<<g, kBlock, 0, s>>>(n, L.rp, L.col, strong, S_rp, S_col); AMG_COUNT();
        int *T_rp = need<int>(pool, n + 1);
        check(cudaMemsetAsync(T_rp, 0, sizeof(int) * (n + 1), s), "memset");
        k_count_cols<<<g, kBlock, 0, s>>>(n, S_rp, S_col, T_rp); AMG_COUNT();
        scan_counts<int>(T_rp, n, pool, s);
        int *cursor = need<int>(pool, n);
        check(cudaMemcpyAsync(cursor, T_rp, sizeof(int) * n, cudaMemcpyDeviceToDevice, s), "copy");
        int *T_col = need<int>(pool, nS);
        k_scatter_transpose<<<g, kBlock, 0, s>>>(n, S_rp, S_col, nullptr, cursor, T_col, nullptr); AMG_COUNT();
        int8_t *state = need<int8_t>(pool, n);
        int8_t *newc = need<int8_t>(pool, n);
        int *remaining = need<int>(pool, 1);
        // rounds in batches of kBatch between read-backs: a round after the
        // split is complete decides nothing and changes nothing
        constexpr int kBatch = 4;
        if (rs_blocks) {
            // block size from the strong pairs inside the blocks, then the
            // blocks' first passes and the repair of F points left without a
            // strong C point
            int *part = need<int>(pool, static_cast<long long>(kRsSizes) * g);
            int *worst = need<int>(pool, kRsSizes);
            k_rs_pairs<<<g, kBlock, 0, s>>>(n, S_rp, S_col, part); AMG_COUNT();
            k_rs_pairs_max<<<1, kBlock, 0, s>>>(g, part, worst); AMG_COUNT();
            int hw[kRsSizes] = {};
            check(cudaMemcpyAsync(hw, worst, sizeof(hw), cudaMemcpyDeviceToHost, s), "read back");
            check(cudaStreamSynchronize(s), "synchronise");
            int B = 128, max_pairs = kRsMaxPairs;
            for (int k = kRsSizes - 1; k >= 0; --k) {
                if (hw[k] <= kRsMaxPairs) {
                    B = 256 << k;
                    max_pairs = std::max(1, hw[k]);
                    break;
                }
            }
            k_rs_block<<<(n + B - 1) / B, kRsThreads, rs_smem(B, max_pairs), s>>>(n, B, max_pairs, S_rp, S_col, T_rp,
                                                                              T_col, state); AMG_COUNT();
            k_rs_repair_mark<<<g, kBlock, 0, s>>>(n, S_rp, S_col, state, newc); AMG_COUNT();
            k_rs_repair_apply<<<g, kBlock, 0, s>>>(n, newc, state); AMG_COUNT();
            check(cudaGetLastError(), "block split");
        } else {
            double *lam = need<double>(pool, n);
            k_pmis_init<<<g, kBlock, 0, s>>>(n, T_rp, seed_l, lam, state); AMG_COUNT();
            for (int round = 0;; round += kBatch) {
                if (round > n) throw Fail{"PMIS split did not finish"};
                for (int b = 0; b < kBatch; ++b) {
                    check(cudaMemsetAsync(remaining, 0, sizeof(int), s), "memset");
                    k_pmis_select<<<g, kBlock, 0, s>>>(n, S_rp, S_col, T_rp, T_col, lam, state, newc); AMG_COUNT();
                    k_pmis_update<<<g, kBlock, 0, s>>>(n, S_rp, S_col, newc, state, remaining); AMG_COUNT();
                }
                if (read_one(remaining, s) == 0) break;
            }
        }
        if (second) {
            int *v = need<int>(pool, n);
            // batched like the PMIS rounds: once a round finds no violating
            // pair, later rounds find none and promote nothing
            for (int round = 0;; round += kBatch) {
                if (round > n) throw Fail{"second pass did not finish"};
                for (int b = 0; b < kBatch; ++b) {
                    check(cudaMemsetAsync(v, 0, sizeof(int) * n, s), "memset");
                    check(cudaMemsetAsync(remaining, 0, sizeof(int), s), "memset");
                    k_h1_violations<<<g, kBlock, 0, s>>>(n, S_rp, S_col, state, v, remaining); AMG_COUNT();
                    k_h1_promote<<<g, kBlock, 0, s>>>(n, S_rp, S_col, T_rp, T_col, v, seed_l, state); AMG_COUNT();
                }
                if (read_one(remaining, s) == 0) break;
            }
        }
        int *cidx = need<int>(pool, n + 1);
        check(cudaMemsetAsync(cidx + n, 0, sizeof(int), s), "memset");
        k_cflag<<<g, kBlock, 0, s>>>(n, state, cidx); AMG_COUNT();
        const int nc = scan_counts<int>(cidx, n, pool, s);
        if (nc == 0 || static_cast<double>(nc) > 0.9 * n) break;
        // P, R = P^T, A_c = R (A P)
        DevCSR P;
        P.n_rows = n;
        P.n_cols = nc;
        P.rp = need<int>(pool, n + 1);
        check(cudaMemsetAsync(P.rp + n, 0, sizeof(int), s), "memset");
        k_interp_count<<<g, kBlock, 0, s>>>(n, L.rp, L.col, strong, state, P.rp); AMG_COUNT();
        P.nnz = scan_counts<int>(P.rp, n, pool, s);
        P.col = need<int>(pool, P.nnz);
        P.val = need<double>(pool, P.nnz);
        k_interp_fill<<<g, kBlock, 0, s>>>(n, L.rp, L.col, L.val, strong, state, cidx, P.rp, P.col, P.val); AMG_COUNT();
        const DevCSR R = transpose_sorted(P, pool, s);
        const DevCSR AP = spgemm(L, P, pool, s);
        const DevCSR Ac = spgemm(R, AP, pool, s);
        dP.push_back(P);
        dR.push_back(R);
        dA.push_back(Ac);
    }
    // the levels stay in the pool; the host receives their row pointers
    levels.assign(dA.size(), HostLevel{});
    for (size_t l = 0; l < dA.size(); ++l) {
        describe(dA[l], levels[l].A, s);
        if (l + 1 < dA.size()) {
            describe(dP[l], levels[l].P, s);
            describe(dR[l], levels[l].R, s);
        }
    }
    check(cudaStreamSynchronize(s), "setup");
    check(cudaGetLastError(), "setup kernels");
}

}  // namespace

int device_plan_products(std::vector<HostLevel> &levels, const std::vector<char> &which, cudaStream_t s,
                         std::string &err) {
    Pool pool;
    try {
        for (size_t l = 0; l < levels.size() && l < which.size(); ++l)
            if (which[l]) plan_products(levels[l], pool, s);
    } catch (const Fail &f) {
        cudaStreamSynchronize(s);
        err = "device planning: " + f.msg;
        return AMG_ERR_CUDA;
    }
    return AMG_OK;
}

int device_build_hierarchy(const HostCSR &A0, double theta, int max_levels, int max_coarse,
                           unsigned long long seed, int split_mode, cudaStream_t s,
                           std::vector<HostLevel> &levels, std::shared_ptr<void> &keep, std::string &err) {
    auto pool = std::make_shared<Pool>();
    try {
        build(A0, theta, max_levels, max_coarse, seed, split_mode, s, levels, *pool);
    } catch (const Fail &f) {
        cudaStreamSynchronize(s);
        err = "device setup: " + f.msg;
        levels.clear();
        return AMG_ERR_CUDA;
    }
    keep = pool;
    return AMG_OK;
}

}  // namespace amg
