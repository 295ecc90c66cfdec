// Tensor-core (tcgen05, sm_103a) form of the GCIN aggregation + node linear
// for layers 2..4 (Eq. GCN, App. A.1), for a GCIN width H of 64 or 32
// (App. B.3): BF16 operands, FP32 accumulation in tensor memory.  One CTA
// owns two consecutive statistic tiles of at most 64 nodes each (a graph's
// last tile is ragged; up to 128 nodes = one M = 128 MMA tile):
//   0. the CTA's row bounds and, when they fit, its entries are staged in
//      shared memory with coalesced loads;
//   1. warps aggregate h_i = sum_j w_ij x_j with FP32 sums (training: FP32
//      rows, H / 4 lanes per row; BF16 inference: bfloat16 rows, H / 8 lanes
//      per row, each lane reading its entry's (column, weight) pair) and store
//      h in BF16 into the A tile (128 x H, K-major, canonical no-swizzle
//      core-matrix layout); W^T goes to the B tile (H x H, K-major) in BF16
//      (pre-packed once per inference in BF16 inference);
//   2. one thread issues H / 16 x tcgen05.mma.kind::f16 (M 128, N H, K 16)
//      into an H-column TMEM accumulator and commits to an mbarrier;
//   3. warps 0..3 read their 32 TMEM lanes (rows) with tcgen05.ld, add the
//      bias, and the CTA writes y (FP32, or bfloat16 in BF16 inference) and
//      the two tiles' mean / M2 statistics (FP32).
// The mbarrier wait is bounded; on timeout the kernel raises an error flag,
// waits (bounded) once more, frees its TMEM columns and returns
// (gcin_tc_selftest exercises that path with no_commit).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace amg {

constexpr int kTcRows = 128;                       // MMA M
template <int H> constexpr int tc_a_bytes() { return kTcRows * H * 2; }        // BF16 A tile (16 / 8 KB)
template <int H> constexpr int tc_b_bytes() { return H * H * 2; }              // BF16 B tile (8 / 2 KB)
template <int H> constexpr int tc_y_bytes() { return kTcRows * (H + 1) * 4; }  // FP32 staging of y over the operands
template <int H> constexpr int tc_op_bytes() {
    return (tc_a_bytes<H>() + tc_b_bytes<H>() > tc_y_bytes<H>()) ? tc_a_bytes<H>() + tc_b_bytes<H>() : tc_y_bytes<H>();
}
// the CTA's adjacency entries (column, weight), staged once when they fit
constexpr int kAggStage = 2048;
constexpr bool kInferBF16Acts = true;   // BF16 inference stores the activations in bfloat16
// the staged entries sit after the A and B tiles and, like them, are dead
// once the MMAs are issued, so the y staging may overlay all three
template <int H> constexpr int tc_stage_off() { return tc_a_bytes<H>() + tc_b_bytes<H>(); }
template <int H> constexpr int tc_smem() {
    return (tc_stage_off<H>() + kAggStage * 8 > tc_y_bytes<H>()) ? tc_stage_off<H>() + kAggStage * 8 : tc_y_bytes<H>();
}
// 8-row groups of a K-major tile of H-wide BF16 rows are H / 8 core matrices of 128 B apart
template <int H> constexpr uint32_t tc_sbo() { return static_cast<uint32_t>(H / 8) * 128u; }

// Byte offset of element (row, k) in a K-major, no-swizzle tile of H-wide
// BF16 rows: core matrices of 8 rows x 16 bytes, K-adjacent cores 128 B
// apart (leading-dimension offset), 8-row groups tc_sbo<H>() apart (stride
// offset: 1024 B for H = 64, 512 B for H = 32).
template <int H>
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    return static_cast<uint32_t>((row >> 3) * tc_sbo<H>() + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// tcgen05 shared-memory matrix descriptor for that layout.
template <int H>
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);        // start address
    d |= static_cast<uint64_t>(128u >> 4) << 16;                // leading-dimension byte offset (K)
    d |= static_cast<uint64_t>(tc_sbo<H>() >> 4) << 32;         // stride-dimension byte offset (rows)
    d |= static_cast<uint64_t>(1u) << 46;                       // fixed 0b001
    return d;                                                   // base offset 0, no swizzle
}

// Instruction descriptor: D F32, A BF16, B BF16, both K-major, N = H, M = 128.
template <int H>
constexpr uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(H >> 3) << 17) | ((kTcRows >> 4) << 24);
}

__device__ __forceinline__ bool tc_try_wait(uint32_t mbar) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(mbar), "r"(0u)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool tc_wait_bounded(uint32_t mbar) {
    for (int it = 0; it < (1 << 20); ++it) {
        if (tc_try_wait(mbar)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

// Sum over the entries of a row of w_p x_{col p}, 8 features per lane
// (L = H / 8 lanes per row; FP32 feature rows gathered as two 16-byte loads,
// or bfloat16 rows (BF) as one, widened exactly); otherwise as agg_rows.
template <int H, bool BF>
__device__ __forceinline__ void agg_rows8(int p0, int p1, const int *__restrict__ col, const float *__restrict__ w,
                                          const void *__restrict__ xin, int hl, float (&h)[8]) {
    constexpr int L = H / 8;
#pragma unroll
    for (int f = 0; f < 8; ++f) h[f] = 0.f;
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
        const int cnt = deg - base;
        const int cmax = min(L, maxdeg - base);
        for (int k = 0; k < cmax; k += 4) {
            int c[4];
            float wk[4];
            float v[4][8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                c[j] = __shfl_sync(0xffffffffu, cj, (k + j) & (L - 1), L);
                wk[j] = __shfl_sync(0xffffffffu, wj, (k + j) & (L - 1), L);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool on = k + j < cnt && k + j < cmax;
                if (BF) {
                    const uint4 r = on ? reinterpret_cast<const uint4 *>(xin)[static_cast<size_t>(c[j]) * L + hl]
                                       : make_uint4(0u, 0u, 0u, 0u);
                    const unsigned q[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        v[j][2 * m] = __uint_as_float(q[m] << 16);
                        v[j][2 * m + 1] = __uint_as_float(q[m] & 0xFFFF0000u);
                    }
                } else {
                    const float4 *row = reinterpret_cast<const float4 *>(xin) + (static_cast<size_t>(c[j]) * L + hl) * 2;
                    const float4 a = on ? row[0] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 b = on ? row[1] : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[j][0] = a.x; v[j][1] = a.y; v[j][2] = a.z; v[j][3] = a.w;
                    v[j][4] = b.x; v[j][5] = b.y; v[j][6] = b.z; v[j][7] = b.w;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k + j < cnt && k + j < cmax) {
#pragma unroll
                    for (int f = 0; f < 8; ++f) h[f] = fmaf(wk[j], v[j][f], h[f]);
                }
            }
        }
    }
}

// agg_rows8 for bfloat16 rows with the CTA's entries staged in shared memory
// as (column, weight) pairs: each lane reads the pair of the entry it adds
// (lanes of one row read the same address) instead of receiving it by shuffles.
template <int H>
__device__ __forceinline__ void agg_rows8_staged(int p0, int p1, const int2 *cw, const uint4 *__restrict__ x8,
                                                 int hl, float (&h)[8]) {
    constexpr int L = H / 8;
    // feature pairs (2m, 2m + 1) accumulate with paired FP32 FMAs (each half
    // rounds exactly as fmaf)
    float2 acc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
    const int deg = p1 - p0;
    int maxdeg = deg;
#pragma unroll
    for (int o = L; o < 32; o <<= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xffffffffu, maxdeg, o));
    for (int k = 0; k < maxdeg; k += 4) {
        uint4 r[4];
        float wk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool on = k + j < deg;
            const int2 e = on ? cw[p0 + k + j] : make_int2(0, 0);
            wk[j] = __int_as_float(e.y);
            r[j] = on ? x8[static_cast<size_t>(e.x) * L + hl] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k + j < deg) {
                const unsigned q[4] = {r[j].x, r[j].y, r[j].z, r[j].w};
                const float2 w2 = make_float2(wk[j], wk[j]);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    acc[m] = __ffma2_rn(w2, make_float2(__uint_as_float(q[m] << 16), __uint_as_float(q[m] & 0xFFFF0000u)),
                                        acc[m]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        h[2 * m] = acc[m].x;
        h[2 * m + 1] = acc[m].y;
    }
}

// B tiles of the node linears of layers 2..4 for the bfloat16 inference
// path: round(W)^T in the tile layout the MMA reads (block l - 1 packs layer
// l), so each CTA copies 8 KB instead of converting W.
template <int H>
__global__ void __launch_bounds__(kBlock) k_pack_wtile(const float *__restrict__ W1, const float *__restrict__ W2,
                                                       const float *__restrict__ W3, unsigned char *__restrict__ out) {
    const float *W = blockIdx.x == 0 ? W1 : blockIdx.x == 1 ? W2 : W3;
    unsigned char *dst = out + static_cast<size_t>(blockIdx.x) * tc_b_bytes<H>();
    for (int e = threadIdx.x; e < H * H; e += kBlock) {
        const int k = e / H, n = e % H;
        *reinterpret_cast<__nv_bfloat16 *>(dst + tc_off<H>(n, k)) = __float2bfloat16_rn(W[e]);
    }
}

// XB (inference): x rows are bfloat16 (8 features per lane), the B tile comes
// pre-packed from wt, and no h is kept.
template <int H, bool XB = false>
__global__ void __launch_bounds__(kBlock, 4) k_agg_lin_tc(const int *__restrict__ rp, const int *__restrict__ col,
                                                       const float *__restrict__ w, const void *__restrict__ xin,
                                                       const float *__restrict__ W,
                                                       const unsigned char *__restrict__ wt,
                                                       const float *__restrict__ bias,
                                                       const int *__restrict__ tstart, int NT,
                                                       float *__restrict__ hout, float *__restrict__ y,
                                                       float *__restrict__ tmean, float *__restrict__ tm2,
                                                       int *__restrict__ err, int no_commit) {
    extern __shared__ __align__(128) unsigned char tc_smem[];
    static_assert(H == 64 || H == 32, "GCIN widths with a tensor-core form: 64, 32");
    constexpr int L = H / 4, R = 32 / L;       // lanes per aggregated row, rows per warp
    constexpr uint32_t kCols = H;              // TMEM accumulator columns (a power of two >= 32)
    unsigned char *sA = tc_smem, *sB = tc_smem + tc_a_bytes<H>();
    // y is staged over the A / B tiles once the MMAs that read them have completed
    float(*sY)[H + 1] = reinterpret_cast<float(*)[H + 1]>(tc_smem);
    int *s_col = reinterpret_cast<int *>(tc_smem + tc_stage_off<H>());
    float *s_w = reinterpret_cast<float *>(s_col + kAggStage);
    int2 *s_cw = reinterpret_cast<int2 *>(s_col);   // the same bytes as (column, weight) pairs (XB)
    __shared__ int s_rp[kTcRows + 1];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_ok;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t a_addr = static_cast<uint32_t>(__cvta_generic_to_shared(sA));
    const uint32_t b_addr = static_cast<uint32_t>(__cvta_generic_to_shared(sB));
    const uint32_t mbar = static_cast<uint32_t>(__cvta_generic_to_shared(&s_mbar));
    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&s_taddr));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B = W^T (row n = output feature, k = input feature), BF16
    if (XB) {
        const uint4 *src = reinterpret_cast<const uint4 *>(wt);
        for (int q = threadIdx.x; q < tc_b_bytes<H>() / 16; q += kBlock) reinterpret_cast<uint4 *>(sB)[q] = src[q];
    } else {
        for (int e = threadIdx.x; e < H * H; e += kBlock) {
            const int k = e / H, n = e % H;
            *reinterpret_cast<__nv_bfloat16 *>(sB + tc_off<H>(n, k)) = __float2bfloat16_rn(W[e]);
        }
    }
    // A = h of the (up to) 128 nodes of tiles 2b, 2b + 1, BF16.  The rows are
    // consecutive, so their bounds and (when at most kAggStage) their entries
    // come in with coalesced loads first; the gathers then wait on nothing else.
    const int t0 = 2 * blockIdx.x;
    const int t1 = min(t0 + 2, NT);
    const int a0 = tstart[t0], nn = tstart[t1] - a0;
    for (int k = threadIdx.x; k <= nn; k += kBlock) s_rp[k] = rp[a0 + k];
    __syncthreads();
    const int e0 = s_rp[0], ne = s_rp[nn] - e0;
    const bool staged = ne <= kAggStage;
    if (staged) {
        for (int p = threadIdx.x; p < ne; p += kBlock) {
            if (XB && kInferBF16Acts) {
                s_cw[p] = make_int2(col[e0 + p], __float_as_int(w[e0 + p]));
            } else {
                s_col[p] = col[e0 + p];
                s_w[p] = w[e0 + p];
            }
        }
    }
    __syncthreads();
    const int *cs = staged ? s_col : col;
    const float *ws = staged ? s_w : w;
    const int off = staged ? e0 : 0;
    if (XB) {
        constexpr int L8 = H / 8, R8 = 32 / L8;
        const int grp = lane / L8, hl = lane % L8;
        for (int k0 = R8 * warp; k0 < kTcRows; k0 += R8 * (kBlock / 32)) {
            const int k = k0 + grp;
            const bool live = k < nn;
            const int p0 = live ? s_rp[k] - off : 0, p1 = live ? s_rp[k + 1] - off : 0;
            float hv[8];
            if (kInferBF16Acts && staged)
                agg_rows8_staged<H>(p0, p1, s_cw, reinterpret_cast<const uint4 *>(xin), hl, hv);
            else
                agg_rows8<H, kInferBF16Acts>(p0, p1, cs, ws, xin, hl, hv);   // zero for rows past the tiles
            // features 8 hl .. 8 hl + 7 are one 16-byte core-matrix row
            uint4 pk;
            __nv_bfloat162 t;
            t = __floats2bfloat162_rn(hv[0], hv[1]);
            pk.x = *reinterpret_cast<unsigned *>(&t);
            t = __floats2bfloat162_rn(hv[2], hv[3]);
            pk.y = *reinterpret_cast<unsigned *>(&t);
            t = __floats2bfloat162_rn(hv[4], hv[5]);
            pk.z = *reinterpret_cast<unsigned *>(&t);
            t = __floats2bfloat162_rn(hv[6], hv[7]);
            pk.w = *reinterpret_cast<unsigned *>(&t);
            *reinterpret_cast<uint4 *>(sA + tc_off<H>(k, 8 * hl)) = pk;
        }
    }
    const int grp = lane / L, hl = lane % L;
    const float4 *x4 = reinterpret_cast<const float4 *>(xin);
    for (int k0 = R * warp; !XB && k0 < kTcRows; k0 += R * (kBlock / 32)) {
        const int k = k0 + grp;
        const bool live = k < nn;
        const int i = a0 + (live ? k : 0);
        const int p0 = live ? s_rp[k] - off : 0, p1 = live ? s_rp[k + 1] - off : 0;
        const float4 hv = agg_rows<H>(p0, p1, cs, ws, x4, hl);     // zero for rows past the tiles
        const __nv_bfloat162 lo = __floats2bfloat162_rn(hv.x, hv.y), hi = __floats2bfloat162_rn(hv.z, hv.w);
        if (live && hout) {   // the rounded h the MMA sees (kept for the backward)
            const float2 rl = __bfloat1622float2(lo), rh = __bfloat1622float2(hi);
            reinterpret_cast<float4 *>(hout)[static_cast<size_t>(i) * L + hl] = make_float4(rl.x, rl.y, rh.x, rh.y);
        }
        // features 4 hl .. 4 hl + 3 are contiguous within one core matrix row
        *reinterpret_cast<__nv_bfloat162 *>(sA + tc_off<H>(k, 4 * hl)) = lo;
        *reinterpret_cast<__nv_bfloat162 *>(sA + tc_off<H>(k, 4 * hl + 2)) = hi;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    // no_commit (self-test only) issues nothing, so the bounded wait below runs out
    if (threadIdx.x == 0 && !no_commit) {
        for (int ks = 0; ks < H / 16; ++ks) {
            const uint64_t ad = tc_desc<H>(a_addr + ks * 256), bd = tc_desc<H>(b_addr + ks * 256);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(taddr), "l"(ad), "l"(bd), "r"(tc_idesc<H>()), "r"(static_cast<uint32_t>(ks))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
    }
    const bool ok = tc_wait_bounded(mbar);
    if (threadIdx.x == 0) s_ok = ok ? 1 : 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool all_ok = s_ok != 0;
    if (all_ok && warp < 4) {
        // warp w reads TMEM lanes 32 w .. 32 w + 31 (its rows), 16 columns at a time
        const int row = 32 * warp + lane;
#pragma unroll
        for (int q16 = 0; q16 < H / 16; ++q16) {
            uint32_t r[16];
            const uint32_t ta = taddr + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(16 * q16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int f = 0; f < 16; ++f) sY[row][16 * q16 + f] = __uint_as_float(r[f]) + bias[16 * q16 + f];
        }
    }
    if (!all_ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        tc_wait_bounded(mbar);          // let an in-flight MMA drain before the columns are freed
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kCols) : "memory");
    if (!all_ok) return;
    // y (coalesced; bfloat16 in BF16 inference) and the statistics of the
    // two 64-node tiles (from the FP32 values)
    for (int e = threadIdx.x; e < nn * (H / 4); e += kBlock) {
        const int k = e / (H / 4), f = 4 * (e % (H / 4));
        const size_t o = static_cast<size_t>(a0 + k) * H + f;
        if (XB && kInferBF16Acts) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(sY[k][f], sY[k][f + 1]);
            __nv_bfloat162 hi = __floats2bfloat162_rn(sY[k][f + 2], sY[k][f + 3]);
            reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(y) + o)[0] =
                make_uint2(*reinterpret_cast<unsigned *>(&lo), *reinterpret_cast<unsigned *>(&hi));
        } else {
            reinterpret_cast<float4 *>(y)[o / 4] = make_float4(sY[k][f], sY[k][f + 1], sY[k][f + 2], sY[k][f + 3]);
        }
    }
    // the first tile may be a graph's ragged last tile: split at tstart[t0 + 1]
    const int n0 = tstart[t0 + 1] - a0;
    tile_stats<H>(sY, n0, tmean + static_cast<size_t>(t0) * H, tm2 + static_cast<size_t>(t0) * H);
    if (t0 + 1 < t1) {
        __syncthreads();
        tile_stats<H>(sY + n0, nn - n0, tmean + static_cast<size_t>(t0 + 1) * H,
                      tm2 + static_cast<size_t>(t0 + 1) * H);
    }
}

}  // namespace amg

namespace amg {

// Tensor-core form of the node-linear backward of layers 2..4 when the
// forward ran on tcgen05 with BF16 operands (App. A.1; the backward of
// Sec. 3.3 differentiates that rounded forward): per CTA two statistic tiles
// (at most 128 nodes),
//   1. dy of every node from the instance-norm backward (FP32, staged in
//      shared memory; the bias gradient is its fixed-order column sum), then
//      BF16 copies of dy into A1 (nodes x H, K = output feature) and into B2
//      (H x 128, K = node: dy transposed), the forward's BF16 h into A2
//      (rows = input feature, K = node) and round(W) into B1 (rows = input
//      feature, K = output feature), all K-major, no swizzle;
//   2. one thread issues D1 = A1 B1^T (dh = dy W^T, 128 x H) and
//      D2 = A2 B2^T (sum_i h_i^T dy_i, rows < H used) into 2H TMEM columns;
//   3. warps 0..3 read both back; dh is written per node, the weight gradient
//      as the first tile's partial (the second tile's partial is zero).
// Nodes past the tiles are zero in A2 / B2, so they add nothing to D2.  The
// mbarrier wait is bounded as in the forward: on timeout the error flag is
// raised, the MMAs are drained (bounded) and the TMEM columns freed.
template <int H> constexpr int tcb_a1_bytes() { return kTcRows * H * 2; }
template <int H> constexpr int tcb_b1_bytes() { return H * H * 2; }
constexpr int tcb_a2_bytes() { return kTcRows * kTcRows * 2; }
template <int H> constexpr int tcb_b2_bytes() { return H * kTcRows * 2; }
template <int H> constexpr int tcb_d_bytes() { return kTcRows * (H + 1) * 4; }
template <int H> constexpr int tcb_smem() {
    return tcb_a1_bytes<H>() + tcb_b1_bytes<H>() + tcb_a2_bytes() + tcb_b2_bytes<H>() + tcb_d_bytes<H>();
}

template <int H>
__global__ void __launch_bounds__(kBlock, 2) k_bwd_lin_tc(const int *__restrict__ tstart, const int *__restrict__ tgraph,
                                                          const int *__restrict__ gptr, int NT,
                                                          const float *__restrict__ y, const float *__restrict__ mu,
                                                          const float *__restrict__ rstd,
                                                          const float *__restrict__ gamma,
                                                          const double *__restrict__ gS1,
                                                          const double *__restrict__ gS2,
                                                          const float *__restrict__ W, const float *__restrict__ hin,
                                                          const float *__restrict__ dyn, float *__restrict__ dh,
                                                          float *__restrict__ dWt, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char tcb_smem_buf[];
    static_assert(H == 64 || H == 32, "GCIN widths with a tensor-core form: 64, 32");
    constexpr uint32_t kCols = (2 * H < 32) ? 32 : 2 * H;   // D1 at column 0, D2 at column H
    unsigned char *sA1 = tcb_smem_buf, *sB1 = sA1 + tcb_a1_bytes<H>();
    unsigned char *sA2 = sB1 + tcb_b1_bytes<H>(), *sB2 = sA2 + tcb_a2_bytes();
    float(*sD)[H + 1] = reinterpret_cast<float(*)[H + 1]>(sB2 + tcb_b2_bytes<H>());
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_ok;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t a1 = static_cast<uint32_t>(__cvta_generic_to_shared(sA1));
    const uint32_t b1 = static_cast<uint32_t>(__cvta_generic_to_shared(sB1));
    const uint32_t a2 = static_cast<uint32_t>(__cvta_generic_to_shared(sA2));
    const uint32_t b2 = static_cast<uint32_t>(__cvta_generic_to_shared(sB2));
    const uint32_t mbar = static_cast<uint32_t>(__cvta_generic_to_shared(&s_mbar));
    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&s_taddr));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int t0 = 2 * blockIdx.x;
    const int t1 = min(t0 + 2, NT);
    const int a0 = tstart[t0], nn = tstart[t1] - a0;
    const int n0 = tstart[t0 + 1] - a0;   // nodes of the first tile
    // B1 = round(W): row = input feature k, K = output feature n (W is [in][out])
    for (int e = threadIdx.x; e < H * H; e += kBlock) {
        const int k = e / H, n = e % H;
        *reinterpret_cast<__nv_bfloat16 *>(sB1 + tc_off<H>(k, n)) = __float2bfloat16_rn(W[e]);
    }
    // 1. dy (instance-norm backward) of every node, FP32 in shared memory
    for (int e = threadIdx.x; e < kTcRows * H; e += kBlock) {
        const int k = e / H, f = e % H;
        float dy = 0.f;
        if (k < nn) {
            const int g = tgraph[k < n0 ? t0 : t0 + 1];
            const float inv_n = 1.f / static_cast<float>(gptr[g + 1] - gptr[g]);
            const float ga = gamma[f], r = rstd[g * H + f];
            const float c1 = ga * static_cast<float>(gS1[g * H + f]) * inv_n;
            const float c2 = ga * static_cast<float>(gS2[g * H + f]) * inv_n;
            const size_t i = static_cast<size_t>(a0 + k) * H + f;
            const float yh = (y[i] - mu[g * H + f]) * r;
            dy = r * (ga * dyn[i] - c1 - yh * c2);
        }
        sD[k][f] = dy;
    }
    __syncthreads();
    // BF16 operands: A1 (dy, node rows), B2 (dy transposed), A2 (h transposed)
    for (int e = threadIdx.x; e < kTcRows * H; e += kBlock) {
        const int k = e / H, f = e % H;
        const __nv_bfloat16 d = __float2bfloat16_rn(sD[k][f]);
        *reinterpret_cast<__nv_bfloat16 *>(sA1 + tc_off<H>(k, f)) = d;
        *reinterpret_cast<__nv_bfloat16 *>(sB2 + tc_off<kTcRows>(f, k)) = d;
        const float hv = k < nn ? hin[static_cast<size_t>(a0 + k) * H + f] : 0.f;   // already BF16 values
        *reinterpret_cast<__nv_bfloat16 *>(sA2 + tc_off<kTcRows>(f, k)) = __float2bfloat16_rn(hv);
    }
    // rows H..127 of A2 only produce rows of D2 that are never read
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    if (threadIdx.x == 0) {
        for (int ks = 0; ks < H / 16; ++ks) {
            const uint64_t ad = tc_desc<H>(a1 + ks * 256), bd = tc_desc<H>(b1 + ks * 256);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(taddr), "l"(ad), "l"(bd), "r"(tc_idesc<H>()), "r"(static_cast<uint32_t>(ks))
                         : "memory");
        }
        for (int ks = 0; ks < kTcRows / 16; ++ks) {
            const uint64_t ad = tc_desc<kTcRows>(a2 + ks * 256), bd = tc_desc<kTcRows>(b2 + ks * 256);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(taddr + static_cast<uint32_t>(H)), "l"(ad), "l"(bd), "r"(tc_idesc<H>()),
                         "r"(static_cast<uint32_t>(ks))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
    }
    // the bias gradient (FP32, fixed node order) while the MMAs run
    float *out0 = dWt + static_cast<size_t>(t0) * (H * H + H);
    if (threadIdx.x < H) {
        float acc = 0.f;
        for (int k = 0; k < nn; ++k) acc += sD[k][threadIdx.x];
        out0[H * H + threadIdx.x] = acc;
        if (t0 + 1 < t1) dWt[static_cast<size_t>(t0 + 1) * (H * H + H) + H * H + threadIdx.x] = 0.f;
    }
    const bool ok = tc_wait_bounded(mbar);
    if (threadIdx.x == 0) s_ok = ok ? 1 : 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool all_ok = s_ok != 0;
    if (all_ok && warp < 4) {
        const int row = 32 * warp + lane;
#pragma unroll
        for (int part = 0; part < 2; ++part) {          // part 0: D1 (dh), part 1: D2 (weight gradient)
#pragma unroll
            for (int half = 0; half < H / 32; ++half) {
                uint32_t r[32];
                const uint32_t ta = taddr + (static_cast<uint32_t>(32 * warp) << 16) +
                                    static_cast<uint32_t>(part * H + 32 * half);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                      "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                      "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(ta)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (part == 0) {
                    if (row < nn) {
#pragma unroll
                        for (int f = 0; f < 32; ++f)
                            dh[static_cast<size_t>(a0 + row) * H + 32 * half + f] = __uint_as_float(r[f]);
                    }
                } else if (row < H) {
#pragma unroll
                    for (int f = 0; f < 32; ++f) out0[row * H + 32 * half + f] = __uint_as_float(r[f]);
                }
            }
        }
    }
    if (!all_ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        tc_wait_bounded(mbar);
    }
    // the second tile's weight partial is zero (its nodes are in the first's sum)
    if (t0 + 1 < t1)
        for (int e = threadIdx.x; e < H * H; e += kBlock) dWt[static_cast<size_t>(t0 + 1) * (H * H + H) + e] = 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kCols) : "memory");
}

}  // namespace amg
