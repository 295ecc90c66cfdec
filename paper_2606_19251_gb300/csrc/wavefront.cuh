// Wavefront smoothing chains on HBM-sized levels (Sec. 2.2, 2.3, 3.1).
//
// One smoothing phase of the V-cycle on a large level is a short chain of
// row-local passes over the pattern of A: for the pseudo-inverse smoother
// (Sec. 3.1) u1 = Q^-1 b, r1 = b - A u1, u2 = u1 + Q^-1 r1, r = b - A u2
// (pre-smoothing from zero and the residual for restriction), or
// u1 = u + P e, r1 = b - A u1, u2 = u1 + Q^-1 r1, r2 = ..., u3 = ...
// (prolongation-correction and post-smoothing); relaxed Jacobi (Sec. 2.3)
// gives the same chains with one pass per sweep.  Run as separate kernels,
// every pass streams A from HBM again.  Here one persistent kernel runs the
// whole chain over row blocks: pass p of block k starts as soon as pass
// p - 1 has finished on every block holding a column of block k's rows, so
// while later passes trail the first by a bounded distance, the entries the
// first pass fetched from HBM are still in the 129 MB L2 when the later
// passes read them.  The pseudo-inverse values are evaluated on the fly
// from a_ij, a_ii, a_jj, s and the level's coefficients (Sec. 3.1), so a
// pass of Q^-1 reads no stored values.
//
// Scheduling: a task is one warp's rows (32 / TPR rows) of one pass.  Tasks
// are numbered round by round: round r holds block r of pass 0, block r - L
// of pass 1, ..., block r - (P - 1) L of pass P - 1, with the lag L (in
// blocks) larger than the distance from a block to the last block its
// columns reach.  So a task only ever waits for lower-numbered tasks.  Warp
// w of the grid (no larger than the warps that fit on the GPU at once) runs
// tasks w, w + W, w + 2 W, ... in that order, so the smallest unfinished task
// always has its inputs and the chain cannot deadlock; with L x P about the
// number of warps, the tasks a task waits for were started a whole grid of
// tasks earlier.  Completion is counted per (pass, group of kWfGroup
// blocks): a finished task adds one to its group's counter with a release
// fence; a dependent task polls the counters of the groups its columns fall
// in with acquire loads until they reach launch number x tasks in the group
// (counters only grow, one set per chain length, so nothing is cleared
// between launches).  Every wait is bounded: after kWfMaxPolls polls (or
// once another wait has given up) the warp records the failure in `err` and
// carries on, so the kernel always ends and the host reports
// AMG_ERR_DEVICE_FLAG.  The last warp to finish advances the launch number.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace amg {

enum WfOp : int {
    kWfResid = 0,    // out = b - A in                    (gathers in)
    kWfQApply = 1,   // out = aux + Q^-1 in               (gathers in; aux on the own rows)
    kWfQB = 2,       // out = Q^-1 b                      (first pseudo-inverse sweep from zero)
    kWfJac = 3,      // out = in + j (b - A in)           (relaxed Jacobi sweep, j = omega / a_ii)
    kWfJac12 = 4,    // out = j b + j (b - A (j b))       (two Jacobi sweeps from zero)
    kWfJacZ = 5,     // out = j b                         (one Jacobi sweep from zero; row-local)
    kWfProlong = 6,  // out = in + P e                    (prolongation-correction; e complete)
};

constexpr int kWfMaxPhases = 8;
constexpr int kWfBufs = 8;                 // level-owned chain buffers
constexpr int kWfThreads = 256;            // 8 warps per CTA, each an independent worker
constexpr int kWfGroup = 16;               // blocks (warp tasks) per completion counter
#ifndef AMG_WF_LAG_PCT
#define AMG_WF_LAG_PCT 100
#endif
#ifndef AMG_WF_CTAS_PER_SM
#define AMG_WF_CTAS_PER_SM 8
#endif
// the passes trail each other by this percentage of a grid of warps' tasks
constexpr int kWfLagPct = AMG_WF_LAG_PCT;
constexpr int kWfCtasPerSM = AMG_WF_CTAS_PER_SM;
constexpr unsigned kWfMaxPolls = 1u << 20; // bounded dependency wait (with back-off: >= ~0.1 s)

template <class T> struct WfArgs {
    int n = 0, nblk = 0, rpt = 0, nphase = 0, lag = 0, ngroup = 0;
    int op[kWfMaxPhases] = {}, in[kWfMaxPhases] = {}, aux[kWfMaxPhases] = {}, out[kWfMaxPhases] = {};
    const int *rp = nullptr, *col = nullptr;
    const T *a = nullptr;
    const T *diag = nullptr;        // a_ii (pseudo-inverse values on the fly)
    const T *q = nullptr;           // stored pseudo-inverse values on A's pattern
    const float *coef = nullptr;    // d0 d1 d2 o1 o2 1/s of this level (on the fly)
    const T *jac = nullptr;         // omega / a_ii
    const int *prp = nullptr, *pcol = nullptr;
    const T *pv = nullptr, *e = nullptr;   // prolongation P (n x n_c) and the coarse correction
    const T *b = nullptr;
    T *v[kWfBufs + 2] = {};         // chain buffers (n each), then two caller vectors
    const int2 *lohi = nullptr;     // per block: first and last group its rows' columns fall in
    unsigned *count = nullptr;      // nphase x ngroup completed-task counters of this chain length
    unsigned *ctrl = nullptr;       // [1] warps finished, [2] launch number of this chain length
    int *err = nullptr;             // set when a dependency wait gave up
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Gathers of vectors written earlier in the same launch go to L2 (ld.cg), so
// no copy an SM's L1 kept from before the producer's write can be read.
template <class T> struct GatherCG {
    const T *x;
    __device__ __forceinline__ T operator()(int j) const { return __ldcg(x + j); }
};

template <class T> struct JacBProd {   // gathered j_j b_j
    const T *jac, *b;
    __device__ __forceinline__ T operator()(int j) const { return __ldg(jac + j) * __ldg(b + j); }
};

// The warp waits until every task of the previous pass in groups lo..hi is
// done: counter >= launch number x tasks in the group.
__device__ __forceinline__ void wf_wait(const unsigned *cnt, int lo, int hi, int nblk, unsigned target, int *err) {
    const int lane = threadIdx.x & 31;
    for (int base = lo; base <= hi; base += 32) {
        const int g = base + lane;
        const bool mine = g <= hi;
        const unsigned need = mine ? target * static_cast<unsigned>(min(kWfGroup, nblk - g * kWfGroup)) : 0u;
        bool ok = !mine;
        unsigned polls = 0;
        while (true) {
            if (!ok) ok = ld_acquire_u32(cnt + g) >= need;
            if (__all_sync(0xffffffffu, ok)) break;
            // every lane takes the same decision (the flag read may differ by lane)
            const bool give_up = ++polls > kWfMaxPolls || ld_volatile_i32(err) != 0;
            if (__any_sync(0xffffffffu, give_up)) {
                if (lane == 0) atomicOr(err, 1);
                return;
            }
            if (polls > 8) __nanosleep(polls < 64 ? 32 : 256);
        }
    }
}

__device__ __forceinline__ float wf_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double wf_div(double a, double b) { return a / b; }

// The level's smoother coefficients (d0, d1, d2, o1, o2) and 1/s.
template <class T> struct WfCoef {
    T d0, d1, d2, o1, o2, inv_s;
};

// Row i of Q^-1 x with the values evaluated from A (Sec. 3.1):
// q_ii = (d0 + d1 x + d2 x^2) / a_ii with x = a_ii / s,
// q_ij = (o1 x + o2 x^2) / (a_ii + a_jj) with x = a_ij / s.
// The first batch of the row's entries and their a_jj come prefetched.
template <class T> __device__ __forceinline__ T qval(const WfCoef<T> &k, int row, int c, T a, T dii, T djj) {
    const T s = a * k.inv_s;
    return (c == row) ? wf_div(k.d0 + (k.d1 + k.d2 * s) * s, dii) : wf_div((k.o1 + k.o2 * s) * s, dii + djj);
}

template <int TPR, class T, class X>
__device__ __forceinline__ T row_qfly_pref(const RowBatch<T> &rb, const T (&dj)[4], int row, const int *__restrict__ col,
                                           const T *__restrict__ a, const T *__restrict__ diag, const WfCoef<T> &k,
                                           T dii, const X &xg) {
    T acc = T(0);
    if (rb.base >= rb.e) return acc;
    T x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (rb.base + j * TPR < rb.e) ? xg(rb.c[j]) : T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (rb.base + j * TPR < rb.e) acc += qval(k, row, rb.c[j], rb.v[j], dii, dj[j]) * x[j];
    for (int base = rb.base + 4 * TPR; base < rb.e; base += 4 * TPR) {
        int c[4];
        T v[4], d[4], y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = base + j * TPR;
            c[j] = p < rb.e ? __ldg(col + p) : row;
            v[j] = p < rb.e ? __ldg(a + p) : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool live = base + j * TPR < rb.e;
            y[j] = live ? xg(c[j]) : T(0);
            d[j] = (live && c[j] != row) ? __ldg(diag + c[j]) : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (base + j * TPR < rb.e) acc += qval(k, row, c[j], v[j], dii, d[j]) * y[j];
    }
    return acc;
}

// One task: pass `ph` on the rows of block `blk` (one warp, 32 / TPR rows):
// the loads that depend on no other task (row bounds, the first batch of
// columns and values, a_jj for the on-the-fly values), then the wait for the
// previous pass on the groups the block's columns fall in, then the gathers,
// the sums and the stores.
template <class T, int TPR, bool FLY>
__device__ __forceinline__ void wf_task(const WfArgs<T> &A, int ph, int blk, unsigned target) {
    const int lane = threadIdx.x & 31;
    const int sub = lane % TPR;
    const int op = A.op[ph];
    const bool qpass = (op == kWfQApply || op == kWfQB);
    const bool qfly = FLY && qpass;
    const int *rp = A.rp, *col = A.col;
    const T *val = (qpass && !FLY) ? A.q : A.a;
    if (op == kWfProlong) {
        rp = A.prp;
        col = A.pcol;
        val = A.pv;
    }
    const int row = blk * A.rpt + lane / TPR;
    const bool live = row < A.n;
    const int2 lh = __ldg(A.lohi + blk);
    RowBatch<T> rb;
    row_prefetch<TPR>(rb, live, sub, rp, row, col, val);
    T dj[4] = {T(0), T(0), T(0), T(0)};
    T dii = T(1);
    WfCoef<T> k{};
    if (qfly) {
        k = WfCoef<T>{T(__ldg(A.coef)), T(__ldg(A.coef + 1)), T(__ldg(A.coef + 2)), T(__ldg(A.coef + 3)),
                      T(__ldg(A.coef + 4)), T(__ldg(A.coef + 5))};
        if (live) {
            dii = __ldg(A.diag + row);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (rb.base + j * TPR < rb.e && rb.c[j] != row) dj[j] = __ldg(A.diag + rb.c[j]);
        }
    }
    if (ph > 0) wf_wait(A.count + static_cast<size_t>(ph - 1) * A.ngroup, lh.x, lh.y, A.nblk, target, A.err);
    const T *in = A.v[A.in[ph]];
    const T *aux = A.v[A.aux[ph]];
    T *out = A.v[A.out[ph]];
    T acc = T(0);
    if (live) {
        switch (op) {
            case kWfResid:
            case kWfJac: acc = row_dot_pref<TPR>(rb, col, val, GatherCG<T>{in}); break;
            case kWfJac12: acc = row_dot_pref<TPR>(rb, col, val, JacBProd<T>{A.jac, A.b}); break;
            case kWfProlong: acc = row_dot_pref<TPR>(rb, col, val, Gather<T>{A.e}); break;
            case kWfQApply:
                if constexpr (FLY) acc = row_qfly_pref<TPR>(rb, dj, row, col, val, A.diag, k, dii, GatherCG<T>{in});
                else acc = row_dot_pref<TPR>(rb, col, val, GatherCG<T>{in});
                break;
            case kWfQB:
                if constexpr (FLY) acc = row_qfly_pref<TPR>(rb, dj, row, col, val, A.diag, k, dii, Gather<T>{A.b});
                else acc = row_dot_pref<TPR>(rb, col, val, Gather<T>{A.b});
                break;
            default: break;
        }
    }
    acc = group_sum<TPR>(acc);
    if (live && sub == 0) {
        T r;
        switch (op) {
            case kWfResid: r = __ldg(A.b + row) - acc; break;
            case kWfQApply: r = __ldcg(aux + row) + acc; break;
            case kWfQB: r = acc; break;
            case kWfJac: {
                const T ui = __ldcg(in + row);
                r = ui + __ldg(A.jac + row) * (__ldg(A.b + row) - acc);
                break;
            }
            case kWfJac12: {
                const T jr = __ldg(A.jac + row), br = __ldg(A.b + row);
                const T u1 = jr * br;
                r = u1 + jr * (br - acc);
                break;
            }
            case kWfJacZ: r = __ldg(A.jac + row) * __ldg(A.b + row); break;
            case kWfProlong: r = __ldcg(in + row) + acc; break;
            default: r = T(0); break;
        }
        out[row] = r;
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        atomicAdd(A.count + static_cast<size_t>(ph) * A.ngroup + blk / kWfGroup, 1u);
    }
}

template <class T, int TPR, bool FLY>
__global__ void __launch_bounds__(kWfThreads) k_wavefront(const WfArgs<T> A) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int nw = static_cast<int>(gridDim.x) * (kWfThreads / 32);
    const int w = static_cast<int>(blockIdx.x) * (kWfThreads / 32) + static_cast<int>(threadIdx.x >> 5);
    unsigned target = 0;
    if (lane == 0) target = ld_acquire_u32(A.ctrl + 2) + 1u;
    target = __shfl_sync(0xffffffffu, target, 0);
    const int P = A.nphase;
    const long long ntick = static_cast<long long>(A.nblk + (P - 1) * A.lag) * P;
    for (long long t = w; t < ntick; t += nw) {
        const int ph = static_cast<int>(t % P);
        const long long blk = t / P - static_cast<long long>(ph) * A.lag;
        if (blk < 0 || blk >= A.nblk) continue;   // warp-uniform: the pipeline's fill and drain
        wf_task<T, TPR, FLY>(A, ph, static_cast<int>(blk), target);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (lane == 0) {
        __threadfence();
        const unsigned done = atomicAdd(A.ctrl + 1, 1u);
        if (done == static_cast<unsigned>(nw) - 1u) {
            __threadfence();
            *reinterpret_cast<volatile unsigned *>(A.ctrl + 1) = 0u;
            __threadfence();
            st_release_u32(A.ctrl + 2, target);
        }
    }
}

// The group range of each block's columns (own group included) and the
// largest distance, in blocks, from a block to the last block its columns
// reach.
inline int wf_block_ranges(int n, const int *rp, const int *col, int rpt, std::vector<int> &lohi) {
    const int nblk = (n + rpt - 1) / rpt;
    lohi.assign(2 * static_cast<size_t>(nblk), 0);
    int reach = 0;
    for (int k = 0; k < nblk; ++k) {
        int lo = k, hi = k;
        const int r1 = std::min(n, (k + 1) * rpt);
        for (int p = rp[k * rpt]; p < rp[r1]; ++p) {
            const int cb = col[p] / rpt;
            lo = std::min(lo, cb);
            hi = std::max(hi, cb);
        }
        reach = std::max(reach, hi - k);
        lohi[2 * k] = lo / kWfGroup;
        lohi[2 * k + 1] = hi / kWfGroup;
    }
    return reach;
}

}  // namespace amg
