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
// Scheduling: the (pass, block) tasks of a chain are numbered on the host in
// an order where every task comes after the tasks it depends on, each pass
// trailing the previous one by `lag` blocks beyond its dependency front.
// CTA c of the grid (no larger than the CTAs that fit on the GPU at once)
// runs tasks c, c + grid, c + 2 grid, ... in that order, so a task only ever
// waits for lower-numbered tasks, each of which its CTA reaches first: the
// smallest unfinished task always has its inputs, and the chain cannot
// deadlock.  Each task first issues the loads that depend on no other task
// (row bounds, columns and values of its rows, and a_jj for the on-the-fly
// values), then waits for the blocks it gathers from, then gathers.  A task
// publishes its completion with a release store of the launch's epoch in a
// per-(pass, block) flag; a dependent task polls the flags with acquire
// loads.  Every wait is bounded: after kWfMaxPolls polls (or once another
// wait has given up) the CTA records the failure in `err` and carries on,
// so the kernel always ends and the host reports AMG_ERR_DEVICE_FLAG.
// The last CTA to finish advances the epoch, so flags need no clearing
// between launches.
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
constexpr int kWfThreads = 256;
#ifndef AMG_WF_ITER
#define AMG_WF_ITER 2
#endif
#ifndef AMG_WF_LAG_PCT
#define AMG_WF_LAG_PCT 200
#endif
#ifndef AMG_WF_CTAS_PER_SM
#define AMG_WF_CTAS_PER_SM 8
#endif
constexpr int kWfIter = AMG_WF_ITER;       // row-group passes of a CTA per task
// each pass trails the previous one by kWfLagPct % of a grid's worth of
// tasks, so the tasks a task waits for were taken about a grid turnover
// earlier and have usually finished
constexpr int kWfLagPct = AMG_WF_LAG_PCT;
constexpr int kWfCtasPerSM = AMG_WF_CTAS_PER_SM;
#ifndef AMG_WF_SLEEP_NS
#define AMG_WF_SLEEP_NS 32
#endif
#ifndef AMG_WF_FENCE
#define AMG_WF_FENCE 1
#endif
#ifndef AMG_WF_MINB
#define AMG_WF_MINB 1
#endif
constexpr unsigned kWfMaxPolls = 1u << 20; // bounded dependency wait (with back-off: >= ~0.1 s)

template <class T> struct WfArgs {
    int n = 0, nblk = 0, brows = 0, ntask = 0, nphase = 0;
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
    const int4 *task = nullptr;     // ntask descriptors: pass, block, first and last block it reads
    unsigned *flags = nullptr;      // kWfMaxPhases x nblk completion epochs
    unsigned *ctrl = nullptr;       // [1] CTAs finished, [2] epoch
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

// Warp 0 waits until pass `ph` is complete (flag == target) on blocks lo..hi.
__device__ __forceinline__ void wf_wait(const unsigned *f, int lo, int hi, unsigned target, int *err) {
    const int lane = threadIdx.x & 31;
    for (int base = lo; base <= hi; base += 32) {
        const int k = base + lane;
        bool ok = k > hi;
        unsigned polls = 0;
        while (true) {
            if (!ok) ok = ld_acquire_u32(f + k) == target;
            if (__all_sync(0xffffffffu, ok)) break;
            // every lane takes the same decision (the flag read may differ by lane)
            const bool give_up = ++polls > kWfMaxPolls || ld_volatile_i32(err) != 0;
            if (__any_sync(0xffffffffu, give_up)) {
                if (lane == 0) atomicOr(err, 1);
                return;
            }
            if (AMG_WF_SLEEP_NS > 0) __nanosleep(polls < 64 ? AMG_WF_SLEEP_NS : 8 * AMG_WF_SLEEP_NS);
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

// One task: pass `ph` of the chain on the rows of block `blk`, after the
// previous pass has finished on blocks lo..hi.  Each thread takes kWfIter
// rows (row groups of TPR lanes): their matrix loads are issued before the
// wait, their gathers after it, and the stores once every row is summed.
template <class T, int TPR, bool FLY>
__device__ __forceinline__ void wf_task(const WfArgs<T> &A, const int4 d, unsigned target) {
    constexpr int RPB = kWfThreads / TPR;
    const int ph = d.x, blk = d.y;
    const int lane = threadIdx.x % TPR;
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
    const int r0 = blk * A.brows;
    const int r1 = min(A.n, r0 + A.brows);
    WfCoef<T> k{};
    if (qfly)
        k = WfCoef<T>{T(__ldg(A.coef)), T(__ldg(A.coef + 1)), T(__ldg(A.coef + 2)), T(__ldg(A.coef + 3)),
                      T(__ldg(A.coef + 4)), T(__ldg(A.coef + 5))};
    // 1. loads that depend on no other task
    RowBatch<T> rb[kWfIter];
    T dj[kWfIter][4], dii[kWfIter];
#pragma unroll
    for (int it = 0; it < kWfIter; ++it) {
        const int row = r0 + it * RPB + static_cast<int>(threadIdx.x) / TPR;
        const bool live = row < r1;
        row_prefetch<TPR>(rb[it], live, lane, rp, row, col, val);
        dii[it] = T(1);
#pragma unroll
        for (int j = 0; j < 4; ++j) dj[it][j] = T(0);
        if (qfly && live) {
            dii[it] = __ldg(A.diag + row);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (rb[it].base + j * TPR < rb[it].e && rb[it].c[j] != row) dj[it][j] = __ldg(A.diag + rb[it].c[j]);
        }
    }
    // 2. the previous pass on the blocks this one gathers from
    if (ph > 0 && threadIdx.x < 32) wf_wait(A.flags + static_cast<size_t>(ph - 1) * A.nblk, d.z, d.w, target, A.err);
    __syncthreads();
    // 3. gathers and sums of every row, then the stores
    const T *in = A.v[A.in[ph]];
    const T *aux = A.v[A.aux[ph]];
    T *out = A.v[A.out[ph]];
    T acc[kWfIter];
#pragma unroll
    for (int it = 0; it < kWfIter; ++it) {
        const int row = r0 + it * RPB + static_cast<int>(threadIdx.x) / TPR;
        T a = T(0);
        if (row < r1) {
            switch (op) {
                case kWfResid:
                case kWfJac: a = row_dot_pref<TPR>(rb[it], col, val, GatherCG<T>{in}); break;
                case kWfJac12: a = row_dot_pref<TPR>(rb[it], col, val, JacBProd<T>{A.jac, A.b}); break;
                case kWfProlong: a = row_dot_pref<TPR>(rb[it], col, val, Gather<T>{A.e}); break;
                case kWfQApply:
                    if constexpr (FLY) a = row_qfly_pref<TPR>(rb[it], dj[it], row, col, val, A.diag, k, dii[it], GatherCG<T>{in});
                    else a = row_dot_pref<TPR>(rb[it], col, val, GatherCG<T>{in});
                    break;
                case kWfQB:
                    if constexpr (FLY) a = row_qfly_pref<TPR>(rb[it], dj[it], row, col, val, A.diag, k, dii[it], Gather<T>{A.b});
                    else a = row_dot_pref<TPR>(rb[it], col, val, Gather<T>{A.b});
                    break;
                default: break;
            }
        }
        acc[it] = group_sum<TPR>(a);
    }
#pragma unroll
    for (int it = 0; it < kWfIter; ++it) {
        const int row = r0 + it * RPB + static_cast<int>(threadIdx.x) / TPR;
        if (row < r1 && lane == 0) {
            T r;
            switch (op) {
                case kWfResid: r = __ldg(A.b + row) - acc[it]; break;
                case kWfQApply: r = __ldcg(aux + row) + acc[it]; break;
                case kWfQB: r = acc[it]; break;
                case kWfJac: {
                    const T ui = __ldcg(in + row);
                    r = ui + __ldg(A.jac + row) * (__ldg(A.b + row) - acc[it]);
                    break;
                }
                case kWfJac12: {
                    const T jr = __ldg(A.jac + row), br = __ldg(A.b + row);
                    const T u1 = jr * br;
                    r = u1 + jr * (br - acc[it]);
                    break;
                }
                case kWfJacZ: r = __ldg(A.jac + row) * __ldg(A.b + row); break;
                case kWfProlong: r = __ldcg(in + row) + acc[it]; break;
                default: r = T(0); break;
            }
            out[row] = r;
        }
    }
}

template <class T, int TPR, bool FLY>
__global__ void __launch_bounds__(kWfThreads, AMG_WF_MINB) k_wavefront(const WfArgs<T> A) {
    __shared__ unsigned s_target;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) s_target = ld_acquire_u32(A.ctrl + 2) + 1u;
    __syncthreads();
    const unsigned target = s_target;
    for (int t = blockIdx.x; t < A.ntask; t += gridDim.x) {
        const int4 d = __ldg(A.task + t);
        wf_task<T, TPR, FLY>(A, d, target);
        __syncthreads();   // every row of the task is stored
        if (threadIdx.x == 0) {
            if (AMG_WF_FENCE) __threadfence();
            st_release_u32(A.flags + static_cast<size_t>(d.x) * A.nblk + d.y, target);
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(A.ctrl + 1, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            *reinterpret_cast<volatile unsigned *>(A.ctrl + 1) = 0u;
            __threadfence();
            st_release_u32(A.ctrl + 2, target);
        }
    }
}

// Task order of an nphase-pass chain over nblk blocks: block k of pass p is
// placed once pass p - 1 has been placed on blocks 0 .. H_k + lag, where
// H_k = max_{k' <= k} hi_{k'} (so every block it reads from comes first).
// Writes one (pass, block, lo, hi) descriptor per task.  Returns false if
// the order fails its own check (each task after the tasks it waits on).
inline bool wf_build_order(int nblk, const std::vector<int> &lohi, int nphase, int lag, std::vector<int> &desc) {
    desc.clear();
    if (nblk <= 0 || nphase <= 0 || nphase > kWfMaxPhases) return false;
    std::vector<int> H(nblk);
    int m = 0;
    for (int k = 0; k < nblk; ++k) {
        m = std::max(m, lohi[2 * k + 1]);
        H[k] = m;
    }
    std::vector<int> next(nphase, 0);
    std::vector<int> order;
    order.reserve(static_cast<size_t>(nphase) * nblk);
    auto code = [nblk](int p, int k) { return p * nblk + k; };
    while (next[nphase - 1] < nblk) {
        if (next[0] < nblk) order.push_back(code(0, next[0]++));
        for (int p = 1; p < nphase; ++p) {
            while (next[p] < nblk) {
                const int k = next[p];
                const long long need = std::min<long long>(nblk, static_cast<long long>(H[k]) + 1 + lag);
                if (next[p - 1] < need) break;
                order.push_back(code(p, k));
                ++next[p];
            }
        }
    }
    // check: position of every task after those of its dependencies
    std::vector<int> pos(static_cast<size_t>(nphase) * nblk, -1);
    for (size_t t = 0; t < order.size(); ++t) {
        if (pos[order[t]] != -1) return false;
        pos[order[t]] = static_cast<int>(t);
    }
    for (int p = 0; p < nphase; ++p)
        for (int k = 0; k < nblk; ++k) {
            const int tk = pos[code(p, k)];
            if (tk < 0) return false;
            if (p == 0) continue;
            for (int j = lohi[2 * k]; j <= lohi[2 * k + 1]; ++j)
                if (pos[code(p - 1, j)] > tk) return false;
        }
    desc.resize(4 * order.size());
    for (size_t t = 0; t < order.size(); ++t) {
        const int p = order[t] / nblk, k = order[t] % nblk;
        desc[4 * t] = p;
        desc[4 * t + 1] = k;
        desc[4 * t + 2] = lohi[2 * k];
        desc[4 * t + 3] = lohi[2 * k + 1];
    }
    return true;
}

}  // namespace amg
