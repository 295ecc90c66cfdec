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
// CTAs take task numbers from a global counter, so a task only ever waits
// for tasks numbered before it, which CTAs that are already running hold:
// the chain cannot deadlock whatever the number of resident CTAs.  A task
// publishes its completion with a release store of the launch's epoch in a
// per-(pass, block) flag; a dependent task polls the flags with acquire
// loads.  Every wait is bounded: after kWfMaxPolls polls (or once another
// wait has given up) the CTA records the failure in `err` and carries on,
// so the kernel always ends and the host reports AMG_ERR_DEVICE_FLAG.
// The last CTA to finish resets the task counter and advances the epoch,
// so flags need no clearing between launches.
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
#define AMG_WF_LAG_PCT 100
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
#ifndef AMG_WF_STATIC
#define AMG_WF_STATIC 0
#endif
#ifndef AMG_WF_SLEEP_NS
#define AMG_WF_SLEEP_NS 32
#endif
#ifndef AMG_WF_FENCE
#define AMG_WF_FENCE 1
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
    const int *lohi = nullptr;      // first and last block holding a column of block k's rows
    const int *order = nullptr;     // ntask codes: pass << 24 | block
    unsigned *flags = nullptr;      // kWfMaxPhases x nblk completion epochs
    unsigned *ctrl = nullptr;       // [0] next task number, [1] CTAs finished, [2] epoch
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
template <int TPR, class T, class X>
__device__ __forceinline__ T row_qfly(int lane, int row, int p0, int e, const int *__restrict__ col,
                                      const T *__restrict__ a, const T *__restrict__ diag, const WfCoef<T> &k,
                                      T dii, const X &xg) {
    T acc = T(0);
    for (int base = p0 + lane; base < e; base += 4 * TPR) {
        int c[4];
        T v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = base + j * TPR;
            c[j] = p < e ? __ldg(col + p) : row;
            v[j] = p < e ? __ldg(a + p) : T(0);
        }
        T x[4], dj[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool live = base + j * TPR < e;
            x[j] = live ? xg(c[j]) : T(0);
            dj[j] = (live && c[j] != row) ? __ldg(diag + c[j]) : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (base + j * TPR < e) {
                const T s = v[j] * k.inv_s;
                const T q = (c[j] == row) ? wf_div(k.d0 + (k.d1 + k.d2 * s) * s, dii)
                                          : wf_div((k.o1 + k.o2 * s) * s, dii + dj[j]);
                acc += q * x[j];
            }
        }
    }
    return acc;
}

template <class T, int TPR, bool FLY>
__device__ __forceinline__ void wf_run(const WfArgs<T> &A, int ph, int blk) {
    constexpr int RPB = kWfThreads / TPR;
    const int lane = threadIdx.x % TPR;
    const int op = A.op[ph];
    const T *in = A.v[A.in[ph]];
    const T *aux = A.v[A.aux[ph]];
    T *out = A.v[A.out[ph]];
    const int r0 = blk * A.brows;
    const int r1 = min(A.n, r0 + A.brows);
    WfCoef<T> k{};
    if constexpr (FLY) {
        if (op == kWfQApply || op == kWfQB)
            k = WfCoef<T>{T(__ldg(A.coef)), T(__ldg(A.coef + 1)), T(__ldg(A.coef + 2)), T(__ldg(A.coef + 3)),
                          T(__ldg(A.coef + 4)), T(__ldg(A.coef + 5))};
    }
    for (int base = r0; base < r1; base += RPB) {
        const int row = base + threadIdx.x / TPR;
        const bool live = row < r1;
        T acc = T(0);
        if (live) {
            if (op == kWfProlong) {
                acc = row_dot<TPR>(lane, __ldg(A.prp + row), __ldg(A.prp + row + 1), A.pcol, A.pv, Gather<T>{A.e});
            } else {
                const int p0 = __ldg(A.rp + row), pe = __ldg(A.rp + row + 1);
                switch (op) {
                    case kWfResid:
                    case kWfJac:
                        acc = row_dot<TPR>(lane, p0, pe, A.col, A.a, GatherCG<T>{in});
                        break;
                    case kWfJac12:
                        acc = row_dot<TPR>(lane, p0, pe, A.col, A.a, JacBProd<T>{A.jac, A.b});
                        break;
                    case kWfQApply:
                        if constexpr (FLY) acc = row_qfly<TPR>(lane, row, p0, pe, A.col, A.a, A.diag, k,
                                                               __ldg(A.diag + row), GatherCG<T>{in});
                        else acc = row_dot<TPR>(lane, p0, pe, A.col, A.q, GatherCG<T>{in});
                        break;
                    case kWfQB:
                        if constexpr (FLY) acc = row_qfly<TPR>(lane, row, p0, pe, A.col, A.a, A.diag, k,
                                                               __ldg(A.diag + row), Gather<T>{A.b});
                        else acc = row_dot<TPR>(lane, p0, pe, A.col, A.q, Gather<T>{A.b});
                        break;
                    default:
                        break;
                }
            }
        }
        acc = group_sum<TPR>(acc);
        if (live && lane == 0) {
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
    }
}

template <class T, int TPR, bool FLY>
__global__ void __launch_bounds__(kWfThreads) k_wavefront(const WfArgs<T> A) {
    __shared__ int s_next;
    __shared__ unsigned s_target;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
        s_target = ld_acquire_u32(A.ctrl + 2) + 1u;
        s_next = AMG_WF_STATIC ? static_cast<int>(blockIdx.x) : atomicAdd(reinterpret_cast<int *>(A.ctrl), 1);
    }
    __syncthreads();
    const unsigned target = s_target;
    int t = s_next;
    while (t < A.ntask) {
        __syncthreads();   // every thread has read s_next
        if (threadIdx.x == 0)   // the next task, early
            s_next = AMG_WF_STATIC ? t + static_cast<int>(gridDim.x) : atomicAdd(reinterpret_cast<int *>(A.ctrl), 1);
        const int code = __ldg(A.order + t);
        const int ph = code >> 24, blk = code & 0xffffff;
        if (ph > 0 && threadIdx.x < 32)
            wf_wait(A.flags + static_cast<size_t>(ph - 1) * A.nblk, __ldg(A.lohi + 2 * blk),
                    __ldg(A.lohi + 2 * blk + 1), target, A.err);
        __syncthreads();
        wf_run<T, TPR, FLY>(A, ph, blk);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (AMG_WF_FENCE) __threadfence();
            st_release_u32(A.flags + static_cast<size_t>(ph) * A.nblk + blk, target);
        }
        t = s_next;
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(A.ctrl + 1, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            *reinterpret_cast<volatile unsigned *>(A.ctrl) = 0u;
            *reinterpret_cast<volatile unsigned *>(A.ctrl + 1) = 0u;
            __threadfence();
            st_release_u32(A.ctrl + 2, target);
        }
    }
}

// Task order of an nphase-pass chain over nblk blocks: block k of pass p is
// placed once pass p - 1 has been placed on blocks 0 .. H_k + lag, where
// H_k = max_{k' <= k} hi_{k'} (so every block it reads from comes first).
// Returns false if the order fails its own check (each task after the
// tasks it waits on).
inline bool wf_build_order(int nblk, const std::vector<int> &lohi, int nphase, int lag, std::vector<int> &order) {
    order.clear();
    if (nblk <= 0 || nphase <= 0 || nphase > kWfMaxPhases || nblk >= (1 << 24)) return false;
    std::vector<int> H(nblk);
    int m = 0;
    for (int k = 0; k < nblk; ++k) {
        m = std::max(m, lohi[2 * k + 1]);
        H[k] = m;
    }
    std::vector<int> next(nphase, 0);
    order.reserve(static_cast<size_t>(nphase) * nblk);
    while (next[nphase - 1] < nblk) {
        if (next[0] < nblk) order.push_back(next[0]++);
        for (int p = 1; p < nphase; ++p) {
            while (next[p] < nblk) {
                const int k = next[p];
                const long long need = std::min<long long>(nblk, static_cast<long long>(H[k]) + 1 + lag);
                if (next[p - 1] < need) break;
                order.push_back((p << 24) | k);
                ++next[p];
            }
        }
    }
    // check: position of every task after those of its dependencies
    std::vector<int> pos(static_cast<size_t>(nphase) * nblk, -1);
    for (size_t t = 0; t < order.size(); ++t) {
        const int p = order[t] >> 24, k = order[t] & 0xffffff;
        if (pos[static_cast<size_t>(p) * nblk + k] != -1) return false;
        pos[static_cast<size_t>(p) * nblk + k] = static_cast<int>(t);
    }
    for (int p = 0; p < nphase; ++p)
        for (int k = 0; k < nblk; ++k) {
            const int tk = pos[static_cast<size_t>(p) * nblk + k];
            if (tk < 0) return false;
            if (p == 0) continue;
            for (int j = lohi[2 * k]; j <= lohi[2 * k + 1]; ++j)
                if (pos[static_cast<size_t>(p - 1) * nblk + j] > tk) return false;
        }
    return true;
}

}  // namespace amg
