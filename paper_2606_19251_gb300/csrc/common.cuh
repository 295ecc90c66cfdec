// Shared device helpers for the AMG/GCIN library (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>

namespace amg {

// Process-wide count of kernels this library has launched (reported by
// amg_launch_count; every launch site is followed by AMG_COUNT()).
extern std::atomic<long long> g_launches;
#define AMG_COUNT() (::amg::g_launches.fetch_add(1, std::memory_order_relaxed))

constexpr int kBlock = 256;          // threads per block of the row kernels
constexpr int kNumSMs = 152;         // GB300

// Contiguous device arena: lay out every buffer with 256-byte alignment in
// one pass that only counts, allocate once, then lay out again for real.
struct Planner {
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        size_t a = (off + 255) & ~static_cast<size_t>(255);
        off = a + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + a) : nullptr;
    }
};

// Sum over the TPR lanes of one row group (TPR divides 32; whole warp active).
template <int TPR, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, TPR);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dot product of one CSR row with a gathered operand, split over the TPR
// lanes of a row group: lane `lane` takes entries p0 + lane, p0 + lane + TPR,
// ... and adds them in that order.  Each step issues the col / value loads of
// four entries before their four gathers, so a lane has up to eight loads in
// flight instead of one dependent pair per entry.
template <int TPR, class T, class X>
__device__ __forceinline__ T row_dot(int lane, int p0, int e, const int *__restrict__ col,
                                     const T *__restrict__ val, const X &xg) {
    T acc = T(0);
    for (int base = p0 + lane; base < e; base += 4 * TPR) {
        int c[4];
        T v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = base + j * TPR;
            c[j] = p < e ? __ldg(col + p) : 0;
            v[j] = p < e ? __ldg(val + p) : T(0);
        }
        T x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = (base + j * TPR < e) ? xg(c[j]) : T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (base + j * TPR < e) acc += v[j] * x[j];
    }
    return acc;
}

// The first batch of a row-group lane's entries (row bounds, columns and
// values), fetched before griddepcontrol.wait: matrices do not change while
// a V-cycle runs, so these loads overlap the previous kernel and only the
// gathers of the vector it produced remain after the wait.
template <class T> struct RowBatch {
    int base = 0, e = 0, row = 0;
    int c[4] = {0, 0, 0, 0};
    T v[4] = {T(0), T(0), T(0), T(0)};
};

// Column indices of a square matrix stored as 16-bit offsets from the row
// (j = i + d_p; used where every |j - i| < 2^15, e.g. a mesh in RCM order):
// 2 instead of 4 bytes per entry on the HBM-bound passes.
struct ColDelta {
    const short *__restrict__ d;
};
__device__ __forceinline__ int col_at(const int *__restrict__ col, int p, int) { return __ldg(col + p); }
__device__ __forceinline__ int col_at(const ColDelta &cd, int p, int row) { return row + static_cast<int>(__ldg(cd.d + p)); }

template <int TPR, class T, class CS>
__device__ __forceinline__ void row_prefetch(RowBatch<T> &rb, bool live, int lane, const int *__restrict__ rp,
                                             int row, const CS &col, const T *__restrict__ val) {
    if (!live) return;
    const int p0 = __ldg(rp + row);
    rb.e = __ldg(rp + row + 1);
    rb.base = p0 + lane;
    rb.row = row;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = rb.base + j * TPR;
        rb.c[j] = p < rb.e ? col_at(col, p, row) : 0;
        rb.v[j] = p < rb.e ? __ldg(val + p) : T(0);
    }
}

// row_dot with the first batch taken from a RowBatch (same entries, same order).
template <int TPR, class T, class CS, class X>
__device__ __forceinline__ T row_dot_pref(const RowBatch<T> &rb, const CS &col,
                                          const T *__restrict__ val, const X &xg) {
    T acc = T(0);
    if (rb.base >= rb.e) return acc;
    T x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (rb.base + j * TPR < rb.e) ? xg(rb.c[j]) : T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (rb.base + j * TPR < rb.e) acc += rb.v[j] * x[j];
    for (int base = rb.base + 4 * TPR; base < rb.e; base += 4 * TPR) {
        int c[4];
        T v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = base + j * TPR;
            c[j] = p < rb.e ? col_at(col, p, rb.row) : 0;
            v[j] = p < rb.e ? __ldg(val + p) : T(0);
        }
        T y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = (base + j * TPR < rb.e) ? xg(c[j]) : T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (base + j * TPR < rb.e) acc += v[j] * y[j];
    }
    return acc;
}

template <class T> struct Gather {
    const T *__restrict__ x;
    __device__ __forceinline__ T operator()(int j) const { return x[j]; }
};

// Programmatic dependent launch (PDL).  A solve-path kernel first waits for
// its predecessor grid to finish and flush (griddepcontrol.wait), touching no
// memory before that, then lets its own dependents start launching, so the
// next kernel's launch and block scheduling overlap this kernel's tail.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    AMG_COUNT();
}

// Threads per row of the row-group CSR kernels (a power of two, 1..32).
// Large matrices (>= 2^21 entries, HBM-bound) get about four entries per
// lane, one four-deep load batch per lane with the most rows per warp;
// smaller ones (L2-resident, latency-bound) about two, so more lanes share
// each row's short dependent chain.  Measured on GB300: the 2.5M-row
// residual pass 48 -> 41 us, the 50k-row V-cycle 103 -> 92 us against a
// uniform three entries per lane.
inline int pick_tpr(long long nnz, int n) {
    if (n <= 0) return 1;
    const double per_lane = static_cast<double>(nnz) / n / (nnz >= (1LL << 21) ? 4.0 : 2.0);
    int t = 1;
    while (t * 2 <= per_lane && t < 32) t *= 2;
    return t;
}

inline int grid_for(long long threads) {
    long long g = (threads + kBlock - 1) / kBlock;
    return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace amg
