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

// Threads per row for CSR kernels, from the average row length.
inline int pick_tpr(long long nnz, int n) {
    if (n <= 0) return 2;
    double avg = static_cast<double>(nnz) / n;
    if (avg <= 2.5) return 2;
    if (avg <= 6.0) return 4;
    if (avg <= 12.0) return 8;
    if (avg <= 24.0) return 16;
    return 32;
}

inline int grid_for(long long threads) {
    long long g = (threads + kBlock - 1) / kBlock;
    return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace amg
