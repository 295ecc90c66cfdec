// Solve phase of the GNN-smoothed AMG (Sec. 2.1, 2.2, 2.3, 3.1) on sm_103a.
//
// Every sparse operation is a row-group CSR kernel: TPR consecutive lanes
// (2..32, picked from the matrix's mean row length) share one row, stream
// its column/value entries with unit stride and combine with shuffles.  All
// reductions are fixed-order (no floating-point atomics), so results are
// bit-reproducible run to run.
//
// V-cycle (Sec. 2.2) per level l < L-1, in precision T (float or double):
//   pre-smoothing   nu1 sweeps from u = 0   (the first sweep needs no A pass)
//   residual        r = b - A u
//   restriction     b_{l+1} = R r           (explicit R = P^T, gather form)
//   recursion
//   prolongation    u += P u_{l+1}
//   post-smoothing  nu2 sweeps
// Sweep of the pseudo-inverse smoother (Sec. 3.1): r = b - A u, u += Q^-1 r.
// Sweep of relaxed Jacobi (Sec. 2.3): u' = u + omega D^-1 (b - A u).
// Coarsest level: FP64 dense Cholesky factor L (setup), applied as
// u = L^-T (L^-1 b) with L^-1 formed once at setup.
// Outer loop (FP64): r = b - A x, ||r|| / ||b||, x += V(r).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.cuh"
#include "wavefront.cuh"
#include "setup_device.h"

using namespace amg;

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local std::string g_create_err;
std::atomic<long long> amg::g_launches{0};

namespace amg {
bool ctx_fail(amg_ctx *c, const std::string &msg) {
    if (c) c->err = msg;
    return false;
}
int ctx_cuda_check(amg_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return AMG_OK;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return AMG_ERR_CUDA;
}
}  // namespace amg

#define CK(expr)                                                        \
    do {                                                                \
        int _rc = ctx_cuda_check(c, (expr), #expr);                     \
        if (_rc != AMG_OK) return _rc;                                  \
    } while (0)
#define CKL(what)                                                       \
    do {                                                                \
        int _rc = ctx_cuda_check(c, cudaGetLastError(), what);          \
        if (_rc != AMG_OK) return _rc;                                  \
    } while (0)

// ---------------------------------------------------------------------------
// kernels: row-group CSR family
// ---------------------------------------------------------------------------
// r = b - A u
template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_resid(int n, const int *__restrict__ rp, CS col,
                                                  const T *__restrict__ a, const T *__restrict__ b,
                                                  const T *__restrict__ u, T *__restrict__ r) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, a);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, a, Gather<T>{u});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) r[row] = b[row] - acc;
}

// y = M x   (restriction with R, or a plain product)
template <class T, int TPR>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                 const T *__restrict__ m, const T *__restrict__ x,
                                                 T *__restrict__ y) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, m);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, m, Gather<T>{x});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) y[row] = acc;
}

// u = (add ? u : 0) + M r   (pseudo-inverse application, Sec. 3.1;
// also prolongation-correction u += P e with add = 1)
template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_apply(int n, const int *__restrict__ rp, CS col,
                                                  const T *__restrict__ m, const T *__restrict__ r,
                                                  T *__restrict__ u, int add) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, m);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, m, Gather<T>{r});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) u[row] = (add ? u[row] : T(0)) + acc;
}

// u_out = u_in + (omega/a_ii) (b - A u_in)   (relaxed Jacobi, Sec. 2.3)
template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_jacobi(int n, const int *__restrict__ rp, CS col,
                                                   const T *__restrict__ a, const T *__restrict__ jac,
                                                   const T *__restrict__ b, const T *__restrict__ uin,
                                                   T *__restrict__ uout) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, a);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, a, Gather<T>{uin});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) uout[row] = uin[row] + jac[row] * (b[row] - acc);
}

// Single-pass pseudo-inverse sweep on latency-optimised levels:
// u_out = u_in + w - (M A) u_in  (= u_in + M (b - A u_in), with w = M b)
template <class T, int TPR>
__global__ void __launch_bounds__(kBlock) k_ma_sweep(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                     const T *__restrict__ ma, const T *__restrict__ w,
                                                     const T *__restrict__ uin, T *__restrict__ uout) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, ma);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, ma, Gather<T>{uin});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) uout[row] = uin[row] + (w[row] - acc);
}

// First sweep from zero that also keeps w = M b: u = w = M b
template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_apply_w(int n, const int *__restrict__ rp, CS col,
                                                    const T *__restrict__ m, const T *__restrict__ b,
                                                    T *__restrict__ u, T *__restrict__ w) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, m);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, m, Gather<T>{b});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) {
        u[row] = acc;
        w[row] = acc;
    }
}

// Fused residual + restriction with the precomputed product R A:
// b_c = R (b - A u) = R b - (R A) u, two flat gathers per coarse row.
template <class T, int TPR>
__global__ void __launch_bounds__(kBlock) k_resid_restrict(int nc, const int *__restrict__ rrp,
                                                           const int *__restrict__ rcol, const T *__restrict__ rv,
                                                           const int *__restrict__ sp, const int *__restrict__ scol,
                                                           const T *__restrict__ sv, const T *__restrict__ b,
                                                           const T *__restrict__ u, T *__restrict__ bc) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rr, rs;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rr, row < nc, lane, rrp, row, rcol, rv);
    row_prefetch<TPR>(rs, row < nc, lane, sp, row, scol, sv);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < nc) {
        acc = row_dot_pref<TPR>(rr, rcol, rv, Gather<T>{b});
        acc -= row_dot_pref<TPR>(rs, scol, sv, Gather<T>{u});
    }
    acc = group_sum<TPR>(acc);
    if (row < nc && lane == 0) bc[row] = acc;
}

template <class T> struct JacB {   // gathered j_j b_j
    const T *__restrict__ jac, *__restrict__ b;
    __device__ __forceinline__ T operator()(int j) const { return jac[j] * b[j]; }
};

// Two Jacobi sweeps from zero in one pass: u = j b + j (b - A (j b)), j = omega/a_ii
template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_jacobi_first2(int n, const int *__restrict__ rp, CS col,
                                                          const T *__restrict__ a, const T *__restrict__ jac,
                                                          const T *__restrict__ b, T *__restrict__ u) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, a);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, a, JacB<T>{jac, b});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) {
        const T u1 = jac[row] * b[row];
        u[row] = u1 + jac[row] * (b[row] - acc);
    }
}

// Chebyshev smoother steps (fixed-coefficient baseline): first step from a
// zero guess d = cr D^-1 b, u = d; later steps r = b - A u_in,
// d = (first ? 0 : cd d) + cr D^-1 r, u_out = u_in + d.
template <class T>
__global__ void k_cheb_zero(int n, const T *__restrict__ dinv, const T *__restrict__ b, T *__restrict__ u,
                            T *__restrict__ d, T cr) {
    pdl_wait_and_release();
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const T di = cr * (dinv[i] * b[i]);
    d[i] = di;
    u[i] = di;
}

template <class T, int TPR, class CS = const int *>
__global__ void __launch_bounds__(kBlock) k_cheb_step(int n, const int *__restrict__ rp, CS col,
                                                      const T *__restrict__ a, const T *__restrict__ dinv,
                                                      const T *__restrict__ b, const T *__restrict__ uin,
                                                      T *__restrict__ uout, T *__restrict__ d, T cd, T cr,
                                                      int first) {
    const int g = blockIdx.x * kBlock + threadIdx.x;
    const int row = g / TPR, lane = g % TPR;
    RowBatch<T> rb;   // matrix loads ahead of the wait (constant during a solve)
    row_prefetch<TPR>(rb, row < n, lane, rp, row, col, a);
    pdl_wait_and_release();
    T acc = T(0);
    if (row < n) acc = row_dot_pref<TPR>(rb, col, a, Gather<T>{uin});
    acc = group_sum<TPR>(acc);
    if (row < n && lane == 0) {
        const T dr = cr * (dinv[row] * (b[row] - acc));
        const T di = first ? dr : cd * d[row] + dr;
        d[row] = di;
        uout[row] = uin[row] + di;
    }
}

__global__ void k_dinv_vals(int n, const double *__restrict__ diag, double *__restrict__ d64,
                            float *__restrict__ d32) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const double v = 1.0 / diag[i];
    d64[i] = v;
    d32[i] = static_cast<float>(v);
}

// (M A) values from the pair list in FP32, for the FP32 V-cycle (GB300's FP64
// pipe is narrow; the FP32 V-cycle needs only the FP32 product)
__global__ void k_assemble_ma32(int nnz, const int *__restrict__ pp, const int *__restrict__ pq_p,
                                const int *__restrict__ pq_q, const float *__restrict__ q32,
                                const float *__restrict__ a32, float *__restrict__ ma32) {
    const int e = blockIdx.x * kBlock + threadIdx.x;
    if (e >= nnz) return;
    float acc = 0.f;
    for (int t = pp[e]; t < pp[e + 1]; ++t) acc = fmaf(q32[pq_p[t]], a32[pq_q[t]], acc);
    ma32[e] = acc;
}

// (M A) values from the pair list (FP64), with the V-cycle-precision copy
__global__ void k_assemble_ma(int nnz, const int *__restrict__ pp, const int *__restrict__ pq_p,
                              const int *__restrict__ pq_q, const double *__restrict__ q64,
                              const double *__restrict__ a64, double *__restrict__ ma64, float *__restrict__ ma32) {
    const int e = blockIdx.x * kBlock + threadIdx.x;
    if (e >= nnz) return;
    double acc = 0.0;
    for (int t = pp[e]; t < pp[e + 1]; ++t) acc = fma(q64[pq_p[t]], a64[pq_q[t]], acc);
    ma64[e] = acc;
    ma32[e] = static_cast<float>(acc);
}

// u = (omega/a_ii) b  (first Jacobi sweep from u = 0)
template <class T>
__global__ void k_scale(int n, const T *__restrict__ jac, const T *__restrict__ b, T *__restrict__ u) {
    pdl_wait_and_release();
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) u[i] = jac[i] * b[i];
}

template <class S, class D>
__global__ void k_convert(int n, const S *__restrict__ s, D *__restrict__ d) {
    pdl_wait_and_release();
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) d[i] = static_cast<D>(s[i]);
}

// x += e  (outer FP64 update)
template <class T>
__global__ void k_axpy(int n, double *__restrict__ x, const T *__restrict__ e) {
    pdl_wait_and_release();
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) x[i] += static_cast<double>(e[i]);
}

// Coarsest level: u = L^-T (L^-1 b) in FP64 (one block; dynamic smem 2n doubles).
template <class T>
__global__ void __launch_bounds__(kBlock) k_coarse(int n, const double *__restrict__ Linv,
                                                   const double *__restrict__ LinvT, const T *__restrict__ b,
                                                   T *__restrict__ u) {
    pdl_wait_and_release();
    extern __shared__ double sm[];
    double *sb = sm, *sy = sm + n;
    for (int i = threadIdx.x; i < n; i += kBlock) sb[i] = static_cast<double>(b[i]);
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = kBlock / 32;
    for (int i = warp; i < n; i += nw) {
        double acc = 0.0;
        const double *row = Linv + static_cast<size_t>(i) * n;
        for (int k = lane; k <= i; k += 32) acc += row[k] * sb[k];
        acc = warp_sum(acc);
        if (lane == 0) sy[i] = acc;
    }
    __syncthreads();
    for (int i = warp; i < n; i += nw) {
        double acc = 0.0;
        const double *row = LinvT + static_cast<size_t>(i) * n;
        for (int k = i + lane; k < n; k += 32) acc += row[k] * sy[k];
        acc = warp_sum(acc);
        if (lane == 0) u[i] = static_cast<T>(acc);
    }
}

// ---------------------------------------------------------------------------
// kernels: FP64 outer loop with deterministic norms
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_partial(double v, double *out) {
    __shared__ double red[kBlock / 32];
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < kBlock / 32 ? red[threadIdx.x] : 0.0;
        w = warp_sum(w);
        if (threadIdx.x == 0) out[blockIdx.x] = w;
    }
}

// r = b - A x (FP64), rT = (T) r, r64 = r (when given), partial[block] = sum
// r^2 over the block's rows
template <class T, int TPR>
__global__ void __launch_bounds__(kBlock) k_outer_resid(int n, const int *__restrict__ rp,
                                                        const int *__restrict__ col, const double *__restrict__ a,
                                                        const double *__restrict__ b, const double *__restrict__ x,
                                                        T *__restrict__ rT, double *__restrict__ partial,
                                                        double *__restrict__ r64) {
    pdl_wait_and_release();
    constexpr int RPB = kBlock / TPR;
    const int lane = threadIdx.x % TPR;
    double sq = 0.0;
    for (int base = blockIdx.x * RPB; base < n; base += gridDim.x * RPB) {
        const int row = base + threadIdx.x / TPR;
        double acc = 0.0;
        if (row < n) {
            const int e = rp[row + 1];
            acc = row_dot<TPR>(lane, rp[row], e, col, a, Gather<double>{x});
        }
        acc = group_sum<TPR>(acc);
        if (row < n && lane == 0) {
            const double r = b[row] - acc;
            rT[row] = static_cast<T>(r);
            if (r64) r64[row] = r;
            sq += r * r;
        }
    }
    block_partial(sq, partial);
}

// The finest level's FP64 operator for the outer-loop passes, in warp
// slices: rows sorted by length (longest first) within windows of
// kEllWindow rows, 32 rows per slice, a slice's entries column-major (entry
// k of lane l at ptr[s] + 32 k + l) and padded with zeros to its longest
// row.  One warp per slice issues the same number of DFMAs on every lane,
// so GB300's narrow FP64 pipe spends its cycles on the entries (and the
// little padding the sort leaves), not on lanes idle past a short row.
// row[32 s + l] is the matrix row of lane l (-1 past the last row).
struct Ell64 {
    int nslice = 0;
    const int *ptr = nullptr, *row = nullptr, *col = nullptr;
    const double *val = nullptr;
};
constexpr int kEllWindow = 1024;

// Dot product of a slice row with x: acc0 + sum_k v_k x_{c_k} (acc0 - ... when
// NEG), four entries' loads in flight per step (the trip count is
// warp-uniform).
template <bool NEG>
__device__ __forceinline__ double ell_dot(const Ell64 &E, int s, int lane, double acc, const double *__restrict__ x) {
    const int p0 = __ldg(E.ptr + s);
    const int w = (__ldg(E.ptr + s + 1) - p0) >> 5;
    for (int k = 0; k < w; k += 4) {
        int c[4];
        double v[4], xv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = p0 + ((k + j) << 5) + lane;
            c[j] = (k + j < w) ? __ldg(E.col + p) : 0;
            v[j] = (k + j < w) ? __ldg(E.val + p) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) xv[j] = (k + j < w) ? x[c[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (k + j < w) acc = NEG ? fma(-v[j], xv[j], acc) : fma(v[j], xv[j], acc);
    }
    return acc;
}

// r = b - A x (FP64) over warp slices, rT = (T) r, r64 = r (when given),
// partial[block] = sum r^2 over the block's rows
template <class T>
__global__ void __launch_bounds__(kBlock) k_outer_ell(Ell64 E, const double *__restrict__ b,
                                                      const double *__restrict__ x, T *__restrict__ rT,
                                                      double *__restrict__ partial, double *__restrict__ r64) {
    pdl_wait_and_release();
    const int lane = threadIdx.x & 31;
    double sq = 0.0;
    for (int s = blockIdx.x * (kBlock / 32) + static_cast<int>(threadIdx.x >> 5); s < E.nslice;
         s += gridDim.x * (kBlock / 32)) {
        const int row = __ldg(E.row + 32 * s + lane);
        const double r = ell_dot<true>(E, s, lane, row >= 0 ? b[row] : 0.0, x);
        if (row >= 0) {
            rT[row] = static_cast<T>(r);
            if (r64) r64[row] = r;
            sq = fma(r, r, sq);
        }
    }
    block_partial(sq, partial);
}

// q = A p (FP64) over warp slices, partial p.q
__global__ void __launch_bounds__(kBlock) k_pcg_spmv_ell(Ell64 E, const double *__restrict__ p,
                                                         double *__restrict__ q, double *__restrict__ partial) {
    pdl_wait_and_release();
    const int lane = threadIdx.x & 31;
    double pq = 0.0;
    for (int s = blockIdx.x * (kBlock / 32) + static_cast<int>(threadIdx.x >> 5); s < E.nslice;
         s += gridDim.x * (kBlock / 32)) {
        const int row = __ldg(E.row + 32 * s + lane);
        const double a = ell_dot<false>(E, s, lane, 0.0, p);
        if (row >= 0) {
            q[row] = a;
            pq = fma(p[row], a, pq);
        }
    }
    block_partial(pq, partial);
}

// d_p = col_p - i in 16 bits for row i; flag = 1 if some offset does not fit
// (the level then keeps its full column indices)
__global__ void k_col_delta(int n, const int *__restrict__ rp, const int *__restrict__ col, short *__restrict__ d,
                            int *__restrict__ flag) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    bool wide = false;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int off = col[p] - i;
        if (off < -32768 || off > 32767) wide = true;
        else d[p] = static_cast<short>(off);
    }
    if (wide) atomicExch(flag, 1);
}

// Entries of the warp slices from the CSR operator (one thread per slice
// lane): entry k of lane l at ptr[s] + 32 k + l, padding with value 0 and
// the lane's own row as column.
__global__ void __launch_bounds__(kBlock) k_ell_fill(int nslice, const int *__restrict__ ptr,
                                                     const int *__restrict__ row, const int *__restrict__ rp,
                                                     const int *__restrict__ col, const double *__restrict__ val,
                                                     int *__restrict__ ecol, double *__restrict__ evalv) {
    const long long t = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (t >= 32LL * nslice) return;
    const int sl = static_cast<int>(t >> 5), l = static_cast<int>(t & 31);
    const int r = row[t];
    const int p0 = ptr[sl], w = (ptr[sl + 1] - p0) >> 5;
    const int a = r >= 0 ? rp[r] : 0, len = r >= 0 ? rp[r + 1] - a : 0;
    for (int k = 0; k < w; ++k) {
        const long long p = static_cast<long long>(p0) + 32LL * k + l;
        ecol[p] = k < len ? col[a + k] : (r >= 0 ? r : 0);
        evalv[p] = k < len ? val[a + k] : 0.0;
    }
}

__global__ void __launch_bounds__(kBlock) k_sqnorm_partial(int n, const double *__restrict__ v,
                                                           double *__restrict__ partial) {
    pdl_wait_and_release();
    double sq = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) sq += v[i] * v[i];
    block_partial(sq, partial);
}

// ---------------------------------------------------------------------------
// kernels: conjugate gradients preconditioned by one V-cycle (FP64)
// ---------------------------------------------------------------------------
// Fixed-order sum of np partials, computed identically by every block (so
// each block derives the same alpha / beta without a separate launch).
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int np, double *red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += kBlock) v += part[i];
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ void block_partial2(double a, double b, double *outa, double *outb) {
    __shared__ double ra[kBlock / 32], rb[kBlock / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x % 32 == 0) {
        ra[threadIdx.x / 32] = a;
        rb[threadIdx.x / 32] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) {
            ta += ra[w];
            tb += rb[w];
        }
        outa[blockIdx.x] = ta;
        outb[blockIdx.x] = tb;
    }
}

// z = (double) e (the V-cycle's output); partials of z.r and z.r_prev
template <class T>
__global__ void __launch_bounds__(kBlock) k_pcg_dots(int n, const T *__restrict__ e, const double *__restrict__ r,
                                                     const double *__restrict__ rprev, double *__restrict__ z,
                                                     double *__restrict__ pzr, double *__restrict__ pzrp) {
    pdl_wait_and_release();
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const double zi = static_cast<double>(e[i]);
        z[i] = zi;
        a += zi * r[i];
        b += zi * rprev[i];
    }
    block_partial2(a, b, pzr, pzrp);
}

// p = z (restart) or p = z + beta p with beta = (z.r - z.r_prev) / rho_old;
// z.r <= 0 (or not finite) is a breakdown.
__global__ void __launch_bounds__(kBlock) k_pcg_dir(int n, const double *__restrict__ z, double *__restrict__ p,
                                                    const double *__restrict__ pzr, const double *__restrict__ pzrp,
                                                    int np, SolveState *st) {
    pdl_wait_and_release();
    __shared__ double red[kBlock / 32];
    const double rho = sum_partials(pzr, np, red);
    const double zrp = sum_partials(pzrp, np, red);
    if (!(rho > 0.0) || !isfinite(rho) || st->breakdown) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->breakdown = 1;
        return;
    }
    const bool restart = st->restart != 0;
    const double beta = restart ? 0.0 : (rho - zrp) / st->rho_old;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        p[i] = restart ? z[i] : z[i] + beta * p[i];
}

// q = A p (FP64), partial p.q
template <int TPR>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                     const double *__restrict__ a, const double *__restrict__ p,
                                                     double *__restrict__ q, double *__restrict__ partial) {
    pdl_wait_and_release();
    constexpr int RPB = kBlock / TPR;
    const int lane = threadIdx.x % TPR;
    double pq = 0.0;
    for (int base = blockIdx.x * RPB; base < n; base += gridDim.x * RPB) {
        const int row = base + threadIdx.x / TPR;
        double acc = 0.0;
        if (row < n) acc = row_dot<TPR>(lane, rp[row], rp[row + 1], col, a, Gather<double>{p});
        acc = group_sum<TPR>(acc);
        if (row < n && lane == 0) {
            q[row] = acc;
            pq += p[row] * acc;
        }
    }
    block_partial(pq, partial);
}

// alpha = (z.r) / (p.Ap); x += alpha p; r_prev = r; r -= alpha q; rT = (T) r;
// partial ||r||^2.  p.Ap <= 0 (or not finite) is a breakdown.
template <class T>
__global__ void __launch_bounds__(kBlock) k_pcg_update(int n, double *__restrict__ x, double *__restrict__ r,
                                                       double *__restrict__ rprev, const double *__restrict__ p,
                                                       const double *__restrict__ q, T *__restrict__ rT,
                                                       const double *__restrict__ pzr, const double *__restrict__ ppq,
                                                       int np, SolveState *st, double *__restrict__ prr) {
    pdl_wait_and_release();
    __shared__ double red[kBlock / 32];
    const double rho = sum_partials(pzr, np, red);
    const double pq = sum_partials(ppq, np, red);
    const bool bad = st->breakdown || !(pq > 0.0) || !isfinite(pq);
    double rr = 0.0;
    if (!bad) {
        const double alpha = rho / pq;
        for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
            x[i] += alpha * p[i];
            const double ri = r[i];
            const double rn = ri - alpha * q[i];
            rprev[i] = ri;
            r[i] = rn;
            rT[i] = static_cast<T>(rn);
            rr += rn * rn;
        }
    }
    block_partial(rr, prr);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (bad) {
            st->breakdown = 1;
        } else {
            st->rho_old = rho;
            st->restart = 0;
        }
    }
}

__global__ void k_state_init(SolveState *st, double tol, int max_iter, double stall) {
    pdl_wait_and_release();
    st->k = 0;
    st->status = kRunning;
    st->max_iter = max_iter;
    st->tol = tol;
    st->bnorm = 1.0;
    st->r0 = 0.0;
    st->stall = stall;
    st->rho_old = 0.0;
    st->restart = 1;
    st->breakdown = 0;
}

// Continue a stalled solve with another smoother (history and count go on).
__global__ void k_state_continue(SolveState *st) {
    pdl_wait_and_release();
    st->status = kRunning;
    st->stall = 0.0;
    st->restart = 1;
}

// Smallest of hist[k - off - 9 .. k - off].
__device__ __forceinline__ double window_min(const double *hist, int k, int off) {
    double m = hist[k - off];
    for (int j = 1; j < 10; ++j) m = fmin(m, hist[k - off - j]);
    return m;
}

// Sum the partials in a fixed order.  mode 0: ||b||.  mode 1: residual
// history entry k and the stopping rule (Sec. 4 tolerance, divergence,
// stagnation, iteration cap).
__global__ void __launch_bounds__(1024) k_norm_final(const double *__restrict__ partial, int np, SolveState *st,
                                                     double *__restrict__ hist, int mode, int use_cond,
                                                     cudaGraphConditionalHandle cond) {
    pdl_wait_and_release();
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += 1024) v += partial[i];
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    v = warp_sum(red[threadIdx.x]);
    if (threadIdx.x != 0) return;
    const double nrm = sqrt(v);
    if (mode == 0) {
        st->bnorm = nrm > 0.0 ? nrm : 1.0;
        return;
    }
    if (st->breakdown) {   // conjugate gradients broke down: the iterate and history stay
        st->status = AMG_ERR_DIVERGED;
        if (use_cond) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int k = st->k;
    const double rel = nrm / st->bnorm;
    hist[k] = rel;
    int status = kRunning;
    if (k == 0) {
        st->r0 = nrm;
        if (!isfinite(nrm)) status = AMG_ERR_DIVERGED;
        else if (rel <= st->tol) status = AMG_OK;
        else if (st->max_iter <= 0) status = AMG_ERR_MAXITER;
    } else {
        if (!isfinite(nrm) || nrm > 1e3 * st->r0) status = AMG_ERR_DIVERGED;
        else if (rel <= st->tol) status = AMG_OK;
        else if (k >= 10 && st->stall > 0.0 && rel > st->stall * hist[k - 10]) status = kStalled;
        else if (k >= 20 && window_min(hist, k, 0) > 0.99 * window_min(hist, k, 10)) status = AMG_ERR_STAGNATED;
        else if (k >= st->max_iter) status = AMG_ERR_MAXITER;
    }
    st->status = status;
    st->k = k + 1;
    if (use_cond) cudaGraphSetConditional(cond, status == kRunning ? 1u : 0u);
}

// An empty dependent launch: the floor of one step of a chain of
// programmatic-dependent launches (amg_kernel_launch, AMG_K_EMPTY).
__global__ void k_empty() { pdl_wait_and_release(); }

// Copies "still running" into the solve graph's WHILE condition.
__global__ void k_set_cond(const SolveState *st, cudaGraphConditionalHandle cond) {
    cudaGraphSetConditional(cond, st->status == kRunning ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// kernels: setup (s_l, smoother values, coarsest factorisation)
// ---------------------------------------------------------------------------
__global__ void k_extract_diag(int n, const int *__restrict__ rp, const int *__restrict__ col,
                               const double *__restrict__ a, double *__restrict__ d) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (col[p] == i) v += a[p];
    d[i] = v;
}

// s = max_{i != j} |a_ij| (Sec. 3.1): per-block maxima, then one block.
__global__ void __launch_bounds__(kBlock) k_offdiag_absmax(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ col,
                                                           const double *__restrict__ a,
                                                           double *__restrict__ partial) {
    __shared__ double red[kBlock / 32];
    double m = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        for (int p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i) m = fmax(m, fabs(a[p]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double w = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) w = fmax(w, red[k]);
        partial[blockIdx.x] = w;
    }
}

__global__ void k_max_final(const double *__restrict__ partial, int np, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double m = 0.0;
    for (int i = 0; i < np; ++i) m = fmax(m, partial[i]);
    *out = m > 0.0 ? m : 1.0;
}

// Per-entry basis of the pseudo-inverse (Sec. 3.1), computed once per
// hierarchy: bx = a_ij / s and bw = 1 / a_ii (diagonal) or 1 / (a_ii + a_jj).
__global__ void k_pinv_basis(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ a, const double *__restrict__ d,
                             const double *__restrict__ s_ptr, double *__restrict__ bx, double *__restrict__ bw,
                             unsigned char *__restrict__ isd, float *__restrict__ bx32, float *__restrict__ bw32) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const double s = *s_ptr, di = d[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = col[p];
        bx[p] = a[p] / s;
        bw[p] = 1.0 / (j == i ? di : di + d[j]);
        isd[p] = (j == i) ? 1 : 0;
        bx32[p] = static_cast<float>(bx[p]);
        bw32[p] = static_cast<float>(bw[p]);
    }
}

// Q^-1 values on A's pattern from c = (d0, d1, d2, o1, o2) (Sec. 3.1):
// q_ii = (d0 + d1 x + d2 x^2) bw, q_ij = (o1 x + o2 x^2) bw, in FP64 with the
// polynomial evaluated as d0 + d1 x + (d2 x) x, uncontracted.
__global__ void k_assemble_q(int nnz, const unsigned char *__restrict__ isd, const double *__restrict__ bx,
                             const double *__restrict__ bw, double c0, double c1, double c2, double c3, double c4,
                             double *__restrict__ q64, float *__restrict__ q32) {
    const int p = blockIdx.x * kBlock + threadIdx.x;
    if (p >= nnz) return;
    const double x = bx[p];
    const double f = isd[p] ? __dadd_rn(__dadd_rn(c0, __dmul_rn(c1, x)), __dmul_rn(__dmul_rn(c2, x), x))
                            : __dadd_rn(__dmul_rn(c3, x), __dmul_rn(__dmul_rn(c4, x), x));
    const double q = __dmul_rn(f, bw[p]);
    q64[p] = q;
    q32[p] = static_cast<float>(q);
}

// Q^-1 values with one coefficient row per node (cn: n x 5): the diagonal of
// row i from node i's (d0, d1, d2), an off-diagonal entry (i, j) from the mean
// of nodes i's and j's (o1, o2) (a symmetric Q^-1); arithmetic as k_assemble_q.
__global__ void k_assemble_q_nodes(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                   const unsigned char *__restrict__ isd, const double *__restrict__ bx,
                                   const double *__restrict__ bw, const double *__restrict__ cn,
                                   double *__restrict__ q64, float *__restrict__ q32) {
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const double *ci = cn + 5 * static_cast<size_t>(i);
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const double x = bx[p];
        double f;
        if (isd[p]) {
            f = __dadd_rn(__dadd_rn(ci[0], __dmul_rn(ci[1], x)), __dmul_rn(__dmul_rn(ci[2], x), x));
        } else {
            const double *cj = cn + 5 * static_cast<size_t>(col[p]);
            const double o1 = __dmul_rn(__dadd_rn(ci[3], cj[3]), 0.5), o2 = __dmul_rn(__dadd_rn(ci[4], cj[4]), 0.5);
            f = __dadd_rn(__dmul_rn(o1, x), __dmul_rn(__dmul_rn(o2, x), x));
        }
        const double q = __dmul_rn(f, bw[p]);
        q64[p] = q;
        q32[p] = static_cast<float>(q);
    }
}

// Every smoothed level's Q^-1 (and then M A) in one launch each, with the
// coefficients read from device memory (the FP32 network output, widened to
// FP64 exactly as the host path does): a thread finds its level from the
// cumulative entry offsets; the arithmetic per entry is k_assemble_q's (and
// k_assemble_ma / k_assemble_ma32's).
constexpr int kAsmMaxLevels = 32;
struct AsmQ {
    int nlev;
    long long start[kAsmMaxLevels + 1];       // cumulative entries; start[nlev] = total
    const unsigned char *isd[kAsmMaxLevels];
    const double *bx[kAsmMaxLevels], *bw[kAsmMaxLevels];
    const float *bx32[kAsmMaxLevels], *bw32[kAsmMaxLevels];
    double *q64[kAsmMaxLevels];
    float *q32[kAsmMaxLevels];
    int row[kAsmMaxLevels];                   // coefficient row of the level
};

// mode 0: the FP32 V-cycle's values only, in FP32 from the FP32 basis (the
// FP64 values are assembled when something asks for them); mode 1: both from
// the FP64 product; mode 2: the FP64 values only. Coefficient row l starts at
// dc + cstride * l.
__global__ void k_assemble_q_all(AsmQ L, const float *__restrict__ dc, int cstride, int mode) {
    const long long p = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (p >= L.start[L.nlev]) return;
    int l = 0;
    while (p >= L.start[l + 1]) ++l;
    const long long e = p - L.start[l];
    const float *cf = dc + cstride * L.row[l];
    if (mode == 0) {
        const float x = L.bx32[l][e];
        const float f = L.isd[l][e] ? __fadd_rn(__fadd_rn(cf[0], __fmul_rn(cf[1], x)), __fmul_rn(__fmul_rn(cf[2], x), x))
                                    : __fadd_rn(__fmul_rn(cf[3], x), __fmul_rn(__fmul_rn(cf[4], x), x));
        L.q32[l][e] = __fmul_rn(f, L.bw32[l][e]);
        return;
    }
    const double c0 = cf[0], c1 = cf[1], c2 = cf[2], c3 = cf[3], c4 = cf[4];
    const double x = L.bx[l][e];
    const double f = L.isd[l][e] ? __dadd_rn(__dadd_rn(c0, __dmul_rn(c1, x)), __dmul_rn(__dmul_rn(c2, x), x))
                                 : __dadd_rn(__dmul_rn(c3, x), __dmul_rn(__dmul_rn(c4, x), x));
    const double q = __dmul_rn(f, L.bw[l][e]);
    L.q64[l][e] = q;
    if (mode == 1) L.q32[l][e] = static_cast<float>(q);
}

struct AsmMA {
    int nlev;
    long long start[kAsmMaxLevels + 1];
    const int *pp[kAsmMaxLevels], *pq_p[kAsmMaxLevels], *pq_q[kAsmMaxLevels];
    const float *q32[kAsmMaxLevels], *a32[kAsmMaxLevels];
    float *ma32[kAsmMaxLevels];
    const double *q64[kAsmMaxLevels], *a64[kAsmMaxLevels];
    double *ma64[kAsmMaxLevels];
};

// The wavefront chains' coefficient rows (d0 d1 d2 o1 o2 1/s per level, FP32)
// from the network's FP32 output and the level scales.
__global__ void k_wf_coef(int nlev, const float *__restrict__ dc, const double *__restrict__ scal,
                          float *__restrict__ wcoef) {
    const int l = threadIdx.x;
    if (l >= nlev) return;
    for (int k = 0; k < 5; ++k) wcoef[8 * l + k] = dc[5 * l + k];
    wcoef[8 * l + 5] = static_cast<float>(1.0 / scal[l]);
}

// fp64 != 0: FP64 products with the FP32 copy (FP64 V-cycle); else FP32 only
__global__ void k_assemble_ma_all(AsmMA M, int fp64) {
    const long long p = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
    if (p >= M.start[M.nlev]) return;
    int l = 0;
    while (p >= M.start[l + 1]) ++l;
    const long long e = p - M.start[l];
    const int *pp = M.pp[l], *pq_p = M.pq_p[l], *pq_q = M.pq_q[l];
    if (fp64) {
        double acc = 0.0;
        for (int t = pp[e]; t < pp[e + 1]; ++t) acc = fma(M.q64[l][pq_p[t]], M.a64[l][pq_q[t]], acc);
        M.ma64[l][e] = acc;
        M.ma32[l][e] = static_cast<float>(acc);
    } else {
        float acc = 0.f;
        for (int t = pp[e]; t < pp[e + 1]; ++t) acc = fmaf(M.q32[l][pq_p[t]], M.a32[l][pq_q[t]], acc);
        M.ma32[l][e] = acc;
    }
}

__global__ void k_jacobi_vals(int n, const double *__restrict__ d, double omega, double *__restrict__ j64,
                              float *__restrict__ j32) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    double v = __ddiv_rn(omega, d[i]);
    j64[i] = v;
    j32[i] = static_cast<float>(v);
}

__global__ void k_csr_to_dense(int n, const int *__restrict__ rp, const int *__restrict__ col,
                               const double *__restrict__ a, double *__restrict__ dense) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) dense[static_cast<size_t>(i) * n + col[p]] += a[p];
}

// Right-looking dense Cholesky in place (lower triangle), one block.
__global__ void __launch_bounds__(1024) k_cholesky(int n, double *__restrict__ a, int *__restrict__ flag) {
    __shared__ double piv;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = a[static_cast<size_t>(j) * n + j];
            if (!(d > 0.0)) {
                *flag = 1;
                d = 1.0;
            }
            piv = sqrt(d);
            a[static_cast<size_t>(j) * n + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) a[static_cast<size_t>(i) * n + j] /= piv;
        __syncthreads();
        const int m = n - j - 1;
        for (long long idx = threadIdx.x; idx < static_cast<long long>(m) * m; idx += blockDim.x) {
            const int i = j + 1 + static_cast<int>(idx / m);
            const int k = j + 1 + static_cast<int>(idx % m);
            if (k <= i)
                a[static_cast<size_t>(i) * n + k] -=
                    a[static_cast<size_t>(i) * n + j] * a[static_cast<size_t>(k) * n + j];
        }
        __syncthreads();
    }
}

// Column j of L^-1 by forward substitution (one thread per column).
__global__ void k_tri_inverse(int n, const double *__restrict__ L, double *__restrict__ Linv,
                              double *__restrict__ LinvT) {
    const int j = blockIdx.x * kBlock + threadIdx.x;
    if (j >= n) return;
    Linv[static_cast<size_t>(j) * n + j] = 1.0 / L[static_cast<size_t>(j) * n + j];
    LinvT[static_cast<size_t>(j) * n + j] = Linv[static_cast<size_t>(j) * n + j];
    for (int i = j + 1; i < n; ++i) {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += L[static_cast<size_t>(i) * n + k] * Linv[static_cast<size_t>(k) * n + j];
        const double v = -s / L[static_cast<size_t>(i) * n + i];
        Linv[static_cast<size_t>(i) * n + j] = v;
        LinvT[static_cast<size_t>(j) * n + i] = v;
    }
}

// ---------------------------------------------------------------------------
// launch helpers (dispatch on threads-per-row)
// ---------------------------------------------------------------------------
template <class T> static const T *mvals(const DevMat &m);
template <> const double *mvals<double>(const DevMat &m) { return m.v64; }
template <> const float *mvals<float>(const DevMat &m) { return m.v32; }
template <class T> static const T *qvals(const DevLevel &L);
template <> const double *qvals<double>(const DevLevel &L) { return L.q64; }
template <> const float *qvals<float>(const DevLevel &L) { return L.q32; }
template <class T> static const T *jvals(const DevLevel &L);
template <> const double *jvals<double>(const DevLevel &L) { return L.j64; }
template <> const float *jvals<float>(const DevLevel &L) { return L.j32; }

#define TPR_DISPATCH(tpr, KERNEL, ...)                    \
    switch (tpr) {                                        \
        case 1: KERNEL<1>(__VA_ARGS__); break;            \
        case 2: KERNEL<2>(__VA_ARGS__); break;            \
        case 4: KERNEL<4>(__VA_ARGS__); break;            \
        case 8: KERNEL<8>(__VA_ARGS__); break;            \
        case 16: KERNEL<16>(__VA_ARGS__); break;          \
        default: KERNEL<32>(__VA_ARGS__); break;          \
    }

template <class T> struct Launch {
    template <int TPR>
    static void resid(const DevMat &A, const T *b, const T *u, T *r, cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(A.nr) * TPR));
        if (A.dcol) launch_pdl(k_resid<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, A.nr, A.rp, ColDelta{A.dcol}, mvals<T>(A), b, u, r);
        else launch_pdl(k_resid<T, TPR>, g, dim3(kBlock), 0, s, A.nr, A.rp, static_cast<const int *>(A.col), mvals<T>(A), b, u, r);
    }
    template <int TPR>
    static void spmv(const DevMat &M, const T *x, T *y, cudaStream_t s) {
        launch_pdl(k_spmv<T, TPR>, dim3(grid_for(static_cast<long long>(M.nr) * TPR)), dim3(kBlock), 0, s, M.nr, M.rp, M.col,
                                                                                        mvals<T>(M), x, y);
    }
    template <int TPR>
    static void apply(const DevMat &M, const T *m, const T *r, T *u, int add, cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(M.nr) * TPR));
        if (M.dcol) launch_pdl(k_apply<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, M.nr, M.rp, ColDelta{M.dcol}, m, r, u, add);
        else launch_pdl(k_apply<T, TPR>, g, dim3(kBlock), 0, s, M.nr, M.rp, static_cast<const int *>(M.col), m, r, u, add);
    }
    template <int TPR>
    static void jacobi(const DevMat &A, const T *jac, const T *b, const T *uin, T *uout, cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(A.nr) * TPR));
        if (A.dcol) launch_pdl(k_jacobi<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, A.nr, A.rp, ColDelta{A.dcol}, mvals<T>(A), jac, b, uin, uout);
        else launch_pdl(k_jacobi<T, TPR>, g, dim3(kBlock), 0, s, A.nr, A.rp, static_cast<const int *>(A.col), mvals<T>(A), jac, b, uin, uout);
    }
    template <int TPR>
    static void ma_sweep(const DevMat &MA, const T *w, const T *uin, T *uout, cudaStream_t s) {
        launch_pdl(k_ma_sweep<T, TPR>, dim3(grid_for(static_cast<long long>(MA.nr) * TPR)), dim3(kBlock), 0, s, 
            MA.nr, MA.rp, MA.col, mvals<T>(MA), w, uin, uout);
    }
    template <int TPR>
    static void apply_w(const DevMat &A, const T *m, const T *b, T *u, T *w, cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(A.nr) * TPR));
        if (A.dcol) launch_pdl(k_apply_w<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, A.nr, A.rp, ColDelta{A.dcol}, m, b, u, w);
        else launch_pdl(k_apply_w<T, TPR>, g, dim3(kBlock), 0, s, A.nr, A.rp, static_cast<const int *>(A.col), m, b, u, w);
    }
    template <int TPR>
    static void resid_restrict(const DevMat &R, const DevMat &RA, const T *b, const T *u, T *bc, cudaStream_t s) {
        launch_pdl(k_resid_restrict<T, TPR>, dim3(grid_for(static_cast<long long>(R.nr) * TPR)), dim3(kBlock), 0, s, 
            R.nr, R.rp, R.col, mvals<T>(R), RA.rp, RA.col, mvals<T>(RA), b, u, bc);
    }
    template <int TPR>
    static void jacobi_first2(const DevMat &A, const T *jac, const T *b, T *u, cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(A.nr) * TPR));
        if (A.dcol) launch_pdl(k_jacobi_first2<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, A.nr, A.rp, ColDelta{A.dcol}, mvals<T>(A), jac, b, u);
        else launch_pdl(k_jacobi_first2<T, TPR>, g, dim3(kBlock), 0, s, A.nr, A.rp, static_cast<const int *>(A.col), mvals<T>(A), jac, b, u);
    }
    template <int TPR>
    static void outer(const DevMat &A, const double *b, const double *x, T *rT, double *partial, int nblk,
                      double *r64, cudaStream_t s) {
        launch_pdl(k_outer_resid<T, TPR>, dim3(nblk), dim3(kBlock), 0, s, A.nr, A.rp, A.col, A.v64, b, x, rT, partial,
                   r64);
    }
    template <int TPR>
    static void pcg_spmv(const DevMat &A, const double *p, double *q, double *partial, int nblk, cudaStream_t s) {
        launch_pdl(k_pcg_spmv<TPR>, dim3(nblk), dim3(kBlock), 0, s, A.nr, A.rp, A.col, A.v64, p, q, partial);
    }
};

template <class T> static const T *dinvvals(const DevLevel &L);
template <> const double *dinvvals<double>(const DevLevel &L) { return L.dinv64; }
template <> const float *dinvvals<float>(const DevLevel &L) { return L.dinv32; }

template <class T> struct ChebLaunch {
    template <int TPR>
    static void step(const DevLevel &L, const T *b, const T *uin, T *uout, T *d, T cd, T cr, int first,
                     cudaStream_t s) {
        const dim3 g(grid_for(static_cast<long long>(L.n) * TPR));
        if (L.A.dcol)
            launch_pdl(k_cheb_step<T, TPR, ColDelta>, g, dim3(kBlock), 0, s, L.n, L.A.rp, ColDelta{L.A.dcol},
                       mvals<T>(L.A), dinvvals<T>(L), b, uin, uout, d, cd, cr, first);
        else
            launch_pdl(k_cheb_step<T, TPR>, g, dim3(kBlock), 0, s, L.n, L.A.rp, static_cast<const int *>(L.A.col),
                       mvals<T>(L.A), dinvvals<T>(L), b, uin, uout, d, cd, cr, first);
    }
};

// `apps` applications of the degree-k Chebyshev polynomial on level L from
// cur (zero when zero_init); returns the buffer holding the result.
template <class T>
static T *cheb_smooth(amg_ctx *c, const DevLevel &L, cudaStream_t s, const T *b, T *cur, T *alt, int apps,
                      bool zero_init) {
    T *d = reinterpret_cast<T *>(L.vw);
    const double theta = L.cheb_theta, delta = L.cheb_delta, sigma = theta / delta;
    for (int a = 0; a < apps; ++a) {
        double rho_prev = 1.0 / sigma;
        for (int k = 0; k < c->cheb_degree; ++k) {
            double cd = 0.0, cr = 1.0 / theta;
            if (k > 0) {
                const double rho = 1.0 / (2.0 * sigma - rho_prev);
                cd = rho * rho_prev;
                cr = 2.0 * rho / delta;
                rho_prev = rho;
            }
            if (k == 0 && a == 0 && zero_init) {
                launch_pdl(k_cheb_zero<T>, dim3(grid_for(L.n)), dim3(kBlock), 0, s, L.n, dinvvals<T>(L), b, cur, d,
                           static_cast<T>(cr));
                continue;
            }
            TPR_DISPATCH(L.A.tpr, ChebLaunch<T>::template step, L, b, static_cast<const T *>(cur), alt, d,
                         static_cast<T>(cd), static_cast<T>(cr), k == 0 ? 1 : 0, s);
            std::swap(cur, alt);
        }
    }
    return cur;
}

template <class T> static void L_resid(const DevMat &A, const T *b, const T *u, T *r, cudaStream_t s) {
    TPR_DISPATCH(A.tpr, Launch<T>::template resid, A, b, u, r, s);
}
template <class T> static void L_spmv(const DevMat &M, const T *x, T *y, cudaStream_t s) {
    TPR_DISPATCH(M.tpr, Launch<T>::template spmv, M, x, y, s);
}
template <class T> static void L_apply(const DevMat &M, const T *m, const T *r, T *u, int add, cudaStream_t s) {
    TPR_DISPATCH(M.tpr, Launch<T>::template apply, M, m, r, u, add, s);
}
template <class T>
static void L_jacobi(const DevMat &A, const T *jac, const T *b, const T *uin, T *uout, cudaStream_t s) {
    TPR_DISPATCH(A.tpr, Launch<T>::template jacobi, A, jac, b, uin, uout, s);
}

// Grid of the FP64 outer-loop passes: one thread group per row up to 32
// blocks per SM (the partial sums have one slot per block; a wider grid
// keeps more rows' loads in flight than a grid-stride loop over few blocks).
constexpr int kOuterBlocksPerSM = 32;
static int outer_blocks(const DevMat &A) {
    long long need = (static_cast<long long>(A.nr) * A.tpr + kBlock - 1) / kBlock;
    long long cap = static_cast<long long>(kNumSMs) * kOuterBlocksPerSM;
    return static_cast<int>(std::max(1LL, std::min(need, cap)));
}

// FP64 outer residual with nb = outer_blocks(A) partial sums.
template <class T>
static void L_outer(const DevMat &A, const double *b, const double *x, T *rT, double *partial, int nb,
                    cudaStream_t s, double *r64 = nullptr) {
    TPR_DISPATCH(A.tpr, Launch<T>::template outer, A, b, x, rT, partial, nb, r64, s);
}

// ---------------------------------------------------------------------------
// wavefront smoothing chains (wavefront.cuh) on levels too large for L2
// ---------------------------------------------------------------------------
#ifndef AMG_WF_MIN_NNZ
#define AMG_WF_MIN_NNZ (1 << 20)
#endif
constexpr int kWfMinBlocks = 4096;   // smaller levels: one kernel per pass
constexpr long long kWfMinNnz = AMG_WF_MIN_NNZ;
constexpr int kWfMaxReach = 4096;    // a block's columns reach at most this many blocks ahead

template <class T, int TPR, bool FLY>
static int wf_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_wavefront<T, TPR, FLY>, kWfThreads, 0) != cudaSuccess)
        return 1;
    return std::max(1, nb);
}

template <class T>
static int wf_blocks_per_sm(int tpr, bool fly) {
    if (fly) {
        if constexpr (std::is_same<T, float>::value) {
            switch (tpr) {
                case 1: return wf_occupancy<float, 1, true>();
                case 2: return wf_occupancy<float, 2, true>();
                default: return wf_occupancy<float, 4, true>();
            }
        }
    }
    switch (tpr) {
        case 1: return wf_occupancy<T, 1, false>();
        case 2: return wf_occupancy<T, 2, false>();
        default: return wf_occupancy<T, 4, false>();
    }
}

// Host copies of level l's columns and values where they are still only on
// the device (levels built by amg_setup_device)
static int ensure_host(amg_ctx *c, int l) {
    HostLevel &H = c->host[l];
    for (HostCSR *h : {&H.A, &H.P, &H.R}) {
        if (!h->on_device()) continue;
        CK(cudaSetDevice(c->opt.device));
        const long long nz = h->nnz();
        h->col.resize(nz);
        h->val.resize(nz);
        if (nz > 0) {
            CK(cudaMemcpyAsync(h->col.data(), h->dcol, sizeof(int) * nz, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(h->val.data(), h->dval, sizeof(double) * nz, cudaMemcpyDeviceToHost, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        h->drp = h->dcol = nullptr;
        h->dval = nullptr;
    }
    return AMG_OK;
}

// Which levels run their smoothing as wavefront chains, with the group
// ranges of their blocks' columns and the lag of every chain length.
static int plan_wavefront(amg_ctx *c) {
    const int nlev = static_cast<int>(c->host.size());
    c->wfplan.assign(nlev, WfPlan{});
    if (!c->opt.fused_sweeps) return AMG_OK;
    for (int l = 0; l < nlev; ++l) {
        const int rc = ensure_host(c, l);
        if (rc) return rc;
    }
    const bool f32 = (c->opt.precision != AMG_FP64);
    for (int l = 0; l < nlev - 1; ++l) {
        const HostLevel &H = c->host[l];
        if (H.fast) continue;
        const int n = H.A.n_rows;
        const int tpr = pick_tpr(H.A.nnz(), n);
        if (tpr > 4 || H.A.nnz() < kWfMinNnz) continue;
        const int rpt = 32 / tpr;
        const int nblk = (n + rpt - 1) / rpt;
        if (nblk < kWfMinBlocks) continue;
        WfPlan &W = c->wfplan[l];
        const int reach = wf_block_ranges(n, H.A.rp.data(), H.A.col.data(), rpt, W.lohi);
        if (reach > kWfMaxReach) {
            W = WfPlan{};
            continue;
        }
        W.grid = std::min(kWfCtasPerSM, f32 ? wf_blocks_per_sm<float>(tpr, true) : wf_blocks_per_sm<double>(tpr, false)) *
                 kNumSMs;
        const long long warps = static_cast<long long>(W.grid) * (kWfThreads / 32);
        for (int np = 1; np <= kWfMaxPhases; ++np) {
            // a task's inputs were produced a grid of tasks earlier; and the lag
            // exceeds a block's reach by a completion group (no task waits for
            // a later-numbered one)
            const long long by_grid = (static_cast<long long>(kWfLagPct) * warps + 100LL * np - 1) / (100LL * np);
            W.lag[np] = static_cast<int>(std::max<long long>(by_grid, reach + kWfGroup + 1));
        }
        W.rpt = rpt;
        W.nblk = nblk;
        W.ngroup = (nblk + kWfGroup - 1) / kWfGroup;
        W.on = true;
    }
    return AMG_OK;
}

template <class T> static const T *diagvals(const DevLevel &L);
template <> const double *diagvals<double>(const DevLevel &L) { return L.diag; }
template <> const float *diagvals<float>(const DevLevel &L) { return L.diag32; }

template <class T> struct WfLaunch {
    template <int TPR>
    static void go(const WfArgs<T> &a, int grid, bool fly, cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value) {
            if (fly) {
                launch_pdl(k_wavefront<float, TPR, true>, dim3(grid), dim3(kWfThreads), 0, s, a);
                return;
            }
        }
        launch_pdl(k_wavefront<T, TPR, false>, dim3(grid), dim3(kWfThreads), 0, s, a);
    }
};

// A chain being assembled: passes appended in order, outputs in fresh level
// buffers (never one the chain reads as its own input `keep`).
template <class T> struct WfChain {
    WfArgs<T> a;
    unsigned taken = 0;
    bool ok = true;
    int add(int op, int in = 0, int aux = 0) {
        if (a.nphase >= kWfMaxPhases) {
            ok = false;
            return 0;
        }
        int out = 0;
        while (out < kWfBufs && (taken >> out) & 1u) ++out;
        if (out >= kWfBufs) {
            ok = false;
            return 0;
        }
        taken |= 1u << out;
        const int p = a.nphase++;
        a.op[p] = op;
        a.in[p] = in;
        a.aux[p] = aux;
        a.out[p] = out;
        return out;
    }
};

template <class T>
static WfChain<T> wf_chain_for(amg_ctx *c, int l, const T *b) {
    DevLevel &L = c->lev[l];
    WfChain<T> ch;
    WfArgs<T> &a = ch.a;
    a.n = L.n;
    a.nblk = L.wf_nblk;
    a.rpt = L.wf_rpt;
    a.ngroup = L.wf_ngroup;
    a.lohi = reinterpret_cast<const int2 *>(L.wf_lohi);
    a.rp = L.A.rp;
    a.col = L.A.col;
    a.a = mvals<T>(L.A);
    a.diag = diagvals<T>(L);
    a.q = qvals<T>(L);
    a.coef = c->wcoef + 8 * l;
    a.jac = jvals<T>(L);
    a.prp = L.P.rp;
    a.pcol = L.P.col;
    a.pv = mvals<T>(L.P);
    a.b = b;
    for (int k = 0; k < kWfBufs; ++k) a.v[k] = reinterpret_cast<T *>(L.wf_buf + static_cast<size_t>(k) * L.n);
    a.err = c->dflag + 1;
    return ch;
}

// Launch an assembled chain; returns false (nothing launched) if it does
// not fit the kernel's pass or buffer limits.
template <class T>
static bool wf_launch(amg_ctx *c, int l, WfChain<T> &ch, cudaStream_t s) {
    DevLevel &L = c->lev[l];
    if (!ch.ok || ch.a.nphase < 1) return false;
    const int P = ch.a.nphase;
    ch.a.lag = L.wf_lag[P];
    // counters of the chains of 1 .. P-1 passes come first: P (P - 1) / 2 groups' worth
    ch.a.count = L.wf_count + static_cast<size_t>(P * (P - 1) / 2) * L.wf_ngroup;
    ch.a.ctrl = L.wf_ctrl + 4 * P;
    const bool fly = std::is_same<T, float>::value && !c->q_nodes;
    const int grid = std::max(1, L.wf_grid);
    switch (L.A.tpr) {
        case 1: WfLaunch<T>::template go<1>(ch.a, grid, fly, s); break;
        case 2: WfLaunch<T>::template go<2>(ch.a, grid, fly, s); break;
        default: WfLaunch<T>::template go<4>(ch.a, grid, fly, s); break;
    }
    return true;
}

// Chains exist for the pseudo-inverse and Jacobi smoothers with at least one
// sweep per phase and passes that fit the kernel.
static bool wf_usable(const amg_ctx *c, const DevLevel &L) {
    if (!L.wf || c->smoother == AMG_SMOOTHER_CHEB || c->opt.nu1 < 1 || c->opt.nu2 < 1) return false;
    const bool gnn = (c->smoother == AMG_SMOOTHER_GNN);
    const int pre = gnn ? 2 * c->opt.nu1 : c->opt.nu1;          // sweeps + residual
    const int post = gnn ? 1 + 2 * c->opt.nu2 : 1 + c->opt.nu2;  // prolongation + sweeps
    return std::max(pre, post) <= kWfMaxPhases;
}

// Pre-smoothing from zero and the residual for restriction as one chain;
// returns the buffer indices of the smoothed u and of r = b - A u.
template <class T>
static bool wf_pre(amg_ctx *c, int l, cudaStream_t s, const T *b, int &u_idx, int &r_idx) {
    WfChain<T> ch = wf_chain_for<T>(c, l, b);
    const int nu1 = c->opt.nu1;
    int u;
    if (c->smoother == AMG_SMOOTHER_GNN) {
        u = ch.add(kWfQB);
        for (int k = 1; k < nu1; ++k) {
            const int r = ch.add(kWfResid, u);
            u = ch.add(kWfQApply, r, u);
        }
    } else if (nu1 >= 2) {
        u = ch.add(kWfJac12);
        for (int k = 2; k < nu1; ++k) u = ch.add(kWfJac, u);
    } else {
        u = ch.add(kWfJacZ);
    }
    const int r = ch.add(kWfResid, u);
    u_idx = u;
    r_idx = r;
    return wf_launch<T>(c, l, ch, s);
}

// Prolongation-correction u += P e and the post-smoothing as one chain;
// returns the smoothed u.
template <class T>
static T *wf_post(amg_ctx *c, int l, cudaStream_t s, const T *b, int u_idx, const T *e) {
    WfChain<T> ch = wf_chain_for<T>(c, l, b);
    ch.a.e = e;
    ch.taken |= 1u << u_idx;
    int u = ch.add(kWfProlong, u_idx);
    for (int k = 0; k < c->opt.nu2; ++k) {
        if (c->smoother == AMG_SMOOTHER_GNN) {
            const int r = ch.add(kWfResid, u);
            u = ch.add(kWfQApply, r, u);
        } else {
            u = ch.add(kWfJac, u);
        }
    }
    if (!wf_launch<T>(c, l, ch, s)) return nullptr;
    return ch.a.v[u];
}

// nsweeps sweeps from the caller's u (amg_smooth_device); nullptr if the
// chain does not fit.
template <class T>
static T *wf_smooth(amg_ctx *c, int l, cudaStream_t s, const T *b, T *u_in, int nsweeps) {
    WfChain<T> ch = wf_chain_for<T>(c, l, b);
    ch.a.v[kWfBufs] = u_in;
    int u = kWfBufs;
    for (int k = 0; k < nsweeps; ++k) {
        if (c->smoother == AMG_SMOOTHER_GNN) {
            const int r = ch.add(kWfResid, u);
            u = ch.add(kWfQApply, r, u);
        } else {
            u = ch.add(kWfJac, u);
        }
    }
    if (!ch.ok || !wf_launch<T>(c, l, ch, s)) return nullptr;
    return ch.a.v[u];
}

// ---------------------------------------------------------------------------
// V-cycle driver
// ---------------------------------------------------------------------------
// Smoothing sweeps on level l; returns the buffer holding the result (Jacobi
// alternates between cur and alt).
template <class T>
static T *smooth(amg_ctx *c, int l, cudaStream_t s, const T *b, T *cur, T *alt, T *r, int nsweeps,
                 bool zero_init) {
    const DevLevel &L = c->lev[l];
    const bool gnn = (c->smoother == AMG_SMOOTHER_GNN);
    if (nsweeps == 0 && zero_init) cudaMemsetAsync(cur, 0, sizeof(T) * L.n, s);
    if (c->smoother == AMG_SMOOTHER_CHEB) return cheb_smooth<T>(c, L, s, b, cur, alt, nsweeps, zero_init);
    for (int k = 0; k < nsweeps; ++k) {
        const bool first = (k == 0 && zero_init);
        if (gnn) {
            if (first) {
                L_apply<T>(L.A, qvals<T>(L), b, cur, 0, s);
            } else {
                L_resid<T>(L.A, b, cur, r, s);
                L_apply<T>(L.A, qvals<T>(L), r, cur, 1, s);
            }
        } else {
            if (first) {
                launch_pdl(k_scale<T>, dim3(grid_for(L.n)), dim3(kBlock), 0, s, L.n, jvals<T>(L), b, cur);
            } else {
                L_jacobi<T>(L.A, jvals<T>(L), b, cur, alt, s);
                std::swap(cur, alt);
            }
        }
    }
    return cur;
}

// Coarsest solve: one warp with a lane per row when n <= 32, else k_coarse.
template <class T>
__global__ void __launch_bounds__(32) k_coarse_warp(int n, const double *__restrict__ Linv,
                                                    const double *__restrict__ LinvT, const T *__restrict__ b,
                                                    T *__restrict__ u) {
    __shared__ double sb[32], sy[32], sL[32 * 33], sLT[32 * 33];
    const int i = threadIdx.x;
    // the factors are constant: stage them before the grid-dependency wait
    for (int e = i; e < n * n; e += 32) {
        sL[(e / n) * 33 + e % n] = Linv[e];
        sLT[(e / n) * 33 + e % n] = LinvT[e];
    }
    pdl_wait_and_release();
    if (i < n) sb[i] = static_cast<double>(b[i]);
    __syncwarp();
    double y = 0.0;
    if (i < n)
        for (int k = 0; k <= i; ++k) y = fma(sL[i * 33 + k], sb[k], y);
    if (i < n) sy[i] = y;
    __syncwarp();
    double x = 0.0;
    if (i < n)
        for (int k = i; k < n; ++k) x = fma(sLT[i * 33 + k], sy[k], x);
    if (i < n) u[i] = static_cast<T>(x);
}

template <class T>
static void launch_coarse(amg_ctx *c, const T *b, T *u, cudaStream_t s) {
    if (c->nL <= 32) {
        launch_pdl(k_coarse_warp<T>, dim3(1), dim3(32), 0, s, c->nL, c->Linv, c->LinvT, b, u);
    } else {
        launch_pdl(k_coarse<T>, dim3(1), dim3(kBlock), 2 * sizeof(double) * c->nL, s, c->nL, c->Linv, c->LinvT, b, u);
    }
}

// Smoothing on a latency-optimised level: every pseudo-inverse sweep is one
// pass with M A (ping-pong between cur and alt); the first sweep from zero
// also keeps w = M b.  Jacobi fuses its first two sweeps from zero.
template <class T>
static T *smooth_fast(amg_ctx *c, int l, cudaStream_t s, const T *b, T *cur, T *alt, int nsweeps, bool zero_init,
                      bool &have_w) {
    const DevLevel &L = c->lev[l];
    const bool gnn = (c->smoother == AMG_SMOOTHER_GNN);
    T *w = reinterpret_cast<T *>(L.vw);
    if (nsweeps == 0) {
        if (zero_init) cudaMemsetAsync(cur, 0, sizeof(T) * L.n, s);
        return cur;
    }
    if (c->smoother == AMG_SMOOTHER_CHEB) return cheb_smooth<T>(c, L, s, b, cur, alt, nsweeps, zero_init);
    int k = 0;
    if (zero_init) {
        if (gnn) {
            TPR_DISPATCH(L.A.tpr, Launch<T>::template apply_w, L.A, qvals<T>(L), b, cur, w, s);
            have_w = true;
            k = 1;
        } else if (nsweeps >= 2) {
            TPR_DISPATCH(L.A.tpr, Launch<T>::template jacobi_first2, L.A, jvals<T>(L), b, cur, s);
            k = 2;
        } else {
            launch_pdl(k_scale<T>, dim3(grid_for(L.n)), dim3(kBlock), 0, s, L.n, jvals<T>(L), b, cur);
            k = 1;
        }
    }
    if (gnn && !have_w) {
        L_apply<T>(L.A, qvals<T>(L), b, w, 0, s);
        have_w = true;
    }
    for (; k < nsweeps; ++k) {
        if (gnn) {
            TPR_DISPATCH(L.MA.tpr, Launch<T>::template ma_sweep, L.MA, w, cur, alt, s);
        } else {
            L_jacobi<T>(L.A, jvals<T>(L), b, cur, alt, s);
        }
        std::swap(cur, alt);
    }
    return cur;
}

// One V-cycle on level l with right-hand side lev[l].vb; returns the result buffer.
template <class T>
static T *vcycle_level(amg_ctx *c, int l, cudaStream_t s) {
    DevLevel &L = c->lev[l];
    T *b = reinterpret_cast<T *>(L.vb);
    T *u = reinterpret_cast<T *>(L.vu);
    T *r = reinterpret_cast<T *>(L.vr);
    T *t = reinterpret_cast<T *>(L.vt);
    const int nlev = static_cast<int>(c->lev.size());
    if (l == nlev - 1) {
        launch_coarse<T>(c, b, u, s);
        return u;
    }
    T *bc = reinterpret_cast<T *>(c->lev[l + 1].vb);
    // the Chebyshev baseline applies its polynomial once per smoothing phase
    const bool cheb = (c->smoother == AMG_SMOOTHER_CHEB);
    const int nu1 = cheb ? (c->opt.nu1 > 0 ? 1 : 0) : c->opt.nu1;
    const int nu2 = cheb ? (c->opt.nu2 > 0 ? 1 : 0) : c->opt.nu2;
    if (L.fast) {
        bool have_w = false;
        T *cur = smooth_fast<T>(c, l, s, b, u, t, nu1, true, have_w);
        T *alt = (cur == u) ? t : u;
        TPR_DISPATCH(L.RA.tpr, Launch<T>::template resid_restrict, L.R, L.RA, b, cur, bc, s);
        T *ec = vcycle_level<T>(c, l + 1, s);
        L_apply<T>(L.P, mvals<T>(L.P), ec, cur, 1, s);
        return smooth_fast<T>(c, l, s, b, cur, alt, nu2, false, have_w);
    }
    if (wf_usable(c, L)) {
        int ui = 0, ri = 0;
        if (wf_pre<T>(c, l, s, b, ui, ri)) {
            WfChain<T> view = wf_chain_for<T>(c, l, b);
            L_spmv<T>(L.R, view.a.v[ri], bc, s);
            T *ec = vcycle_level<T>(c, l + 1, s);
            T *res = wf_post<T>(c, l, s, b, ui, ec);
            if (res) return res;
        }
    }
    T *cur = smooth<T>(c, l, s, b, u, t, r, nu1, true);
    T *alt = (cur == u) ? t : u;
    L_resid<T>(L.A, b, cur, r, s);
    L_spmv<T>(L.R, r, bc, s);
    T *ec = vcycle_level<T>(c, l + 1, s);
    L_apply<T>(L.P, mvals<T>(L.P), ec, cur, 1, s);
    return smooth<T>(c, l, s, b, cur, alt, r, nu2, false);
}

static Ell64 ell_of(const amg_ctx *c) {
    Ell64 E;
    E.nslice = c->ell_nslice;
    E.ptr = c->ell_ptr;
    E.row = c->ell_row;
    E.col = c->ell_col;
    E.val = c->ell_val;
    return E;
}

// Blocks of the warp-slice passes: one warp per slice, grid capped like the
// CSR outer passes (one partial-sum slot per block).
static int ell_blocks(const amg_ctx *c) {
    const long long need = (static_cast<long long>(c->ell_nslice) + kBlock / 32 - 1) / (kBlock / 32);
    return static_cast<int>(std::max(1LL, std::min<long long>(need, static_cast<long long>(kNumSMs) * kOuterBlocksPerSM)));
}

// FP64 outer residual r = b - A x with its FP32 copy and norm partials;
// returns the number of partial sums.
template <class T>
static int launch_outer(amg_ctx *c, cudaStream_t s, T *rT, double *r64) {
    if (c->ell_nslice > 0) {
        const int nb = ell_blocks(c);
        launch_pdl(k_outer_ell<T>, dim3(nb), dim3(kBlock), 0, s, ell_of(c), static_cast<const double *>(c->db),
                   static_cast<const double *>(c->dx), rT, c->partials, r64);
        return nb;
    }
    const DevMat &A = c->lev[0].A;
    const int nb = outer_blocks(A);
    L_outer<T>(A, c->db, c->dx, rT, c->partials, nb, s, r64);
    return nb;
}

template <class T>
static void enqueue_outer_residual(amg_ctx *c, cudaStream_t s, int use_cond = 0,
                                   cudaGraphConditionalHandle cond = 0) {
    double *r64 = (c->opt.outer == AMG_OUTER_PCG) ? c->pcg : nullptr;   // CG keeps r in FP64
    const int nb = launch_outer<T>(c, s, reinterpret_cast<T *>(c->lev[0].vb), r64);
    launch_pdl(k_norm_final, dim3(1), dim3(1024), 0, s, c->partials, nb, c->state, c->hist, 1, use_cond, cond);
}

// One conjugate-gradient iteration preconditioned by a V-cycle on r (held in
// FP64 in pcg[0..n) and in the V-cycle precision in lev[0].vb).
template <class T>
static void enqueue_pcg_iteration(amg_ctx *c, cudaStream_t s, int use_cond, cudaGraphConditionalHandle cond) {
    const DevMat &A = c->lev[0].A;
    const int n = c->lev[0].n;
    const int nb = c->ell_nslice > 0 ? ell_blocks(c) : outer_blocks(A);
    double *r = c->pcg, *rprev = r + n, *z = rprev + n, *p = z + n, *q = p + n;
    double *P0 = c->partials, *P1 = P0 + c->n_partials, *P2 = P1 + c->n_partials, *P3 = P2 + c->n_partials;
    T *e = vcycle_level<T>(c, 0, s);
    launch_pdl(k_pcg_dots<T>, dim3(nb), dim3(kBlock), 0, s, n, static_cast<const T *>(e),
               static_cast<const double *>(r), static_cast<const double *>(rprev), z, P0, P1);
    launch_pdl(k_pcg_dir, dim3(nb), dim3(kBlock), 0, s, n, static_cast<const double *>(z), p,
               static_cast<const double *>(P0), static_cast<const double *>(P1), nb, c->state);
    if (c->ell_nslice > 0)
        launch_pdl(k_pcg_spmv_ell, dim3(nb), dim3(kBlock), 0, s, ell_of(c), static_cast<const double *>(p), q, P2);
    else
        TPR_DISPATCH(A.tpr, Launch<T>::template pcg_spmv, A, p, q, P2, nb, s);
    launch_pdl(k_pcg_update<T>, dim3(nb), dim3(kBlock), 0, s, n, c->dx, r, rprev, static_cast<const double *>(p),
               static_cast<const double *>(q), reinterpret_cast<T *>(c->lev[0].vb), static_cast<const double *>(P0),
               static_cast<const double *>(P2), nb, c->state, P3);
    launch_pdl(k_norm_final, dim3(1), dim3(1024), 0, s, static_cast<const double *>(P3), nb, c->state, c->hist, 1,
               use_cond, cond);
}

template <class T>
static void enqueue_init(amg_ctx *c, cudaStream_t s, double tol, int max_iter) {
    const int n0 = c->lev[0].n;
    const int nb = std::min(grid_for(n0), kNumSMs * 8);
    const double stall = (c->smoother == AMG_SMOOTHER_GNN) ? c->stall_ratio : 0.0;
    cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), s);   // wavefront wait flag of this solve
    launch_pdl(k_state_init, dim3(1), dim3(1), 0, s, c->state, tol, max_iter, stall);
    launch_pdl(k_sqnorm_partial, dim3(nb), dim3(kBlock), 0, s, n0, c->db, c->partials);
    launch_pdl(k_norm_final, dim3(1), dim3(1024), 0, s, c->partials, nb, c->state, c->hist, 0, 0, 0);
    enqueue_outer_residual<T>(c, s);
}

template <class T>
static void enqueue_iteration(amg_ctx *c, cudaStream_t s, int use_cond = 0, cudaGraphConditionalHandle cond = 0) {
    if (c->opt.outer == AMG_OUTER_PCG) {
        enqueue_pcg_iteration<T>(c, s, use_cond, cond);
        return;
    }
    T *e = vcycle_level<T>(c, 0, s);
    launch_pdl(k_axpy<T>, dim3(grid_for(c->lev[0].n)), dim3(kBlock), 0, s, c->lev[0].n, c->dx, e);
    enqueue_outer_residual<T>(c, s, use_cond, cond);
}

static void free_graph(SolveGraph &G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = SolveGraph{};
}

// Build (once per hierarchy and smoother) the whole-solve graph.
template <class T>
static int ensure_graph(amg_ctx *c) {
    SolveGraph &G = c->sgraph[c->smoother + 3 * c->opt.outer];
    if (G.exec && G.version == c->hier_version && G.q_nodes == static_cast<int>(c->q_nodes)) return AMG_OK;
    free_graph(G);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    G.graph = g;
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    SolveState *st = c->state;
    void *args[] = {&st, &cond};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void *>(k_set_cond);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t setnode;
    CK(cudaGraphAddKernelNode(&setnode, g, nullptr, 0, &kp));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, g, &setnode, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const long long before = g_launches.load();
    CK(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_iteration<T>(c, c->stream, 1, cond);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &captured);
    G.body_kernels = g_launches.load() - before;
    g_launches.fetch_sub(G.body_kernels);
    CK(e);
    CK(cudaGraphInstantiate(&G.exec, g, 0));
    G.version = c->hier_version;
    G.q_nodes = static_cast<int>(c->q_nodes);
    return AMG_OK;
}

// Solve on the staging buffers c->db / c->dx.
template <class T>
static int solve_staged(amg_ctx *c, cudaStream_t s, double tol, int *n_vc, double *hist) {
    const int max_iter = c->opt.max_iter;
    int rc = ensure_graph<T>(c);
    if (rc) return rc;
    enqueue_init<T>(c, s, tol, max_iter);
    CKL("solve init launch");
    const SolveGraph &G = c->sgraph[c->smoother + 3 * c->opt.outer];
    CK(cudaGraphLaunch(G.exec, s));
    CK(cudaMemcpyAsync(c->h_state, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int nh = c->h_state->k;
    g_launches.fetch_add(1 + static_cast<long long>(nh - 1) * G.body_kernels);
    c->last_rerouted = 0;
    if (c->h_state->status == kStalled) {
        // the learned smoother stopped converging: reroute to Jacobi and go on
        // from the current iterate (Sec. 3.3 fallback)
        c->smoother = AMG_SMOOTHER_JACOBI;
        c->last_rerouted = 1;
        rc = ensure_graph<T>(c);
        if (rc) return rc;
        launch_pdl(k_state_continue, dim3(1), dim3(1), 0, s, c->state);
        const SolveGraph &GJ = c->sgraph[AMG_SMOOTHER_JACOBI + 3 * c->opt.outer];
        CK(cudaGraphLaunch(GJ.exec, s));
        CK(cudaMemcpyAsync(c->h_state, c->state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        g_launches.fetch_add(1 + static_cast<long long>(c->h_state->k - nh) * GJ.body_kernels);
        nh = c->h_state->k;
    }
    if (n_vc) *n_vc = nh - 1;
    if (hist) CK(cudaMemcpyAsync(hist, c->hist, sizeof(double) * nh, cudaMemcpyDeviceToHost, s));
    int wferr = 0;
    CK(cudaMemcpyAsync(&wferr, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (wferr) {
        ctx_fail(c, "a wavefront smoothing kernel gave up waiting for a dependency (bounded wait ran out)");
        return AMG_ERR_DEVICE_FLAG;
    }
    return c->h_state->status;
}

// ---------------------------------------------------------------------------
// hierarchy upload
// ---------------------------------------------------------------------------
static const int kMaxCoarseDense = 4096;

static void free_graph(SolveGraph &G);

static void free_device(amg_ctx *c) {
    c->ell_nslice = 0;   // the slices live in the arena
    c->ell_ptr = c->ell_row = c->ell_col = nullptr;
    c->ell_val = nullptr;
    train_bufs_free(c);
    for (auto &G : c->sgraph) free_graph(G);
    if (c->arena) cudaFree(c->arena);
    c->arena = nullptr;
    c->arena_bytes = 0;
    c->lev.clear();
    c->nL = 0;
    c->have_q = false;
}

static void layout_mat(Planner &pl, DevMat &m, const HostCSR &h) {
    m.nr = h.n_rows;
    m.nc = h.n_cols;
    m.nnz = static_cast<int>(h.nnz());
    m.tpr = pick_tpr(h.nnz(), h.n_rows);
    m.rp = pl.take<int>(h.n_rows + 1);
    m.col = pl.take<int>(std::max<long long>(1, h.nnz()));
    m.v64 = pl.take<double>(std::max<long long>(1, h.nnz()));
    m.v32 = pl.take<float>(std::max<long long>(1, h.nnz()));
}

// Warp slices of the finest level's FP64 operator (see Ell64): rows sorted
// by length, longest first, within windows of kEllWindow rows (stable, so
// equal lengths keep their order: a counting sort per window), the slice
// widths and offsets; k_ell_fill then copies the entries on the device.
static void build_ell(amg_ctx *c) {
    const HostCSR &A = c->host[0].A;
    const int n = A.n_rows;
    const int nslice = (n + 31) / 32;
    std::vector<int> rows(static_cast<size_t>(nslice) * 32, -1);
    std::vector<int> start;
    for (int w0 = 0; w0 < n; w0 += kEllWindow) {
        const int w1 = std::min(n, w0 + kEllWindow);
        int maxlen = 0;
        for (int i = w0; i < w1; ++i) maxlen = std::max(maxlen, A.rp[i + 1] - A.rp[i]);
        // bucket of length len starts after all longer rows of the window
        start.assign(static_cast<size_t>(maxlen) + 2, 0);
        for (int i = w0; i < w1; ++i) ++start[maxlen - (A.rp[i + 1] - A.rp[i]) + 1];
        for (int k = 1; k <= maxlen + 1; ++k) start[k] += start[k - 1];
        for (int i = w0; i < w1; ++i) rows[w0 + start[maxlen - (A.rp[i + 1] - A.rp[i])]++] = i;
    }
    c->h_ell_ptr.assign(nslice + 1, 0);
    for (int sl = 0; sl < nslice; ++sl) {
        int w = 0;
        for (int l = 0; l < 32; ++l) {
            const int r = rows[32 * sl + l];
            if (r >= 0) w = std::max(w, A.rp[r + 1] - A.rp[r]);
        }
        c->h_ell_ptr[sl + 1] = c->h_ell_ptr[sl] + 32 * w;
    }
    c->ell_entries = static_cast<long long>(c->h_ell_ptr[nslice]);
    c->h_ell_row.swap(rows);
    c->ell_nslice = nslice;
}

static void layout(amg_ctx *c, Planner &pl) {
    const int nlev = static_cast<int>(c->host.size());
    c->lev.assign(nlev, DevLevel{});
    for (int l = 0; l < nlev; ++l) {
        DevLevel &L = c->lev[l];
        const HostLevel &H = c->host[l];
        L.n = H.A.n_rows;
        layout_mat(pl, L.A, H.A);
        if (l < nlev - 1) {
            layout_mat(pl, L.P, H.P);
            layout_mat(pl, L.R, H.R);
            // 16-bit column offsets for the two-pass (HBM-sized) levels; dropped
            // after the upload if some offset does not fit
            if (!H.fast) L.A.dcol = pl.take<short>(std::max(1, L.A.nnz));
        }
        L.diag = pl.take<double>(L.n);
        L.bx = pl.take<double>(std::max(1, L.A.nnz));
        L.isd = pl.take<unsigned char>(std::max(1, L.A.nnz));
        L.bw = pl.take<double>(std::max(1, L.A.nnz));
        L.bx32 = pl.take<float>(std::max(1, L.A.nnz));
        L.bw32 = pl.take<float>(std::max(1, L.A.nnz));
        L.q64 = pl.take<double>(std::max(1, L.A.nnz));
        L.q32 = pl.take<float>(std::max(1, L.A.nnz));
        L.j64 = pl.take<double>(L.n);
        L.j32 = pl.take<float>(L.n);
        L.dinv64 = pl.take<double>(L.n);
        L.dinv32 = pl.take<float>(L.n);
        L.fast = H.fast;
        if (H.fast) {
            layout_mat(pl, L.MA, H.MA);
            layout_mat(pl, L.RA, H.RA);
            L.pp = pl.take<int>(H.pair_ptr.size());
            L.pq_p = pl.take<int>(std::max<size_t>(1, H.pair_p.size()));
            L.pq_q = pl.take<int>(std::max<size_t>(1, H.pair_q.size()));
        }
        const WfPlan &W = c->wfplan[l];
        L.wf = W.on;
        if (W.on) {
            L.wf_rpt = W.rpt;
            L.wf_nblk = W.nblk;
            L.wf_ngroup = W.ngroup;
            L.wf_grid = W.grid;
            std::copy(W.lag, W.lag + 9, L.wf_lag);
            L.wf_lohi = pl.take<int>(W.lohi.size());
            // counters of every chain length 1..8: (1 + 2 + ... + 8) x ngroup
            L.wf_count = pl.take<unsigned>(static_cast<size_t>(kWfMaxPhases * (kWfMaxPhases + 1) / 2) * W.ngroup);
            L.wf_ctrl = pl.take<unsigned>(4 * (kWfMaxPhases + 1));
            L.wf_buf = pl.take<double>(static_cast<size_t>(kWfBufs) * L.n);
            L.diag32 = pl.take<float>(L.n);
        }
        L.vw = pl.take<double>(L.n);
        L.vb = pl.take<double>(L.n);
        L.vu = pl.take<double>(L.n);
        L.vr = pl.take<double>(L.n);
        L.vt = pl.take<double>(L.n);
    }
    const int nL = c->host.back().A.n_rows;
    c->nL = nL;
    c->Ldense = pl.take<double>(static_cast<size_t>(nL) * nL);
    c->Linv = pl.take<double>(static_cast<size_t>(nL) * nL);
    c->LinvT = pl.take<double>(static_cast<size_t>(nL) * nL);
    const int n0 = c->host[0].A.n_rows;
    c->ell_ptr = pl.take<int>(c->h_ell_ptr.size());
    c->ell_row = pl.take<int>(c->h_ell_row.size());
    c->ell_col = pl.take<int>(std::max(1LL, c->ell_entries));
    c->ell_val = pl.take<double>(std::max(1LL, c->ell_entries));
    c->db = pl.take<double>(n0);
    c->dx = pl.take<double>(n0);
    c->pcg = pl.take<double>(5 * static_cast<size_t>(n0));
    c->n_partials = kNumSMs * kOuterBlocksPerSM;        // blocks of a capped grid
    c->partials = pl.take<double>(5 * c->n_partials);  // up to 5 partial sums per block
    c->scal = pl.take<double>(nlev);
    c->wcoef = pl.take<float>(8 * static_cast<size_t>(nlev));
    c->state = pl.take<SolveState>(1);
    c->hist = pl.take<double>(c->opt.max_iter + 1);
    c->dflag = pl.take<int>(4);
    c->dcol_flag = pl.take<int>(nlev);
}

// from the host, or device to device for a level built on the device
static int upload_mat(amg_ctx *c, const DevMat &m, const HostCSR &h, cudaStream_t s) {
    const bool dev = h.on_device();
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(m.rp, dev ? h.drp : h.rp.data(), sizeof(int) * (h.n_rows + 1), kind, s));
    if (h.nnz() > 0) {
        CK(cudaMemcpyAsync(m.col, dev ? h.dcol : h.col.data(), sizeof(int) * h.nnz(), kind, s));
        CK(cudaMemcpyAsync(m.v64, dev ? h.dval : h.val.data(), sizeof(double) * h.nnz(), kind, s));
        launch_pdl(k_convert<double, float>, dim3(grid_for(h.nnz())), dim3(kBlock), 0, s, m.nnz, m.v64, m.v32);
    }
    return AMG_OK;
}

// Levels whose M A pair list stays small are latency-bound at any size this
// library meets (their working set sits in the 129 MB L2): they take the
// single-pass sweeps and the fused residual + restriction.
static const long long kFastPairs = 8LL << 20;

static int plan_fast_levels(amg_ctx *c) {
    const int nlev = static_cast<int>(c->host.size());
    std::vector<char> which(nlev, 0);
    for (int l = 0; l < nlev; ++l) {
        HostLevel &H = c->host[l];
        H.fast = false;
        H.MA = HostCSR{};
        H.RA = HostCSR{};
        H.pair_ptr.clear();
        H.pair_p.clear();
        H.pair_q.clear();
        if (l == nlev - 1) continue;
        long long pairs = 0;
        for (int k = 0; k < H.A.n_rows; ++k) {
            const long long d = H.A.rp[k + 1] - H.A.rp[k];
            pairs += d * d;
        }
        if (pairs > kFastPairs) continue;
        which[l] = 1;
        H.fast = true;
    }
    // M A pattern + pair list and R A, built on the device
    std::string why;
    const int rc = device_plan_products(c->host, which, c->stream, why);
    if (rc) ctx_fail(c, why);
    return rc;
}

static int upload(amg_ctx *c) {
    free_device(c);
    ++c->hier_version;
    c->stall_ratio = 0.0;   // the in-solve check belongs to a mesh
    int prc = plan_fast_levels(c);
    if (prc) return prc;
    prc = plan_wavefront(c);
    if (prc) return prc;
    build_ell(c);
    c->q_nodes = false;
    Planner pl;
    layout(c, pl);
    c->arena_bytes = pl.off;
    CK(cudaMalloc(&c->arena, c->arena_bytes));
    pl = Planner{};
    pl.base = c->arena;
    layout(c, pl);
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->arena, 0, c->arena_bytes, s));
    const int nlev = static_cast<int>(c->host.size());
    c->scales.assign(nlev, 1.0);
    for (int l = 0; l < nlev; ++l) {
        DevLevel &L = c->lev[l];
        const HostLevel &H = c->host[l];
        int rc = upload_mat(c, L.A, H.A, s);
        if (rc) return rc;
        if (L.A.dcol && L.A.nnz > 0) {
            k_col_delta<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.A.rp, L.A.col, L.A.dcol, c->dcol_flag + l); AMG_COUNT();
        }
        if (l < nlev - 1) {
            if ((rc = upload_mat(c, L.P, H.P, s))) return rc;
            if ((rc = upload_mat(c, L.R, H.R, s))) return rc;
        }
        if (L.fast) {
            if ((rc = upload_mat(c, L.MA, H.MA, s))) return rc;
            if ((rc = upload_mat(c, L.RA, H.RA, s))) return rc;
            CK(cudaMemcpyAsync(L.pp, H.pair_ptr.data(), sizeof(int) * H.pair_ptr.size(), cudaMemcpyHostToDevice, s));
            if (!H.pair_p.empty()) {
                CK(cudaMemcpyAsync(L.pq_p, H.pair_p.data(), sizeof(int) * H.pair_p.size(), cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(L.pq_q, H.pair_q.data(), sizeof(int) * H.pair_q.size(), cudaMemcpyHostToDevice, s));
            }
        }
        k_extract_diag<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.A.rp, L.A.col, L.A.v64, L.diag); AMG_COUNT();
        if (L.wf) {
            const WfPlan &W = c->wfplan[l];
            CK(cudaMemcpyAsync(L.wf_lohi, W.lohi.data(), sizeof(int) * W.lohi.size(), cudaMemcpyHostToDevice, s));
            launch_pdl(k_convert<double, float>, dim3(grid_for(L.n)), dim3(kBlock), 0, s, L.n,
                       static_cast<const double *>(L.diag), L.diag32);
        }
        const int nb = std::min(grid_for(L.n), kNumSMs * 8);
        k_offdiag_absmax<<<nb, kBlock, 0, s>>>(L.n, L.A.rp, L.A.col, L.A.v64, c->partials); AMG_COUNT();
        k_max_final<<<1, 32, 0, s>>>(c->partials, nb, c->scal + l); AMG_COUNT();
        k_jacobi_vals<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.diag, c->opt.omega, L.j64, L.j32); AMG_COUNT();
        k_dinv_vals<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.diag, L.dinv64, L.dinv32); AMG_COUNT();
        k_pinv_basis<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.A.rp, L.A.col, L.A.v64, L.diag, c->scal + l, L.bx,
                                                      L.bw, L.isd, L.bx32, L.bw32); AMG_COUNT();
    }
    c->jac_omega = c->opt.omega;
    CK(cudaMemcpyAsync(c->ell_ptr, c->h_ell_ptr.data(), sizeof(int) * c->h_ell_ptr.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->ell_row, c->h_ell_row.data(), sizeof(int) * c->h_ell_row.size(), cudaMemcpyHostToDevice, s));
    {
        const DevMat &A0 = c->lev[0].A;
        k_ell_fill<<<grid_for(32LL * c->ell_nslice), kBlock, 0, s>>>(c->ell_nslice, c->ell_ptr, c->ell_row, A0.rp,
                                                                      A0.col, A0.v64, c->ell_col, c->ell_val); AMG_COUNT();
    }
    // coarsest level: dense FP64 Cholesky and the inverse factor
    const DevLevel &Lc = c->lev.back();
    const int nL = c->nL;
    k_csr_to_dense<<<grid_for(nL), kBlock, 0, s>>>(nL, Lc.A.rp, Lc.A.col, Lc.A.v64, c->Ldense); AMG_COUNT();
    k_cholesky<<<1, 1024, 0, s>>>(nL, c->Ldense, c->dflag); AMG_COUNT();
    CK(cudaFuncSetAttribute(k_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8 * kMaxCoarseDense));
    CK(cudaFuncSetAttribute(k_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 8 * kMaxCoarseDense));
    k_tri_inverse<<<grid_for(nL), kBlock, 0, s>>>(nL, c->Ldense, c->Linv, c->LinvT); AMG_COUNT();
    CKL("hierarchy setup kernels");
    int flag = 0;
    std::vector<int> wide(nlev, 0);
    CK(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->scales.data(), c->scal, sizeof(double) * nlev, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(wide.data(), c->dcol_flag, sizeof(int) * nlev, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int l = 0; l < nlev; ++l)
        if (wide[l]) c->lev[l].A.dcol = nullptr;    // an offset past 16 bits: full indices
    c->h_ell_row = std::vector<int>();    // copied: the host row order is not kept
    if (flag) {
        c->err = "coarsest-level matrix is not positive definite";
        free_device(c);
        return AMG_ERR_NOT_SPD;
    }
    // device-built levels now live in the arena: later host copies come from there
    for (int l = 0; l < nlev; ++l) {
        HostLevel &H = c->host[l];
        const DevLevel &L = c->lev[l];
        const std::pair<HostCSR *, const DevMat *> mats[3] = {{&H.A, &L.A}, {&H.P, &L.P}, {&H.R, &L.R}};
        for (const auto &hm : mats) {
            if (!hm.first->on_device()) continue;
            hm.first->drp = hm.second->rp;
            hm.first->dcol = hm.second->col;
            hm.first->dval = hm.second->v64;
        }
    }
    c->smoother = AMG_SMOOTHER_JACOBI;
    return AMG_OK;
}

static bool to_host(const amg_csr *m, HostCSR &h, std::string &why) {
    if (!m || !m->row_ptr || (m->nnz > 0 && (!m->col || !m->val)) || m->n_rows < 0 || m->n_cols < 0 ||
        m->nnz < 0 || m->nnz > 2000000000LL) {
        why = "null or invalid CSR";
        return false;
    }
    h.n_rows = m->n_rows;
    h.n_cols = m->n_cols;
    h.rp.assign(m->row_ptr, m->row_ptr + m->n_rows + 1);
    if (h.rp.back() != m->nnz) {
        why = "row_ptr[n] != nnz";
        return false;
    }
    h.col.assign(m->col, m->col + m->nnz);
    h.val.assign(m->val, m->val + m->nnz);
    return true;
}


// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void amg_default_options(amg_options *o) {
    if (!o) return;
    o->nu1 = 2;
    o->nu2 = 2;
    o->max_levels = 10;
    o->max_coarse = 64;
    o->max_iter = 500;
    o->precision = AMG_FP32_IN_FP64;
    o->smoother = AMG_SMOOTHER_JACOBI;
    o->omega = 2.0 / 3.0;
    o->theta = 0.25;
    o->device = 0;
    o->gnn_precision = AMG_GNN_BF16;
    o->outer = AMG_OUTER_REFINE;
    o->fused_sweeps = 0;
}

int amg_create(amg_ctx **ctx, const amg_options *opt) {
    if (!ctx) {
        g_create_err = "ctx is NULL";
        return AMG_ERR_ARG;
    }
    *ctx = nullptr;
    amg_options o;
    amg_default_options(&o);
    if (opt) o = *opt;
    if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 64 || o.nu2 > 64 || o.max_levels < 1 || o.max_levels > 32 ||
        o.max_coarse < 1 || o.max_iter < 0 || o.max_iter > 100000 ||
        (o.precision != AMG_FP64 && o.precision != AMG_FP32_IN_FP64) ||
        (o.smoother != AMG_SMOOTHER_JACOBI && o.smoother != AMG_SMOOTHER_GNN) || !(o.theta >= 0.0) ||
        (o.gnn_precision != AMG_GNN_FP32 && o.gnn_precision != AMG_GNN_BF16) ||
        (o.outer != AMG_OUTER_REFINE && o.outer != AMG_OUTER_PCG) || (o.fused_sweeps != 0 && o.fused_sweeps != 1) ||
        !(o.theta <= 1.0) || !std::isfinite(o.omega)) {
        g_create_err = "invalid amg_options";
        return AMG_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
        g_create_err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return AMG_ERR_CUDA;
    }
    amg_ctx *c = new (std::nothrow) amg_ctx();
    if (!c) {
        g_create_err = "out of host memory";
        return AMG_ERR_ARG;
    }
    c->opt = o;
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_state, sizeof(SolveState));
    if (e != cudaSuccess) {
        g_create_err = std::string("stream/pinned allocation: ") + cudaGetErrorString(e);
        if (c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return AMG_ERR_CUDA;
    }
    g_create_err.clear();
    *ctx = c;
    return AMG_OK;
}

void amg_destroy(amg_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->opt.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gnn) gcin_engine_free(c->gnn);
    free_device(c);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *amg_last_error(const amg_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int amg_load_hierarchy(amg_ctx *c, int n_levels, const amg_csr *A, const amg_csr *P, const amg_csr *R) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (n_levels < 1 || !A || (n_levels > 1 && !P)) return ctx_fail(c, "bad n_levels or NULL arrays"), AMG_ERR_ARG;
    std::vector<HostLevel> h(n_levels);
    std::string why;
    for (int l = 0; l < n_levels; ++l) {
        if (!to_host(&A[l], h[l].A, why) || !validate_csr(h[l].A, true, why))
            return ctx_fail(c, "A[" + std::to_string(l) + "]: " + why), AMG_ERR_ARG;
        if (l < n_levels - 1) {
            if (!to_host(&P[l], h[l].P, why) || !validate_csr(h[l].P, false, why))
                return ctx_fail(c, "P[" + std::to_string(l) + "]: " + why), AMG_ERR_ARG;
            if (R) {
                if (!to_host(&R[l], h[l].R, why) || !validate_csr(h[l].R, false, why))
                    return ctx_fail(c, "R[" + std::to_string(l) + "]: " + why), AMG_ERR_ARG;
            } else {
                h[l].R = transpose(h[l].P);
            }
        }
    }
    for (int l = 0; l + 1 < n_levels; ++l) {
        const int n = h[l].A.n_rows, nc = h[l + 1].A.n_rows;
        if (h[l].P.n_rows != n || h[l].P.n_cols != nc || h[l].R.n_rows != nc || h[l].R.n_cols != n)
            return ctx_fail(c, "P/R dimensions disagree with A at level " + std::to_string(l)), AMG_ERR_ARG;
    }
    if (h.back().A.n_rows > kMaxCoarseDense)
        return ctx_fail(c, "coarsest level larger than 4096 rows: dense Cholesky refused"), AMG_ERR_ARG;
    if (h[0].A.n_rows < 1) return ctx_fail(c, "empty matrix"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    c->host = std::move(h);
    return upload(c);
}

int amg_setup(amg_ctx *c, const amg_csr *A) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    HostCSR h;
    std::string why;
    if (!to_host(A, h, why) || !validate_csr(h, true, why)) return ctx_fail(c, "A: " + why), AMG_ERR_ARG;
    if (h.n_rows < 1) return ctx_fail(c, "empty matrix"), AMG_ERR_ARG;
    std::vector<HostLevel> levels;
    build_hierarchy(h, c->opt.theta, c->opt.max_levels, c->opt.max_coarse, levels);
    if (levels.back().A.n_rows > kMaxCoarseDense)
        return ctx_fail(c, "coarsening stalled above 4096 rows: dense Cholesky refused"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    c->host = std::move(levels);
    return upload(c);
}

int amg_setup_device(amg_ctx *c, const amg_csr *A, unsigned long long seed, int split) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (split < 0 || split > (AMG_SPLIT_SECOND_PASS | AMG_SPLIT_RS_BLOCKS))
        return ctx_fail(c, "unknown split"), AMG_ERR_ARG;
    HostCSR h;
    std::string why;
    if (!to_host(A, h, why) || !validate_csr(h, true, why)) return ctx_fail(c, "A: " + why), AMG_ERR_ARG;
    if (h.n_rows < 1) return ctx_fail(c, "empty matrix"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    std::vector<HostLevel> levels;
    std::shared_ptr<void> built;   // the levels' device memory until the upload has copied them
    const int rc = device_build_hierarchy(h, c->opt.theta, c->opt.max_levels, c->opt.max_coarse, seed, split,
                                          c->stream, levels, built, why);
    if (rc) return ctx_fail(c, why), rc;
    if (levels.back().A.n_rows > kMaxCoarseDense)
        return ctx_fail(c, "coarsening stalled above 4096 rows: dense Cholesky refused"), AMG_ERR_ARG;
    levels[0].A = std::move(h);    // the input's host copy stands for level 0
    c->host = std::move(levels);
    const int urc = upload(c);     // device to device; the host copies of the coarse levels come on demand
    if (urc) c->host.clear();      // their device memory goes with `built`
    return urc;
}

int amg_num_levels(const amg_ctx *c) { return c ? static_cast<int>(c->lev.size()) : 0; }

int amg_level_info(const amg_ctx *c, int level, int *n, long long *nnz_A, long long *nnz_P) {
    if (!c || level < 0 || level >= static_cast<int>(c->host.size())) return AMG_ERR_ARG;
    const HostLevel &H = c->host[level];
    if (n) *n = H.A.n_rows;
    if (nnz_A) *nnz_A = H.A.nnz();
    if (nnz_P) *nnz_P = (level + 1 < static_cast<int>(c->host.size())) ? H.P.nnz() : 0;
    return AMG_OK;
}

int amg_get_level(const amg_ctx *cc, int level, int *A_rp, int *A_col, double *A_val, int *P_rp, int *P_col,
                  double *P_val) {
    amg_ctx *c = const_cast<amg_ctx *>(cc);
    if (!c || level < 0 || level >= static_cast<int>(c->host.size())) return AMG_ERR_ARG;
    const int hrc = ensure_host(c, level);
    if (hrc) return hrc;
    const HostLevel &H = c->host[level];
    if (!A_rp || !A_col || !A_val) return AMG_ERR_ARG;
    std::copy(H.A.rp.begin(), H.A.rp.end(), A_rp);
    std::copy(H.A.col.begin(), H.A.col.end(), A_col);
    std::copy(H.A.val.begin(), H.A.val.end(), A_val);
    if (level + 1 < static_cast<int>(c->host.size()) && P_rp && P_col && P_val) {
        std::copy(H.P.rp.begin(), H.P.rp.end(), P_rp);
        std::copy(H.P.col.begin(), H.P.col.end(), P_col);
        std::copy(H.P.val.begin(), H.P.val.end(), P_val);
    }
    return AMG_OK;
}

int amg_get_scales(const amg_ctx *c, double *s_out) {
    if (!c || !s_out) return AMG_ERR_ARG;
    if (c->lev.empty()) return AMG_ERR_STATE;
    std::copy(c->scales.begin(), c->scales.end(), s_out);
    return AMG_OK;
}

int amg_set_jacobi(amg_ctx *c, double omega) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!std::isfinite(omega)) return ctx_fail(c, "omega not finite"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    if (omega != c->jac_omega) {
        for (auto &L : c->lev) {
            k_jacobi_vals<<<grid_for(L.n), kBlock, 0, c->stream>>>(L.n, L.diag, omega, L.j64, L.j32); AMG_COUNT();
        }
        CKL("jacobi values");
        CK(cudaStreamSynchronize(c->stream));
        c->jac_omega = omega;
    }
    c->smoother = AMG_SMOOTHER_JACOBI;
    return AMG_OK;
}

int amg_set_chebyshev(amg_ctx *c, int degree) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (degree < 1 || degree > 16) return ctx_fail(c, "Chebyshev degree outside 1..16"), AMG_ERR_ARG;
    if (c->cheb_version != c->hier_version) {
        const int nlev = static_cast<int>(c->lev.size());
        for (int l = 0; l < nlev - 1; ++l) {
            DevLevel &L = c->lev[l];
            const int hrc = ensure_host(c, l);
            if (hrc) return hrc;
            const double rho = power_estimate(c->host[l].A, 20);
            if (!(rho > 0.0) || !std::isfinite(rho)) return ctx_fail(c, "power estimate failed"), AMG_ERR_ARG;
            const double lo = rho / 30.0, hi = 1.1 * rho;
            L.cheb_rho = rho;
            L.cheb_theta = 0.5 * (hi + lo);
            L.cheb_delta = 0.5 * (hi - lo);
        }
        c->cheb_version = c->hier_version;
    }
    if (degree != c->cheb_degree) {   // the captured graphs hold the polynomial's steps
        for (int o = 0; o < 2; ++o) free_graph(c->sgraph[AMG_SMOOTHER_CHEB + 3 * o]);
        c->cheb_degree = degree;
    }
    c->smoother = AMG_SMOOTHER_CHEB;
    return AMG_OK;
}

int amg_get_chebyshev(const amg_ctx *c, int level, double *rho, double *theta, double *delta) {
    if (!c || level < 0 || level >= static_cast<int>(c->lev.size()) - 1) return AMG_ERR_ARG;
    if (c->cheb_version != c->hier_version) return AMG_ERR_STATE;
    const DevLevel &L = c->lev[level];
    if (rho) *rho = L.cheb_rho;
    if (theta) *theta = L.cheb_theta;
    if (delta) *delta = L.cheb_delta;
    return AMG_OK;
}
}  // extern "C"

namespace amg {
// Enqueue the assembly of Q^-1 (and M A on latency-optimised levels) from
// coefficients in device memory (G x 5 FP32, level order) without a host
// round trip; the caller validates the coefficients after its own
// synchronisation and selects the smoother.
static AsmQ asm_q_levels(const amg_ctx *c) {
    AsmQ Q{};
    for (int l = 0; l + 1 < static_cast<int>(c->lev.size()); ++l) {
        const DevLevel &L = c->lev[l];
        const int k = Q.nlev++;
        Q.start[k + 1] = Q.start[k] + L.A.nnz;
        Q.isd[k] = L.isd;
        Q.bx[k] = L.bx;
        Q.bw[k] = L.bw;
        Q.bx32[k] = L.bx32;
        Q.bw32[k] = L.bw32;
        Q.q64[k] = L.q64;
        Q.q32[k] = L.q32;
        Q.row[k] = l;
    }
    return Q;
}

int enqueue_coeff_assembly(amg_ctx *c, const float *d_coef, cudaStream_t s) {
    const int nlev = static_cast<int>(c->lev.size());
    if (nlev - 1 > kAsmMaxLevels) return ctx_fail(c, "too many levels for the batched assembly"), AMG_ERR_ARG;
    // all levels' Q^-1 in one launch, then all latency-optimised levels' M A;
    // the FP32 V-cycle needs only the FP32 values (the coefficients stay in
    // wcoef for an FP64 assembly on request)
    const AsmQ Q = asm_q_levels(c);
    const bool fp64 = c->opt.precision == AMG_FP64;
    AsmMA M{};
    for (int l = 0; l < nlev - 1; ++l) {
        const DevLevel &L = c->lev[l];
        if (L.fast) {
            const int j = M.nlev++;
            M.start[j + 1] = M.start[j] + L.MA.nnz;
            M.pp[j] = L.pp;
            M.pq_p[j] = L.pq_p;
            M.pq_q[j] = L.pq_q;
            M.q32[j] = L.q32;
            M.a32[j] = L.A.v32;
            M.ma32[j] = L.MA.v32;
            M.q64[j] = L.q64;
            M.a64[j] = L.A.v64;
            M.ma64[j] = L.MA.v64;
        }
    }
    if (Q.nlev > 0 && Q.start[Q.nlev] > 0) {
        k_assemble_q_all<<<grid_for(Q.start[Q.nlev]), kBlock, 0, s>>>(Q, d_coef, 5, fp64 ? 1 : 0); AMG_COUNT();
    }
    if (M.nlev > 0 && M.start[M.nlev] > 0) {
        k_assemble_ma_all<<<grid_for(M.start[M.nlev]), kBlock, 0, s>>>(M, fp64 ? 1 : 0); AMG_COUNT();
    }
    c->q64_stale = !fp64;
    if (nlev > 1) {
        k_wf_coef<<<1, 32, 0, s>>>(nlev - 1, d_coef, c->scal, c->wcoef); AMG_COUNT();
    }
    CKL("assemble pseudo-inverse");
    return AMG_OK;
}

int set_coeffs_device(amg_ctx *c, const double *coef, int n_rows, cudaStream_t s) {
    const int nlev = static_cast<int>(c->lev.size());
    for (int l = 0; l < nlev - 1; ++l) {
        const DevLevel &L = c->lev[l];
        const double *q = coef + 5 * l;
        for (int k = 0; k < 5; ++k)
            if (!std::isfinite(q[k])) return ctx_fail(c, "non-finite coefficient"), AMG_ERR_ARG;
        k_assemble_q<<<grid_for(L.A.nnz), kBlock, 0, s>>>(L.A.nnz, L.isd, L.bx, L.bw, q[0], q[1], q[2], q[3],
                                                          q[4], L.q64, L.q32); AMG_COUNT();
        if (L.fast && c->opt.precision == AMG_FP64) {
            k_assemble_ma<<<grid_for(L.MA.nnz), kBlock, 0, s>>>(L.MA.nnz, L.pp, L.pq_p, L.pq_q, L.q64, L.A.v64,
                                                                L.MA.v64, L.MA.v32); AMG_COUNT();
        } else if (L.fast) {
            k_assemble_ma32<<<grid_for(L.MA.nnz), kBlock, 0, s>>>(L.MA.nnz, L.pp, L.pq_p, L.pq_q, L.q32, L.A.v32,
                                                                  L.MA.v32); AMG_COUNT();
        }
    }
    (void)n_rows;
    {
        std::vector<float> wc(8 * static_cast<size_t>(nlev), 0.0f);
        for (int l = 0; l < nlev - 1; ++l) {
            for (int k = 0; k < 5; ++k) wc[8 * l + k] = static_cast<float>(coef[5 * l + k]);
            wc[8 * l + 5] = static_cast<float>(1.0 / c->scales[l]);
        }
        CK(cudaMemcpyAsync(c->wcoef, wc.data(), sizeof(float) * wc.size(), cudaMemcpyHostToDevice, s));
        c->q_nodes = false;
        c->q64_stale = false;
    }
    CKL("assemble pseudo-inverse");
    // the solve kernels fetch matrix values ahead of their grid-dependency
    // wait: finish writing them before any of those kernels is launched
    CK(cudaStreamSynchronize(s));
    c->have_q = true;
    c->smoother = AMG_SMOOTHER_GNN;
    return AMG_OK;
}
}  // namespace amg

extern "C" {

int amg_set_coeffs(amg_ctx *c, const double *coef, int n_rows) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!coef || n_rows < static_cast<int>(c->lev.size()) - 1)
        return ctx_fail(c, "need one coefficient row per smoothed level"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    int rc = set_coeffs_device(c, coef, n_rows, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return AMG_OK;
}

int amg_set_node_coeffs(amg_ctx *c, const double *coef, long long n_values) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    const int nlev = static_cast<int>(c->lev.size());
    long long need = 0;
    for (int l = 0; l < nlev - 1; ++l) need += 5LL * c->lev[l].n;
    if (!coef || n_values != need)
        return ctx_fail(c, "need 5 coefficients per node of every smoothed level"), AMG_ERR_ARG;
    for (long long k = 0; k < need; ++k)
        if (!std::isfinite(coef[k])) return ctx_fail(c, "non-finite coefficient"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    cudaStream_t s = c->stream;
    if (need == 0) {
        c->have_q = true;
        c->q_nodes = true;
        c->smoother = AMG_SMOOTHER_GNN;
        return AMG_OK;
    }
    double *d_c = nullptr;
    CK(cudaMalloc(&d_c, sizeof(double) * need));
    cudaError_t e = cudaMemcpyAsync(d_c, coef, sizeof(double) * need, cudaMemcpyHostToDevice, s);
    long long off = 0;
    for (int l = 0; l < nlev - 1 && e == cudaSuccess; ++l) {
        const DevLevel &L = c->lev[l];
        k_assemble_q_nodes<<<grid_for(L.n), kBlock, 0, s>>>(L.n, L.A.rp, L.A.col, L.isd, L.bx, L.bw, d_c + off,
                                                             L.q64, L.q32); AMG_COUNT();
        if (L.fast && c->opt.precision == AMG_FP64) {
            k_assemble_ma<<<grid_for(L.MA.nnz), kBlock, 0, s>>>(L.MA.nnz, L.pp, L.pq_p, L.pq_q, L.q64, L.A.v64,
                                                                L.MA.v64, L.MA.v32); AMG_COUNT();
        } else if (L.fast) {
            k_assemble_ma32<<<grid_for(L.MA.nnz), kBlock, 0, s>>>(L.MA.nnz, L.pp, L.pq_p, L.pq_q, L.q32, L.A.v32,
                                                                  L.MA.v32); AMG_COUNT();
        }
        off += 5LL * L.n;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_c);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "assemble per-node pseudo-inverse");
    c->have_q = true;
    c->q_nodes = true;   // the wavefront chains read the stored values
    c->q64_stale = false;
    c->smoother = AMG_SMOOTHER_GNN;
    return AMG_OK;
}

int amg_get_smoother(const amg_ctx *cc, int level, double *q_out) {
    amg_ctx *c = const_cast<amg_ctx *>(cc);
    if (!c || !q_out || level < 0 || level >= static_cast<int>(c->lev.size()) - 1) return AMG_ERR_ARG;
    const DevLevel &L = c->lev[level];
    CK(cudaSetDevice(c->opt.device));
    if (c->smoother == AMG_SMOOTHER_CHEB) return ctx_fail(c, "the Chebyshev smoother has no explicit Q^-1"), AMG_ERR_STATE;
    if (c->smoother == AMG_SMOOTHER_GNN) {
        if (c->q64_stale) {
            // the network's coefficients were assembled for the FP32 V-cycle
            // only: form the FP64 values from the kept FP32 coefficients
            const AsmQ Q = asm_q_levels(c);
            if (Q.start[Q.nlev] > 0) {
                k_assemble_q_all<<<grid_for(Q.start[Q.nlev]), kBlock, 0, c->stream>>>(Q, c->wcoef, 8, 2); AMG_COUNT();
            }
            CKL("assemble FP64 pseudo-inverse");
            c->q64_stale = false;
        }
        CK(cudaMemcpyAsync(q_out, L.q64, sizeof(double) * L.A.nnz, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<double> j(L.n);
        CK(cudaMemcpyAsync(j.data(), L.j64, sizeof(double) * L.n, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const int hrc = ensure_host(c, level);
        if (hrc) return hrc;
        const HostCSR &A = c->host[level].A;
        for (int i = 0; i < A.n_rows; ++i)
            for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) q_out[p] = (A.col[p] == i) ? j[i] : 0.0;
    }
    return AMG_OK;
}

static int solve_dispatch(amg_ctx *c, cudaStream_t s, double tol, int *n_vc, double *hist) {
    if (c->opt.precision == AMG_FP64) return solve_staged<double>(c, s, tol, n_vc, hist);
    return solve_staged<float>(c, s, tol, n_vc, hist);
}

static int check_ready(amg_ctx *c) {
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (c->smoother == AMG_SMOOTHER_GNN && !c->have_q)
        return ctx_fail(c, "pseudo-inverse smoother selected without coefficients"), AMG_ERR_STATE;
    return AMG_OK;
}

int amg_solve(amg_ctx *c, const double *b, double *x, double rtol, int *n_vc, double *hist) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!b || !x || !(rtol >= 0.0)) return ctx_fail(c, "NULL vector or negative tolerance"), AMG_ERR_ARG;
    int rc = check_ready(c);
    if (rc) return rc;
    CK(cudaSetDevice(c->opt.device));
    const int n0 = c->lev[0].n;
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(c->db, b, sizeof(double) * n0, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->dx, x, sizeof(double) * n0, cudaMemcpyHostToDevice, s));
    rc = solve_dispatch(c, s, rtol, n_vc, hist);
    if (rc == AMG_ERR_CUDA) return rc;
    CK(cudaMemcpyAsync(x, c->dx, sizeof(double) * n0, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (rc != AMG_OK && rc != AMG_ERR_DEVICE_FLAG)
        c->err = "solve ended without reaching the tolerance (status " + std::to_string(rc) + ")";
    else if (c->last_rerouted) c->err = "learned smoother stalled; solve finished with Jacobi (rerouted)";
    return rc;
}

int amg_solve_device(amg_ctx *c, const double *d_b, double *d_x, double rtol, void *stream, int *n_vc,
                     double *hist) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!d_b || !d_x || !(rtol >= 0.0)) return ctx_fail(c, "NULL vector or negative tolerance"), AMG_ERR_ARG;
    int rc = check_ready(c);
    if (rc) return rc;
    CK(cudaSetDevice(c->opt.device));
    const int n0 = c->lev[0].n;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(c->db, d_b, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->dx, d_x, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
    rc = solve_dispatch(c, s, rtol, n_vc, hist);
    if (rc == AMG_ERR_CUDA) return rc;
    CK(cudaMemcpyAsync(d_x, c->dx, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (rc != AMG_OK && rc != AMG_ERR_DEVICE_FLAG)
        c->err = "solve ended without reaching the tolerance (status " + std::to_string(rc) + ")";
    else if (c->last_rerouted) c->err = "learned smoother stalled; solve finished with Jacobi (rerouted)";
    return rc;
}

int amg_vcycle_device(amg_ctx *c, const double *d_r, double *d_e, void *stream) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!d_r || !d_e) return ctx_fail(c, "NULL vector"), AMG_ERR_ARG;
    int rc = check_ready(c);
    if (rc) return rc;
    CK(cudaSetDevice(c->opt.device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n0 = c->lev[0].n;
    if (c->opt.precision == AMG_FP64) {
        CK(cudaMemcpyAsync(c->lev[0].vb, d_r, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
        double *e = vcycle_level<double>(c, 0, s);
        CK(cudaMemcpyAsync(d_e, e, sizeof(double) * n0, cudaMemcpyDeviceToDevice, s));
    } else {
        launch_pdl(k_convert<double, float>, dim3(grid_for(n0)), dim3(kBlock), 0, s, n0, d_r, reinterpret_cast<float *>(c->lev[0].vb));
        float *e = vcycle_level<float>(c, 0, s);
        launch_pdl(k_convert<float, double>, dim3(grid_for(n0)), dim3(kBlock), 0, s, n0, e, d_e);
    }
    CKL("vcycle");
    return AMG_OK;
}

}  // extern "C"

template <class T>
static void smooth_level_device(amg_ctx *c, int l, const double *d_b, double *d_u, int nsw, cudaStream_t s) {
    DevLevel &L = c->lev[l];
    const int n = L.n;
    T *b = reinterpret_cast<T *>(L.vb), *u = reinterpret_cast<T *>(L.vu);
    launch_pdl(k_convert<double, T>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, d_b, b);
    launch_pdl(k_convert<double, T>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, d_u, u);
    T *res = nullptr;
    if (nsw > 0 && L.wf && c->smoother != AMG_SMOOTHER_CHEB) {
        cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), s);
        res = wf_smooth<T>(c, l, s, b, u, nsw);
    }
    if (!res) res = smooth<T>(c, l, s, b, u, reinterpret_cast<T *>(L.vt), reinterpret_cast<T *>(L.vr), nsw, false);
    launch_pdl(k_convert<T, double>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, res, d_u);
}

extern "C" {

int amg_smooth_device(amg_ctx *c, int level, const double *d_b, double *d_u, int n_sweeps, void *stream) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    int rc = check_ready(c);
    if (rc) return rc;
    if (!d_b || !d_u || n_sweeps < 0 || level < 0 || level >= static_cast<int>(c->lev.size()) - 1)
        return ctx_fail(c, "bad level, sweep count or vector"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->opt.precision == AMG_FP64) smooth_level_device<double>(c, level, d_b, d_u, n_sweeps, s);
    else smooth_level_device<float>(c, level, d_b, d_u, n_sweeps, s);
    CKL("smooth");
    return AMG_OK;
}

int amg_spmv_device(amg_ctx *c, int level, const double *d_x, double *d_y, void *stream) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!d_x || !d_y || level < 0 || level >= static_cast<int>(c->lev.size()))
        return ctx_fail(c, "bad level or vector"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevLevel &L = c->lev[level];
    const int n = L.n;
    if (c->opt.precision == AMG_FP64) {
        L_spmv<double>(L.A, d_x, d_y, s);
    } else {
        float *x = reinterpret_cast<float *>(L.vu), *y = reinterpret_cast<float *>(L.vr);
        launch_pdl(k_convert<double, float>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, d_x, x);
        L_spmv<float>(L.A, x, y, s);
        launch_pdl(k_convert<float, double>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, y, d_y);
    }
    CKL("spmv");
    return AMG_OK;
}

int amg_judge(amg_ctx *c, const double *b, int n_cycles, double *metric) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!b || !metric || n_cycles < 1 || n_cycles > 10000) return ctx_fail(c, "bad argument"), AMG_ERR_ARG;
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!c->have_q) return ctx_fail(c, "no pseudo-inverse coefficients set"), AMG_ERR_STATE;
    CK(cudaSetDevice(c->opt.device));
    const int n0 = c->lev[0].n;
    cudaStream_t s = c->stream;
    const int saved_iter = c->opt.max_iter;
    const int saved_sm = c->smoother;
    const int saved_outer = c->opt.outer;
    std::vector<double> hg(n_cycles + 1, 0.0), hj(n_cycles + 1, 0.0);
    int kg = 0, kj = 0, stg = AMG_OK, stj = AMG_OK, rc = AMG_OK;
    c->opt.max_iter = n_cycles;
    c->opt.outer = AMG_OUTER_REFINE;   // the metric compares the stationary V-cycle iteration (Sec. 3.3)
    for (int pass = 0; pass < 2 && rc != AMG_ERR_CUDA; ++pass) {
        c->smoother = pass == 0 ? AMG_SMOOTHER_GNN : AMG_SMOOTHER_JACOBI;
        rc = ctx_cuda_check(c, cudaMemcpyAsync(c->db, b, sizeof(double) * n0, cudaMemcpyHostToDevice, s), "copy b");
        if (!rc) rc = ctx_cuda_check(c, cudaMemsetAsync(c->dx, 0, sizeof(double) * n0, s), "zero x");
        if (!rc) rc = solve_dispatch(c, s, 0.0, pass == 0 ? &kg : &kj, pass == 0 ? hg.data() : hj.data());
        if (pass == 0) stg = rc; else stj = rc;
    }
    c->opt.max_iter = saved_iter;
    c->smoother = saved_sm;
    c->opt.outer = saved_outer;
    if (rc == AMG_ERR_CUDA || stg == AMG_ERR_CUDA) return AMG_ERR_CUDA;
    if (stg == AMG_ERR_DIVERGED) *metric = INFINITY;
    else if (stj == AMG_ERR_DIVERGED) *metric = -INFINITY;
    else {
        const int m = std::min(kg, kj);
        *metric = std::log10(hg[m] / hj[m]);
    }
    return AMG_OK;
}

int amg_reroute(amg_ctx *c, const double *b, int n_cycles, double *metric, int *smoother) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (!b || n_cycles < 4 || n_cycles > 10000) return ctx_fail(c, "bad argument (n_cycles >= 4)"), AMG_ERR_ARG;
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!c->have_q) return ctx_fail(c, "no pseudo-inverse coefficients set"), AMG_ERR_STATE;
    CK(cudaSetDevice(c->opt.device));
    const int n0 = c->lev[0].n;
    cudaStream_t s = c->stream;
    const int saved_iter = c->opt.max_iter;
    const int saved_outer = c->opt.outer;
    std::vector<double> h[2];
    int k[2] = {0, 0}, st[2] = {AMG_OK, AMG_OK}, rc = AMG_OK;
    c->opt.max_iter = n_cycles;
    c->opt.outer = AMG_OUTER_REFINE;   // probe with the stationary V-cycle iteration (Sec. 3.3)
    for (int pass = 0; pass < 2 && rc != AMG_ERR_CUDA; ++pass) {
        c->smoother = pass == 0 ? AMG_SMOOTHER_GNN : AMG_SMOOTHER_JACOBI;
        h[pass].assign(n_cycles + 1, 0.0);
        rc = ctx_cuda_check(c, cudaMemcpyAsync(c->db, b, sizeof(double) * n0, cudaMemcpyHostToDevice, s), "copy b");
        if (!rc) rc = ctx_cuda_check(c, cudaMemsetAsync(c->dx, 0, sizeof(double) * n0, s), "zero x");
        if (!rc) rc = solve_dispatch(c, s, 0.0, &k[pass], h[pass].data());
        st[pass] = rc;
    }
    c->opt.max_iter = saved_iter;
    c->opt.outer = saved_outer;
    c->smoother = AMG_SMOOTHER_GNN;
    if (rc == AMG_ERR_CUDA || st[0] == AMG_ERR_CUDA) return AMG_ERR_CUDA;
    // metric 1: log10(||r_n^GNN|| / ||r_n^J||) (Sec. 3.3); metric 2: the same
    // ratio for the reduction over the last quarter of the cycles, which
    // exposes smoothers that start well but converge slowly.  Both stop at the
    // first cycle at which either relative residual is down to kProbeFloor:
    // past it both iterations sit at rounding level and their ratios are noise.
    constexpr double kProbeFloor = 1e-12;
    auto floor_cycle = [&](int pass) {
        for (int t = 1; t <= k[pass]; ++t)
            if (h[pass][t] <= kProbeFloor) return t;
        return k[pass];
    };
    double m;
    if (st[0] == AMG_ERR_DIVERGED) {
        m = INFINITY;
    } else if (st[1] == AMG_ERR_DIVERGED) {
        m = -INFINITY;
    } else {
        const int n = std::min(floor_cycle(0), floor_cycle(1));
        const int q = std::max(1, n / 4);
        const double m1 = std::log10(h[0][n] / h[1][n]);
        const double m2 = (n > q) ? std::log10((h[0][n] / h[0][n - q]) / (h[1][n] / h[1][n - q])) : m1;
        // a stagnating learned smoother counts only if it stalled above the floor
        const bool stalled = st[0] == AMG_ERR_STAGNATED && st[1] != AMG_ERR_STAGNATED && floor_cycle(0) == k[0] &&
                             h[0][k[0]] > kProbeFloor;
        m = stalled ? INFINITY : std::max(m1, m2);
    }
    if (metric) *metric = m;
    if (m < 0.0 && st[1] != AMG_ERR_DIVERGED) {
        // arm the in-solve check: over any 10 cycles the learned smoother must
        // gain at least half the decades Jacobi gained in this probe
        const int n = floor_cycle(1), q = std::max(1, n / 4);
        const double rate10 = std::pow(h[1][n] / h[1][n - q], 10.0 / q);
        c->stall_ratio = (rate10 > 0.0 && rate10 < 1.0) ? std::sqrt(rate10) : 0.0;
    }
    if (!(m < 0.0)) {
        rc = amg_set_jacobi(c, c->jac_omega);
        if (rc) return rc;
        c->err = "pseudo-inverse smoother rerouted to Jacobi (metric " + std::to_string(m) + ")";
    }
    if (smoother) *smoother = c->smoother;
    return AMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// measurement aids: algorithmic byte model and single-kernel launches
// ---------------------------------------------------------------------------
namespace {
// bytes of one row-group pass over M: rp, col, values, gathered vector x,
// plus `vec_rw` further vectors of n_rows entries
double pass_bytes(const DevMat &M, int tb, double gathered, double vec_rw) {
    return 4.0 * (M.nr + 1) + (4.0 + tb) * M.nnz + tb * gathered + tb * vec_rw * M.nr;
}

// Chebyshev: `apps` polynomial applications of cheb_degree steps; a step
// reads dinv, b, u_in, d and writes d, u_out; the zero-guess first step
// reads dinv, b and writes d, u
double cheb_bytes(const amg_ctx *c, const DevLevel &L, int tb, int apps, bool zero_init) {
    double b = 0.0;
    for (int a = 0; a < apps; ++a)
        for (int k = 0; k < c->cheb_degree; ++k)
            b += (k == 0 && a == 0 && zero_init) ? 4.0 * tb * L.n : pass_bytes(L.A, tb, L.n, 6);
    return b;
}

double smooth_bytes(const amg_ctx *c, const DevLevel &L, int tb, int nsweeps, bool zero_init) {
    if (c->smoother == AMG_SMOOTHER_CHEB) return cheb_bytes(c, L, tb, nsweeps, zero_init);
    const bool gnn = (c->smoother == AMG_SMOOTHER_GNN);
    double b = 0.0;
    for (int k = 0; k < nsweeps; ++k) {
        const bool first = (k == 0 && zero_init);
        if (gnn) {
            if (first) b += pass_bytes(L.A, tb, L.n, 1);                       // u = Q b
            else b += pass_bytes(L.A, tb, L.n, 2) + pass_bytes(L.A, tb, L.n, 2);   // r = b - A u ; u += Q r
        } else {
            if (first) b += 3.0 * tb * L.n;                                    // u = jac b
            else b += pass_bytes(L.A, tb, L.n, 3);                            // u' = u + jac (b - A u)
        }
    }
    return b;
}

double smooth_fast_bytes(const amg_ctx *c, const DevLevel &L, int tb, int nsweeps, bool zero_init) {
    if (c->smoother == AMG_SMOOTHER_CHEB) return cheb_bytes(c, L, tb, nsweeps, zero_init);
    const bool gnn = (c->smoother == AMG_SMOOTHER_GNN);
    double b = 0.0;
    int k = 0;
    if (nsweeps == 0) return zero_init ? tb * L.n : 0.0;
    if (zero_init) {
        if (gnn) { b += pass_bytes(L.A, tb, L.n, 2); k = 1; }              // u = w = M b
        else if (nsweeps >= 2) { b += pass_bytes(L.A, tb, 2.0 * L.n, 1); k = 2; }   // two Jacobi sweeps
        else { b += 3.0 * tb * L.n; k = 1; }
    } else if (gnn && c->opt.nu1 == 0) {
        b += pass_bytes(L.A, tb, L.n, 1);                                  // w = M b
    }
    for (; k < nsweeps; ++k)
        b += gnn ? pass_bytes(L.MA, tb, L.n, 2) : pass_bytes(L.A, tb, L.n, 3);   // u' = u + w - (M A) u
    return b;
}

double vcycle_bytes_level(const amg_ctx *c, int l, int tb) {
    const DevLevel &L = c->lev[l];
    const int nlev = static_cast<int>(c->lev.size());
    if (l == nlev - 1) return 8.0 * c->nL * c->nL + 2.0 * tb * c->nL;
    const bool cheb = (c->smoother == AMG_SMOOTHER_CHEB);
    const int nu1 = cheb ? (c->opt.nu1 > 0 ? 1 : 0) : c->opt.nu1;
    const int nu2 = cheb ? (c->opt.nu2 > 0 ? 1 : 0) : c->opt.nu2;
    double b;
    if (L.fast) {
        b = smooth_fast_bytes(c, L, tb, nu1, true);
        b += pass_bytes(L.R, tb, L.n, 1) + pass_bytes(L.RA, tb, L.n, 0);   // b_c = R b - (R A) u
        b += vcycle_bytes_level(c, l + 1, tb);
        b += pass_bytes(L.P, tb, L.P.nc, 2);
        b += smooth_fast_bytes(c, L, tb, nu2, false);
        return b;
    }
    b = smooth_bytes(c, L, tb, nu1, true);
    b += pass_bytes(L.A, tb, L.n, 2);                           // residual
    b += pass_bytes(L.R, tb, L.n, 1);                           // restriction
    b += vcycle_bytes_level(c, l + 1, tb);
    b += pass_bytes(L.P, tb, L.P.nc, 2);                        // prolongation-correction
    b += smooth_bytes(c, L, tb, nu2, false);
    return b;
}

template <class T>
int kernel_launch(amg_ctx *c, int which, int l, int reps, cudaStream_t s, double *bytes) {
    DevLevel &L = c->lev[l];
    const int tb = sizeof(T);
    T *b = reinterpret_cast<T *>(L.vb), *u = reinterpret_cast<T *>(L.vu);
    T *r = reinterpret_cast<T *>(L.vr), *t = reinterpret_cast<T *>(L.vt);
    const int last = static_cast<int>(c->lev.size()) - 1;
    double by = 0.0;
    switch (which) {
        case AMG_K_RESIDUAL:
            by = pass_bytes(L.A, tb, L.n, 2);
            for (int k = 0; k < reps; ++k) L_resid<T>(L.A, b, u, r, s);
            break;
        case AMG_K_PINV:
            if (!c->have_q) return ctx_fail(c, "no pseudo-inverse coefficients set"), AMG_ERR_STATE;
            by = pass_bytes(L.A, tb, L.n, 2);
            for (int k = 0; k < reps; ++k) L_apply<T>(L.A, qvals<T>(L), r, u, 1, s);
            break;
        case AMG_K_JACOBI:
            by = pass_bytes(L.A, tb, L.n, 3);
            for (int k = 0; k < reps; ++k) L_jacobi<T>(L.A, jvals<T>(L), b, (k & 1) ? t : u, (k & 1) ? u : t, s);
            break;
        case AMG_K_RESTRICT:
            if (l >= last) return ctx_fail(c, "no restriction on the coarsest level"), AMG_ERR_ARG;
            by = pass_bytes(L.R, tb, L.n, 1);
            for (int k = 0; k < reps; ++k) L_spmv<T>(L.R, r, reinterpret_cast<T *>(c->lev[l + 1].vb), s);
            break;
        case AMG_K_PROLONG:
            if (l >= last) return ctx_fail(c, "no prolongation on the coarsest level"), AMG_ERR_ARG;
            by = pass_bytes(L.P, tb, L.P.nc, 2);
            for (int k = 0; k < reps; ++k) L_apply<T>(L.P, mvals<T>(L.P), reinterpret_cast<T *>(c->lev[l + 1].vu), u, 1, s);
            break;
        case AMG_K_OUTER: {
            const DevMat &A = c->lev[0].A;
            by = 4.0 * (A.nr + 1) + 12.0 * A.nnz + 16.0 * A.nr + tb * A.nr;
            for (int k = 0; k < reps; ++k) launch_outer<T>(c, s, reinterpret_cast<T *>(c->lev[0].vr), nullptr);
            break;
        }
        case AMG_K_MASWEEP:
            if (!L.fast || !c->have_q) return ctx_fail(c, "level has no M A product (not latency-optimised or no coefficients)"), AMG_ERR_STATE;
            by = pass_bytes(L.MA, tb, L.n, 2);
            for (int k = 0; k < reps; ++k) {
                TPR_DISPATCH(L.MA.tpr, Launch<T>::template ma_sweep, L.MA, reinterpret_cast<const T *>(L.vw),
                             (k & 1) ? t : u, (k & 1) ? u : t, s);
            }
            break;
        case AMG_K_VCYCLE:
            by = vcycle_bytes_level(c, 0, tb);
            for (int k = 0; k < reps; ++k) vcycle_level<T>(c, 0, s);
            break;
        case AMG_K_EMPTY:
            by = 0.0;
            for (int k = 0; k < reps; ++k) launch_pdl(k_empty, dim3(1), dim3(kBlock), 0, s);
            break;
        case AMG_K_WF_PRE:
        case AMG_K_WF_POST: {
            if (!wf_usable(c, L) || l >= last)
                return ctx_fail(c, "level runs no wavefront chain (L2-sized level, Chebyshev, or fused_sweeps = 0)"),
                       AMG_ERR_STATE;
            if (c->smoother == AMG_SMOOTHER_GNN && !c->have_q)
                return ctx_fail(c, "no pseudo-inverse coefficients set"), AMG_ERR_STATE;
            const bool pre = (which == AMG_K_WF_PRE);
            // the method's bytes of the passes the chain runs (as if unfused)
            by = pre ? smooth_bytes(c, L, tb, c->opt.nu1, true) + pass_bytes(L.A, tb, L.n, 2)
                     : pass_bytes(L.P, tb, L.P.nc, 2) + smooth_bytes(c, L, tb, c->opt.nu2, false);
            const T *e = reinterpret_cast<const T *>(c->lev[l + 1].vu);
            cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), s);
            for (int k = 0; k < reps; ++k) {
                int ui = 0, ri = 0;
                if (pre) wf_pre<T>(c, l, s, b, ui, ri);
                else wf_post<T>(c, l, s, b, 2, e);
            }
            break;
        }
        default:
            return ctx_fail(c, "unknown kernel id"), AMG_ERR_ARG;
    }
    if (bytes) *bytes = by;
    return ctx_cuda_check(c, cudaGetLastError(), "kernel launch");
}
}  // namespace

extern "C" {

long long amg_launch_count(void) { return amg::g_launches.load(); }

int amg_last_solve_rerouted(const amg_ctx *c) { return c ? c->last_rerouted : 0; }

int amg_vcycle_bytes(const amg_ctx *c, double *bytes) {
    if (!c || !bytes) return AMG_ERR_ARG;
    if (c->lev.empty()) return AMG_ERR_STATE;
    *bytes = vcycle_bytes_level(c, 0, c->opt.precision == AMG_FP64 ? 8 : 4);
    return AMG_OK;
}

int amg_kernel_launch(amg_ctx *c, int which, int level, int reps, void *stream, double *bytes) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (level < 0 || level >= static_cast<int>(c->lev.size()) || reps < 0)
        return ctx_fail(c, "bad level or repetition count"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->opt.precision == AMG_FP64) return kernel_launch<double>(c, which, level, reps, s, bytes);
    return kernel_launch<float>(c, which, level, reps, s, bytes);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free residual norm (caller owns every buffer; scratch is static)
// ---------------------------------------------------------------------------
namespace {
// Per-block partial sums of ||r||^2 and ||b||^2.  Lives for the life of the
// process on every device that loads this library; shared by all calls.
constexpr int kStaticSlots = kNumSMs * 8;      // blocks of one launch at most
constexpr int kNoAllocMaxRows = (1 << 26) - 1; // row * 32 lanes must fit in int
static __device__ __align__(256) double g_static_partials[2 * kStaticSlots];

// r = b - A x in FP64 (r stored when r_out != NULL); partials of r.r and b.b
template <int TPR>
__global__ void __launch_bounds__(kBlock) k_resid_norm_static(int n, const int *__restrict__ rp,
                                                              const int *__restrict__ col,
                                                              const double *__restrict__ a,
                                                              const double *__restrict__ b,
                                                              const double *__restrict__ x,
                                                              double *__restrict__ r_out,
                                                              double *__restrict__ scratch) {
    constexpr int RPB = kBlock / TPR;
    const int lane = threadIdx.x % TPR;
    double rr = 0.0, bb = 0.0;
    for (int base = blockIdx.x * RPB; base < n; base += gridDim.x * RPB) {
        const int row = base + threadIdx.x / TPR;
        double acc = 0.0;
        if (row < n) {
            const int e = rp[row + 1];
            acc = row_dot<TPR>(lane, rp[row], e, col, a, Gather<double>{x});
        }
        acc = group_sum<TPR>(acc);
        if (row < n && lane == 0) {
            const double r = b[row] - acc;
            if (r_out) r_out[row] = r;
            rr += r * r;
            bb += b[row] * b[row];
        }
    }
    block_partial(rr, scratch);
    __syncthreads();
    block_partial(bb, scratch + kStaticSlots);
}

// out[0] = ||b - A x||_2, out[1] = ||b||_2 from the first np partials (fixed order)
__global__ void __launch_bounds__(1024) k_resid_norm_static_final(int np, double *__restrict__ out) {
    __shared__ double red[2][32];
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < np; i += 1024) {
        v[0] += g_static_partials[i];
        v[1] += g_static_partials[kStaticSlots + i];
    }
    for (int k = 0; k < 2; ++k) {
        double w = warp_sum(v[k]);
        if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = w;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = 0; k < 2; ++k) {
            double w = warp_sum(red[k][threadIdx.x]);
            if (threadIdx.x == 0) out[k] = sqrt(w);
        }
    }
}

__global__ void k_zero2(double *out) {
    out[0] = 0.0;
    out[1] = 0.0;
}

// Device address of g_static_partials, looked up once per device.
std::mutex g_static_mutex;
double *g_static_addr[64] = {};

int static_scratch_for(int dev, double **ptr) {
    if (dev < 0 || dev >= 64) {
        g_create_err = "device ordinal out of range for the static scratch table";
        return AMG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess || !p) {
            g_create_err = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
            return AMG_ERR_CUDA;
        }
        g_static_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_static_addr[dev];
    return AMG_OK;
}
}  // namespace

extern "C" int amg_residual_norm_noalloc(int n, long long nnz, const int *d_row_ptr, const int *d_col,
                                         const double *d_val, const double *d_b, const double *d_x,
                                         double *d_r, double *d_out, void *stream) {
    g_create_err.clear();
    if (n < 0 || n > kNoAllocMaxRows || nnz < 0 || nnz > 2147483647LL) {
        g_create_err = "amg_residual_norm_noalloc: n must be in [0, 67108863] and nnz in [0, 2^31-1]";
        return AMG_ERR_ARG;
    }
    if (!d_out || (n > 0 && (!d_row_ptr || !d_b || !d_x || (nnz > 0 && (!d_col || !d_val))))) {
        g_create_err = "amg_residual_norm_noalloc: NULL device pointer";
        return AMG_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_create_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return AMG_ERR_CUDA;
    }
    double *scratch = nullptr;
    int rc = static_scratch_for(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        k_zero2<<<1, 1, 0, s>>>(d_out); AMG_COUNT();
    } else {
        const int tpr = pick_tpr(nnz, n);
        const long long need = (static_cast<long long>(n) * tpr + kBlock - 1) / kBlock;
        const int nb = static_cast<int>(std::max(1LL, std::min<long long>(need, kStaticSlots)));
        switch (tpr) {
            case 1: k_resid_norm_static<1><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
            case 2: k_resid_norm_static<2><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
            case 4: k_resid_norm_static<4><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
            case 8: k_resid_norm_static<8><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
            case 16: k_resid_norm_static<16><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
            default: k_resid_norm_static<32><<<nb, kBlock, 0, s>>>(n, d_row_ptr, d_col, d_val, d_b, d_x, d_r, scratch); break;
        }
        AMG_COUNT();
        k_resid_norm_static_final<<<1, 1024, 0, s>>>(nb, d_out); AMG_COUNT();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_create_err = std::string("amg_residual_norm_noalloc launch: ") + cudaGetErrorString(e);
        return AMG_ERR_CUDA;
    }
    return AMG_OK;
}

// ---------------------------------------------------------------------------
// Training loss and the hand-written V-cycle adjoint (Sec. 3.3, N_vc = 1)
// ---------------------------------------------------------------------------
// Forward: one V-cycle from u = 0 with the pseudo-inverse smoother, keeping
// every sweep's input residual r_k per level (the checkpoints).  A sweep is
// u' = u + M r, r = b - A u, M = Q^-1(c) symmetric, so its adjoint is
//   dL/dM_ij += ubar'_i r_j,  rbar = M ubar',  ubar = ubar' - A rbar,  bbar += rbar,
// restriction and prolongation swap (R^T = P), and the coarse solve is
// self-adjoint.  dL/dc_k = sum_ij dL/dM_ij dM_ij/dc_k with
//   dM_ii/d(d0, d1, d2) = (1, x, x^2) / a_ii,          x = a_ii / s
//   dM_ij/d(o1, o2)     = (x, x^2) / (a_ii + a_jj),    x = a_ij / s.
namespace {

template <class T, int TPR>
__global__ void __launch_bounds__(kBlock) k_coef_grad(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                      const double *__restrict__ bx, const double *__restrict__ bw,
                                                      const T *__restrict__ ubar, const T *__restrict__ r,
                                                      double *__restrict__ partial) {
    constexpr int RPB = kBlock / TPR;
    const int lane = threadIdx.x % TPR;
    double g[5] = {0, 0, 0, 0, 0};
    for (int base = blockIdx.x * RPB; base < n; base += gridDim.x * RPB) {
        const int row = base + threadIdx.x / TPR;
        double acc[5] = {0, 0, 0, 0, 0};
        if (row < n) {
            const double ui = static_cast<double>(ubar[row]);
            for (int p = rp[row] + lane; p < rp[row + 1]; p += TPR) {
                const int j = col[p];
                const double x = bx[p], w = ui * static_cast<double>(r[j]) * bw[p];
                if (j == row) {
                    acc[0] += w;
                    acc[1] += w * x;
                    acc[2] += w * x * x;
                } else {
                    acc[3] += w * x;
                    acc[4] += w * x * x;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) g[k] += group_sum<TPR>(acc[k]);
    }
    __shared__ double red[5][kBlock / 32];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = (lane == 0) ? g[k] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += red[threadIdx.x][w];
        partial[blockIdx.x * 5 + threadIdx.x] = t;
    }
}

__global__ void k_coef_grad_final(int np, const double *__restrict__ partial, double *__restrict__ dc) {
    if (threadIdx.x >= 5) return;
    double t = 0.0;
    for (int b = 0; b < np; ++b) t += partial[b * 5 + threadIdx.x];
    dc[threadIdx.x] += t;
}

template <class T>
__global__ void k_add(int n, T *__restrict__ y, const T *__restrict__ x) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) y[i] += x[i];
}

template <class T>
__global__ void k_scale_copy(int n, T *__restrict__ y, const T *__restrict__ x, double a) {
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < n) y[i] = static_cast<T>(a * static_cast<double>(x[i]));
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_dot_partial(int n, const T *__restrict__ x, const T *__restrict__ y,
                                                        double *__restrict__ partial) {
    double s = 0.0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        s += static_cast<double>(x[i]) * static_cast<double>(y[i]);
    block_partial(s, partial);
}

__global__ void k_sum_final(int np, const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += 1024) v += partial[i];
    v = warp_sum(v);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = warp_sum(red[threadIdx.x]);
        if (threadIdx.x == 0) *out = v;
    }
}

struct TrainBufs {
    int ncyc = 0, nsw = 0, nlev = 0;
    std::vector<double *> ck;      // [cycle][level][sweep]: slot 0 = that cycle's b_l, k >= 1 = r of sweep k
    std::vector<double *> ubar, tmp, bbar, zero;
    double *xu = nullptr;          // level-0 iterate of the multi-cycle loss
    double *dcoef = nullptr;       // n_levels x 5
    double *scal = nullptr;        // 4 doubles
    char *arena = nullptr;
    double *slot(int cyc, int l, int k) const { return ck[(static_cast<size_t>(cyc) * nlev + l) * nsw + k]; }
};

int train_bufs(amg_ctx *c, TrainBufs &tb, int ncyc) {
    const int nlev = static_cast<int>(c->lev.size());
    const int nsw = std::max(1, c->opt.nu1 + c->opt.nu2);
    tb.ncyc = ncyc;
    tb.nsw = nsw;
    tb.nlev = nlev;
    auto lay = [&](Planner &pl) {
        tb.ck.assign(static_cast<size_t>(ncyc) * nlev * nsw, nullptr);
        tb.ubar.assign(nlev, nullptr);
        tb.tmp.assign(nlev, nullptr);
        tb.bbar.assign(nlev, nullptr);
        tb.zero.assign(nlev, nullptr);
        for (int l = 0; l < nlev; ++l) {
            const int n = c->lev[l].n;
            for (int q = 0; q < ncyc; ++q)
                for (int k = 0; k < nsw; ++k) tb.ck[(static_cast<size_t>(q) * nlev + l) * nsw + k] = pl.take<double>(n);
            tb.ubar[l] = pl.take<double>(n);
            tb.tmp[l] = pl.take<double>(n);
            tb.bbar[l] = pl.take<double>(n);
            tb.zero[l] = pl.take<double>(n);
        }
        tb.xu = pl.take<double>(c->lev[0].n);
        tb.dcoef = pl.take<double>(static_cast<size_t>(nlev) * 5);
        tb.scal = pl.take<double>(4);
    };
    Planner pl;
    lay(pl);
    cudaError_t e = cudaMalloc(&tb.arena, pl.off);
    if (e != cudaSuccess) return ctx_cuda_check(c, e, "cudaMalloc training buffers");
    const size_t bytes = pl.off;
    pl = Planner{};
    pl.base = tb.arena;
    lay(pl);
    return ctx_cuda_check(c, cudaMemsetAsync(tb.arena, 0, bytes, c->stream), "memset training buffers");
}

template <class T>
T *fwd_level_ckpt(amg_ctx *c, TrainBufs &tb, int cyc, int l, cudaStream_t s) {
    DevLevel &L = c->lev[l];
    T *b = reinterpret_cast<T *>(L.vb), *u = reinterpret_cast<T *>(L.vu), *r = reinterpret_cast<T *>(L.vr);
    const int nlev = static_cast<int>(c->lev.size());
    const int nu1 = c->opt.nu1, nu2 = c->opt.nu2, nsw = nu1 + nu2;
    if (l == nlev - 1) {
        launch_pdl(k_coarse<T>, dim3(1), dim3(kBlock), 2 * sizeof(double) * c->nL, s, c->nL, c->Linv, c->LinvT, b, u);
        return u;
    }
    auto ck = [&](int k) { return reinterpret_cast<T *>(tb.slot(cyc, l, k)); };
    cudaMemcpyAsync(ck(0), b, sizeof(T) * L.n, cudaMemcpyDeviceToDevice, s);
    if (nu1 == 0) cudaMemsetAsync(u, 0, sizeof(T) * L.n, s);
    for (int k = 0; k < nu1; ++k) {
        if (k == 0) {
            L_apply<T>(L.A, qvals<T>(L), b, u, 0, s);
        } else {
            L_resid<T>(L.A, b, u, ck(k), s);
            L_apply<T>(L.A, qvals<T>(L), ck(k), u, 1, s);
        }
    }
    L_resid<T>(L.A, b, u, r, s);
    L_spmv<T>(L.R, r, reinterpret_cast<T *>(c->lev[l + 1].vb), s);
    T *e = fwd_level_ckpt<T>(c, tb, cyc, l + 1, s);
    L_apply<T>(L.P, mvals<T>(L.P), e, u, 1, s);
    for (int k = nu1; k < nsw; ++k) {
        L_resid<T>(L.A, b, u, ck(k), s);
        L_apply<T>(L.A, qvals<T>(L), ck(k), u, 1, s);
    }
    (void)nsw;
    return u;
}

template <class T>
void coef_grad(amg_ctx *c, TrainBufs &tb, int l, const T *ubar, const T *r, cudaStream_t s) {
    const DevLevel &L = c->lev[l];
    const DevMat &A = L.A;
    const int nb = outer_blocks(A);
#define CG_LAUNCH(TP)                                                                                          \
    k_coef_grad<T, TP><<<nb, kBlock, 0, s>>>(A.nr, A.rp, A.col, L.bx, L.bw, ubar, r, c->partials); \
    AMG_COUNT();
    switch (A.tpr) {
        case 1: CG_LAUNCH(1) break;
        case 2: CG_LAUNCH(2) break;
        case 4: CG_LAUNCH(4) break;
        case 8: CG_LAUNCH(8) break;
        case 16: CG_LAUNCH(16) break;
        default: CG_LAUNCH(32) break;
    }
#undef CG_LAUNCH
    k_coef_grad_final<<<1, 32, 0, s>>>(nb, c->partials, tb.dcoef + 5 * l); AMG_COUNT();
}

// Backward of one sweep u' = u + M r (r = b - A u): accumulate dL/dc, then
// ubar <- ubar - A (M ubar) into `spare`, bbar += M ubar.  Returns the new ubar.
template <class T>
T *sweep_adjoint(amg_ctx *c, TrainBufs &tb, int l, T *ubar, T *spare, const T *r, T *bbar, cudaStream_t s) {
    const DevLevel &L = c->lev[l];
    coef_grad<T>(c, tb, l, ubar, r, s);
    T *rbar = reinterpret_cast<T *>(L.vt);            // free during the backward pass
    L_apply<T>(L.A, qvals<T>(L), ubar, rbar, 0, s);   // rbar = M ubar
    L_resid<T>(L.A, ubar, rbar, spare, s);            // spare = ubar - A rbar
    k_add<T><<<grid_for(L.n), kBlock, 0, s>>>(L.n, bbar, rbar); AMG_COUNT();
    return spare;
}

// Backward of the V-cycle on level l: tb.ubar[l] = dL/d(level output) in,
// tb.bbar[l] = dL/d(level right-hand side) out.
template <class T>
void bwd_level(amg_ctx *c, TrainBufs &tb, int cyc, int l, cudaStream_t s) {
    DevLevel &L = c->lev[l];
    const int nlev = static_cast<int>(c->lev.size());
    const int nu1 = c->opt.nu1, nu2 = c->opt.nu2, nsw = nu1 + nu2;
    T *ub = reinterpret_cast<T *>(tb.ubar[l]), *sp = reinterpret_cast<T *>(tb.tmp[l]);
    T *bb = reinterpret_cast<T *>(tb.bbar[l]);
    if (l == nlev - 1) {   // u = A_L^-1 b is self-adjoint
        launch_pdl(k_coarse<T>, dim3(1), dim3(kBlock), 2 * sizeof(double) * c->nL, s, c->nL, c->Linv, c->LinvT, ub, bb);
        return;
    }
    auto ck = [&](int k) { return reinterpret_cast<const T *>(tb.slot(cyc, l, k)); };
    cudaMemsetAsync(bb, 0, sizeof(T) * L.n, s);
    for (int k = nsw - 1; k >= nu1; --k) {
        T *nu = sweep_adjoint<T>(c, tb, l, ub, sp, ck(k), bb, s);
        sp = ub;
        ub = nu;
    }
    // prolongation u += P e: ebar = P^T ubar = R ubar
    L_spmv<T>(L.R, ub, reinterpret_cast<T *>(tb.ubar[l + 1]), s);
    bwd_level<T>(c, tb, cyc, l + 1, s);
    // restriction b_{l+1} = R (b - A u): rhobar = R^T bbar_{l+1} = P bbar_{l+1}
    T *rhobar = reinterpret_cast<T *>(L.vt);
    L_spmv<T>(L.P, reinterpret_cast<const T *>(tb.bbar[l + 1]), rhobar, s);
    k_add<T><<<grid_for(L.n), kBlock, 0, s>>>(L.n, bb, rhobar); AMG_COUNT();
    L_resid<T>(L.A, ub, rhobar, sp, s);
    std::swap(ub, sp);
    for (int k = nu1 - 1; k >= 1; --k) {
        T *nu = sweep_adjoint<T>(c, tb, l, ub, sp, ck(k), bb, s);
        sp = ub;
        ub = nu;
    }
    if (nu1 >= 1) {        // first sweep from zero: u = M b
        coef_grad<T>(c, tb, l, ub, ck(0), s);
        L_apply<T>(L.A, qvals<T>(L), ub, reinterpret_cast<T *>(L.vt), 0, s);
        k_add<T><<<grid_for(L.n), kBlock, 0, s>>>(L.n, bb, reinterpret_cast<const T *>(L.vt)); AMG_COUNT();
    }
}

// Multi-V-cycle loss (Sec. 3.3): u_n = u_{n-1} + B(f - A u_{n-1}) (the
// stationary V-cycle in refinement form), L = sum_n log10(||r_n|| / ||r_{n-1}||)
// = log10(||r_N|| / ||f||).  Backward: ubar_N = -A r_N / (ln10 ||r_N||^2);
// for n = N..1: rbar = B^T ubar (level adjoint, accumulating dL/dc), ubar -= A rbar.
template <class T>
int loss_grad(amg_ctx *c, TrainBufs &tb, const double *f, int nvc, double *loss, double *dc) {
    cudaStream_t s = c->stream;
    DevLevel &L0 = c->lev[0];
    const int n0 = L0.n, nlev = static_cast<int>(c->lev.size());
    T *fT = reinterpret_cast<T *>(tb.tmp[0]);
    T *xu = reinterpret_cast<T *>(tb.xu);
    T *b0 = reinterpret_cast<T *>(L0.vb);
    CK(cudaMemcpyAsync(c->db, f, sizeof(double) * n0, cudaMemcpyHostToDevice, s));
    launch_pdl(k_convert<double, T>, dim3(grid_for(n0)), dim3(kBlock), 0, s, n0, c->db, fT);
    CK(cudaMemsetAsync(xu, 0, sizeof(T) * n0, s));
    for (int q = 0; q < nvc; ++q) {
        L_resid<T>(L0.A, fT, xu, b0, s);          // r_{q} = f - A u_q -> level-0 right-hand side
        T *e = fwd_level_ckpt<T>(c, tb, q, 0, s);
        k_add<T><<<grid_for(n0), kBlock, 0, s>>>(n0, xu, e); AMG_COUNT();
    }
    T *rN = reinterpret_cast<T *>(L0.vr);
    L_resid<T>(L0.A, fT, xu, rN, s);
    const int nb = std::min(grid_for(n0), kNumSMs * 8);
    k_dot_partial<T><<<nb, kBlock, 0, s>>>(n0, rN, rN, c->partials); AMG_COUNT();
    k_sum_final<<<1, 1024, 0, s>>>(nb, c->partials, tb.scal); AMG_COUNT();
    k_dot_partial<T><<<nb, kBlock, 0, s>>>(n0, fT, fT, c->partials); AMG_COUNT();
    k_sum_final<<<1, 1024, 0, s>>>(nb, c->partials, tb.scal + 1); AMG_COUNT();
    double h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, tb.scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double rr = h[0], ff = h[1];
    if (!(rr > 0.0) || !(ff > 0.0) || !std::isfinite(rr))
        return ctx_fail(c, "loss undefined: zero or non-finite residual"), AMG_ERR_DIVERGED;
    *loss = 0.5 * std::log10(rr / ff);
    // ubar_N = -A (r_N / (ln10 ||r_N||^2)) into ubar[0].  The carried adjoint
    // and its scratch use xu and vr of level 0, which the level adjoint never
    // touches (it works in ubar/tmp/bbar and vt).
    T *seed = xu;                                   // the forward iterate is no longer needed
    T *ub0 = reinterpret_cast<T *>(tb.ubar[0]);
    k_scale_copy<T><<<grid_for(n0), kBlock, 0, s>>>(n0, seed, rN, 1.0 / (std::log(10.0) * rr)); AMG_COUNT();
    L_resid<T>(L0.A, reinterpret_cast<const T *>(tb.zero[0]), seed, ub0, s);
    CK(cudaMemsetAsync(tb.dcoef, 0, sizeof(double) * 5 * nlev, s));
    T *uacc = rN;                                   // dL/du_q carried across cycles (r_N no longer needed)
    CK(cudaMemcpyAsync(uacc, ub0, sizeof(T) * n0, cudaMemcpyDeviceToDevice, s));
    for (int q = nvc - 1; q >= 0; --q) {
        CK(cudaMemcpyAsync(ub0, uacc, sizeof(T) * n0, cudaMemcpyDeviceToDevice, s));   // ebar = ubar_{q+1}
        bwd_level<T>(c, tb, q, 0, s);                                                // bbar[0] = rbar_q
        if (q > 0) {
            L_resid<T>(L0.A, uacc, reinterpret_cast<const T *>(tb.bbar[0]), seed, s);   // ubar_q = ubar - A rbar
            std::swap(uacc, seed);
        }
    }
    CKL("V-cycle adjoint");
    CK(cudaMemcpyAsync(dc, tb.dcoef, sizeof(double) * 5 * nlev, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

}  // namespace

extern "C" int amg_loss_grad(amg_ctx *c, const double *coef, const double *f, int n_vc, double *loss, double *dc) {
    if (!c) return AMG_ERR_ARG;
    c->err.clear();
    if (c->lev.empty()) return ctx_fail(c, "no hierarchy loaded"), AMG_ERR_STATE;
    if (!coef || !f || !loss || !dc || n_vc < 1 || n_vc > 64) return ctx_fail(c, "bad argument"), AMG_ERR_ARG;
    CK(cudaSetDevice(c->opt.device));
    const int nlev = static_cast<int>(c->lev.size());
    int rc = set_coeffs_device(c, coef, nlev, c->stream);
    if (rc) return rc;
    if (c->train && static_cast<TrainBufs *>(c->train)->ncyc < n_vc) train_bufs_free(c);
    if (!c->train) {
        TrainBufs *tb = new TrainBufs();
        rc = train_bufs(c, *tb, n_vc);
        if (rc) {
            if (tb->arena) cudaFree(tb->arena);
            delete tb;
            return rc;
        }
        c->train = tb;
    }
    TrainBufs &tb = *static_cast<TrainBufs *>(c->train);
    if (c->opt.precision == AMG_FP64) return loss_grad<double>(c, tb, f, n_vc, loss, dc);
    return loss_grad<float>(c, tb, f, n_vc, loss, dc);
}

namespace amg {
void train_bufs_free(amg_ctx *c) {
    if (!c->train) return;
    TrainBufs *tb = static_cast<TrainBufs *>(c->train);
    if (tb->arena) cudaFree(tb->arena);
    delete tb;
    c->train = nullptr;
}
}  // namespace amg
