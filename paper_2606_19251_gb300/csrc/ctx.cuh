// Internal state of an amg_ctx (device hierarchy, work vectors, solve state).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "amg_gnn.h"
#include "common.cuh"
#include "setup_host.h"

namespace amg {

// CSR matrix on the device; values in FP64 and FP32 (the V-cycle precision).
struct DevMat {
    int nr = 0, nc = 0, nnz = 0, tpr = 2;
    int *rp = nullptr, *col = nullptr;
    short *dcol = nullptr;                     // col - row in 16 bits (square levels whose offsets fit), or null
    double *v64 = nullptr;
    float *v32 = nullptr;
};

struct DevLevel {
    int n = 0;
    DevMat A, P, R;                            // P: n x n_{l+1}; R: n_{l+1} x n
    double *diag = nullptr;                    // a_ii (FP64)
    double *bx = nullptr, *bw = nullptr;       // pseudo-inverse basis a_ij/s and 1/a_ii or 1/(a_ii+a_jj)
    float *bx32 = nullptr, *bw32 = nullptr;    // the same in FP32 (assembly for the FP32 V-cycle)
    unsigned char *isd = nullptr;              // 1 on the diagonal entries of A's pattern
    double *q64 = nullptr; float *q32 = nullptr;   // pseudo-inverse values on A's pattern
    double *j64 = nullptr; float *j32 = nullptr;   // omega / a_ii
    double *dinv64 = nullptr; float *dinv32 = nullptr;   // 1 / a_ii (Chebyshev smoother)
    double cheb_theta = 0.0, cheb_delta = 0.0, cheb_rho = 0.0;   // Chebyshev interval (host)
    // V-cycle vectors; storage sized for n doubles, used as float or double
    double *vb = nullptr, *vu = nullptr, *vr = nullptr, *vt = nullptr;
    // latency-optimised levels (L2-resident): single-pass sweeps with M A and
    // fused residual + restriction
    bool fast = false;
    DevMat MA;                                 // pattern of M A, values from the pair list
    DevMat RA;                                 // R A for the fused residual + restriction
    int *pp = nullptr, *pq_p = nullptr, *pq_q = nullptr;
    double *vw = nullptr;                      // w = M b of the current V-cycle
    // wavefront smoothing chains (levels too large for L2; wavefront.cuh)
    bool wf = false;
    int wf_rpt = 0, wf_nblk = 0, wf_ngroup = 0, wf_grid = 0;
    int wf_lag[9] = {};                        // lag (blocks) of a p-pass chain, p = 1..8
    int *wf_lohi = nullptr;                    // per block: first and last group of its columns
    unsigned *wf_count = nullptr;              // completed-task counters, p x ngroup for each p = 1..8
    unsigned *wf_ctrl = nullptr;               // 4 words per chain length: finished warps, launch number
    double *wf_buf = nullptr;                  // kWfBufs chain vectors (n doubles of storage each)
    float *diag32 = nullptr;                   // a_ii in FP32 (pseudo-inverse values on the fly)
};

// Host-side plan of a level's wavefront chains (built at upload).
struct WfPlan {
    bool on = false;
    int rpt = 0, nblk = 0, ngroup = 0, grid = 0;
    int lag[9] = {};
    std::vector<int> lohi;                     // 2 x nblk
};

enum : int { kRunning = 1, kStalled = 2 };

struct SolveState {
    int k;          // index of the next residual-history entry
    int status;     // kRunning or an AMG_* status
    int max_iter;
    int pad;
    double tol;
    double bnorm;   // ||b|| (1 if b = 0)
    double r0;      // ||b - A x0||
    double stall;   // > 0: a 10-cycle reduction worse than this ends the learned smoother's run
    double rho_old; // conjugate gradients: z.r of the previous iteration
    int restart;    // conjugate gradients: next direction is p = z
    int breakdown;  // conjugate gradients: z.r or p.Ap not positive
};

// Whole-solve CUDA graph: a kernel node copies the device-side status into
// a conditional handle, and a WHILE node repeats the captured iteration body
// (V-cycle, x += e, outer residual, norm and stopping rule) until the rule
// clears the handle.  One graph per smoother, rebuilt when the hierarchy changes.
struct SolveGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long version = -1;
    long long body_kernels = 0;
    int q_nodes = -1;    // the pseudo-inverse source the captured chains use
};

struct GcinEngine;
void gcin_engine_free(GcinEngine *e);

}  // namespace amg

struct amg_ctx {
    amg_options opt{};
    std::string err;
    std::vector<amg::HostLevel> host;          // host copy of the hierarchy
    std::vector<amg::DevLevel> lev;
    std::vector<double> scales;                // s_l (host copy)
    int nL = 0;                                // coarsest size
    double *Linv = nullptr, *LinvT = nullptr, *Ldense = nullptr;
    double *db = nullptr, *dx = nullptr;       // n_0 FP64 staging of b and x
    double *partials = nullptr;                // per-block partial sums
    int n_partials = 0;
    double *scal = nullptr;                    // device s_l
    amg::SolveState *state = nullptr;
    double *hist = nullptr;                    // max_iter + 1
    int *dflag = nullptr;
    int *dcol_flag = nullptr;                  // per level: 1 if a column offset does not fit 16 bits
    char *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t stream = nullptr;
    amg::SolveState *h_state = nullptr;        // pinned host mirror
    int smoother = AMG_SMOOTHER_JACOBI;
    bool have_q = false;
    double jac_omega = 2.0 / 3.0;
    amg::GcinEngine *gnn = nullptr;
    long long hier_version = 0;                // bumped by every hierarchy upload
    void *train = nullptr;                     // training (adjoint) buffers, created on demand
    amg::SolveGraph sgraph[6];                 // per smoother + 3 x outer iteration
    int cheb_degree = 3;
    long long cheb_version = -1;               // hierarchy version the Chebyshev intervals belong to
    double *pcg = nullptr;                     // conjugate gradients: r, r_prev, z, p, q (n_0 each)
    double stall_ratio = 0.0;                  // armed by amg_reroute for the learned smoother
    int last_rerouted = 0;                     // the last solve switched to Jacobi
    float *wcoef = nullptr;                    // per level: d0 d1 d2 o1 o2 1/s (FP32, wavefront chains)
    // finest level's FP64 operator in warp slices (outer-loop passes)
    int ell_nslice = 0;
    int *ell_ptr = nullptr, *ell_row = nullptr, *ell_col = nullptr;
    double *ell_val = nullptr;
    long long ell_entries = 0;                 // 32 x the sum of the slice widths
    std::vector<int> h_ell_ptr, h_ell_row;
    bool q_nodes = false;                      // Q^-1 from per-node coefficients (stored values only)
    bool q64_stale = false;                    // only the FP32 Q^-1 was assembled (coefficients kept in wcoef)
    std::vector<amg::WfPlan> wfplan;           // per level
};

namespace amg {
// helpers shared between translation units
bool ctx_fail(amg_ctx *c, const std::string &msg);
int ctx_cuda_check(amg_ctx *c, cudaError_t e, const char *what);
int set_coeffs_device(amg_ctx *c, const double *coef, int n_rows, cudaStream_t s);
int enqueue_coeff_assembly(amg_ctx *c, const float *d_coef, cudaStream_t s);
void train_bufs_free(amg_ctx *c);
}  // namespace amg
