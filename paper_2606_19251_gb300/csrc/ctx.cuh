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
    double *v64 = nullptr;
    float *v32 = nullptr;
};

struct DevLevel {
    int n = 0;
    DevMat A, P, R;                            // P: n x n_{l+1}; R: n_{l+1} x n
    double *diag = nullptr;                    // a_ii (FP64)
    double *q64 = nullptr; float *q32 = nullptr;   // pseudo-inverse values on A's pattern
    double *j64 = nullptr; float *j32 = nullptr;   // omega / a_ii
    // V-cycle vectors; storage sized for n doubles, used as float or double
    double *vb = nullptr, *vu = nullptr, *vr = nullptr, *vt = nullptr;
};

enum : int { kRunning = 1 };

struct SolveState {
    int k;          // index of the next residual-history entry
    int status;     // kRunning or an AMG_* status
    int max_iter;
    int pad;
    double tol;
    double bnorm;   // ||b|| (1 if b = 0)
    double r0;      // ||b - A x0||
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
};

namespace amg {
// helpers shared between translation units
bool ctx_fail(amg_ctx *c, const std::string &msg);
int ctx_cuda_check(amg_ctx *c, cudaError_t e, const char *what);
int set_coeffs_device(amg_ctx *c, const double *coef, int n_rows, cudaStream_t s);
void train_bufs_free(amg_ctx *c);
}  // namespace amg
