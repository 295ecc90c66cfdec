// Host-side AMG setup (Sec. 2.2): Ruge-Stueben coarsening, direct
// interpolation, Galerkin coarse operators.  Runs once per matrix, off the
// solve path; its output is uploaded by the device code.
#pragma once
#include <string>
#include <vector>

namespace amg {

struct HostCSR {
    int n_rows = 0, n_cols = 0;
    std::vector<int> rp, col;
    std::vector<double> val;
    // Device-built levels: col and val stay on the device (drp, dcol, dval)
    // until a host copy is asked for; rp is on the host as well.
    const int *drp = nullptr, *dcol = nullptr;
    const double *dval = nullptr;
    bool on_device() const { return dcol != nullptr; }
    long long nnz() const {
        return on_device() ? static_cast<long long>(rp.back()) : static_cast<long long>(col.size());
    }
};

struct HostLevel {
    HostCSR A;   // n_l x n_l
    HostCSR P;   // n_l x n_{l+1}   (empty on the coarsest level)
    HostCSR R;   // n_{l+1} x n_l, R = P^T
    // latency-optimised levels only: pattern of M A (M = Q^-1) and its pair list
    bool fast = false;
    HostCSR MA;
    HostCSR RA;        // R A (n_{l+1} x n_l): fused residual + restriction b_c = R b - (R A) u
    std::vector<int> pair_ptr, pair_p, pair_q;
};

// Checks CSR structure; square/diag requirements only when asked.
bool validate_csr(const HostCSR& M, bool square_with_diag, std::string& why);

HostCSR transpose(const HostCSR& M);

// Classical RS first pass with strength threshold theta; split[i] = 1 for C.
void rs_split(const HostCSR& A, double theta, std::vector<int>& split,
              std::vector<int>& S_rp, std::vector<int>& S_col);

HostCSR direct_interpolation(const HostCSR& A, const std::vector<int>& S_rp,
                             const std::vector<int>& S_col, const std::vector<int>& split);

// A_c = P^T A P on the structural pattern of the product.
HostCSR galerkin(const HostCSR& A, const HostCSR& P, const HostCSR& R);

// Row-by-row sparse product X Y keeping the structural pattern.
HostCSR spgemm(const HostCSR &X, const HostCSR &Y);

// Largest eigenvalue of D^-1 A by n_power power iterations (FP64):
// v0_i = frac(i 2654435761 / 2^32) + 0.5 normalised, w = D^-1 A v,
// estimate = ||w|| of the last iteration, v = w / ||w||.
double power_estimate(const HostCSR &A, int n_power);

// Setup-AMG-Hierarchy of Algorithm 1 (finest level first).
void build_hierarchy(const HostCSR& A0, double theta, int max_levels, int max_coarse,
                     std::vector<HostLevel>& levels);

}  // namespace amg
