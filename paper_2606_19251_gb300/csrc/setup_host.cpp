// Host-side AMG setup (Sec. 2.2; Algorithm 1 step 2).
//
// Classical Ruge-Stueben with strength threshold theta (Sec. 4: 0.25):
//   j is a strong dependency of i  iff  j != i and -a_ij >= theta max_{k!=i} (-a_ik)
// First pass only: points without strong connections in either direction
// are F; then the undecided point of largest measure (ties: lowest index)
// becomes C and its undecided strong dependents become F.  The measure is
// |S^T cap U| + 2 |S^T cap F|, kept up to date incrementally.
// Direct interpolation for F rows: w_ij = -alpha_i a_ij / d_i over the strong
// C neighbours, alpha_i = (sum of negative off-diagonals) / (sum of negative
// strong-C couplings), d_i = a_ii + sum of positive off-diagonals.
// Galerkin A_c = R A P with R = P^T keeps the structural product pattern.
#include "setup_host.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <queue>
#include <utility>

namespace amg {

bool validate_csr(const HostCSR& M, bool square_with_diag, std::string& why) {
    if (M.n_rows < 0 || M.n_cols < 0) { why = "negative dimension"; return false; }
    if (static_cast<int>(M.rp.size()) != M.n_rows + 1) { why = "row_ptr has wrong length"; return false; }
    if (M.rp[0] != 0) { why = "row_ptr[0] != 0"; return false; }
    for (int i = 0; i < M.n_rows; ++i)
        if (M.rp[i + 1] < M.rp[i]) { why = "row_ptr not monotone"; return false; }
    if (static_cast<long long>(M.rp[M.n_rows]) != M.nnz() || M.val.size() != M.col.size()) {
        why = "row_ptr[n] != nnz"; return false;
    }
    for (int i = 0; i < M.n_rows; ++i) {
        bool diag = false;
        for (int p = M.rp[i]; p < M.rp[i + 1]; ++p) {
            int j = M.col[p];
            if (j < 0 || j >= M.n_cols) { why = "column index out of range"; return false; }
            if (p > M.rp[i] && M.col[p - 1] >= j) { why = "columns not strictly ascending"; return false; }
            if (j == i) diag = true;
        }
        if (square_with_diag && !diag) { why = "missing diagonal entry"; return false; }
    }
    if (square_with_diag && M.n_rows != M.n_cols) { why = "matrix not square"; return false; }
    return true;
}

HostCSR transpose(const HostCSR& M) {
    HostCSR T;
    T.n_rows = M.n_cols;
    T.n_cols = M.n_rows;
    T.rp.assign(T.n_rows + 1, 0);
    for (int j : M.col) T.rp[j + 1]++;
    for (int i = 0; i < T.n_rows; ++i) T.rp[i + 1] += T.rp[i];
    T.col.resize(M.col.size());
    T.val.resize(M.col.size());
    std::vector<int> next(T.rp.begin(), T.rp.end() - 1);
    for (int i = 0; i < M.n_rows; ++i)
        for (int p = M.rp[i]; p < M.rp[i + 1]; ++p) {
            int q = next[M.col[p]]++;
            T.col[q] = i;
            T.val[q] = M.val[p];
        }
    return T;
}

void rs_split(const HostCSR& A, double theta, std::vector<int>& split,
              std::vector<int>& S_rp, std::vector<int>& S_col) {
    const int n = A.n_rows;
    // strong dependencies S_i (ascending columns)
    S_rp.assign(n + 1, 0);
    S_col.clear();
    for (int i = 0; i < n; ++i) {
        bool has_off = false;
        double m = 0.0;
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
            if (A.col[p] == i) continue;
            double neg = -A.val[p];
            if (!has_off || neg > m) m = neg;
            has_off = true;
        }
        if (has_off && m > 0.0) {
            const double thr = theta * m;
            for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
                if (A.col[p] != i && -A.val[p] >= thr) S_col.push_back(A.col[p]);
        }
        S_rp[i + 1] = static_cast<int>(S_col.size());
    }
    // S^T: points strongly depending on i
    std::vector<int> T_rp(n + 1, 0), T_col(S_col.size());
    for (int j : S_col) T_rp[j + 1]++;
    for (int i = 0; i < n; ++i) T_rp[i + 1] += T_rp[i];
    {
        std::vector<int> next(T_rp.begin(), T_rp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int p = S_rp[i]; p < S_rp[i + 1]; ++p) T_col[next[S_col[p]]++] = i;
    }
    enum : int { F = 0, C = 1, U = -1 };
    std::vector<int> state(n, U);
    std::vector<long long> lam(n);
    for (int i = 0; i < n; ++i) {
        lam[i] = T_rp[i + 1] - T_rp[i];
        if (S_rp[i + 1] == S_rp[i] && T_rp[i + 1] == T_rp[i]) state[i] = F;
    }
    // max-heap on (lambda, -index): top = largest measure, lowest index
    using Key = std::pair<long long, int>;
    std::priority_queue<Key> heap;
    for (int i = 0; i < n; ++i)
        if (state[i] == U) heap.push(Key(lam[i], -i));
    while (!heap.empty()) {
        Key top = heap.top();
        heap.pop();
        const int i = -top.second;
        if (state[i] != U || top.first != lam[i]) continue;   // stale entry
        state[i] = C;
        for (int p = T_rp[i]; p < T_rp[i + 1]; ++p) {
            const int j = T_col[p];
            if (state[j] != U) continue;
            state[j] = F;
            for (int q = S_rp[j]; q < S_rp[j + 1]; ++q) {
                const int k = S_col[q];
                if (state[k] == U) heap.push(Key(++lam[k], -k));
            }
        }
        for (int q = S_rp[i]; q < S_rp[i + 1]; ++q) {
            const int k = S_col[q];
            if (state[k] == U) heap.push(Key(--lam[k], -k));
        }
    }
    split.assign(n, 0);
    for (int i = 0; i < n; ++i) split[i] = (state[i] == C) ? 1 : 0;
}

HostCSR direct_interpolation(const HostCSR& A, const std::vector<int>& S_rp,
                             const std::vector<int>& S_col, const std::vector<int>& split) {
    const int n = A.n_rows;
    std::vector<int> cidx(n, -1);
    int nc = 0;
    for (int i = 0; i < n; ++i)
        if (split[i]) cidx[i] = nc++;
    HostCSR P;
    P.n_rows = n;
    P.n_cols = nc;
    P.rp.assign(n + 1, 0);
    std::vector<char> strong_c(n, 0);
    for (int i = 0; i < n; ++i) {
        if (split[i]) {
            P.col.push_back(cidx[i]);
            P.val.push_back(1.0);
            P.rp[i + 1] = static_cast<int>(P.col.size());
            continue;
        }
        bool any = false;
        for (int q = S_rp[i]; q < S_rp[i + 1]; ++q)
            if (split[S_col[q]]) { strong_c[S_col[q]] = 1; any = true; }
        if (any) {
            double a_ii = 0.0, neg_all = 0.0, pos_all = 0.0, neg_c = 0.0;
            for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
                const int j = A.col[p];
                const double a = A.val[p];
                if (j == i) {
                    a_ii += a;
                } else if (a < 0.0) {
                    neg_all += a;
                    if (strong_c[j]) neg_c += a;
                } else if (a > 0.0) {
                    pos_all += a;
                }
            }
            const double d = a_ii + pos_all;
            const double alpha = neg_all / neg_c;
            for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
                const int j = A.col[p];
                if (j != i && strong_c[j]) {
                    P.col.push_back(cidx[j]);
                    P.val.push_back(-alpha * A.val[p] / d);
                }
            }
            for (int q = S_rp[i]; q < S_rp[i + 1]; ++q) strong_c[S_col[q]] = 0;
        }
        P.rp[i + 1] = static_cast<int>(P.col.size());
    }
    return P;
}

// Row-by-row sparse product C = X Y keeping the structural pattern.
HostCSR spgemm(const HostCSR& X, const HostCSR& Y) {
    HostCSR C;
    C.n_rows = X.n_rows;
    C.n_cols = Y.n_cols;
    C.rp.assign(C.n_rows + 1, 0);
    std::vector<int> mark(Y.n_cols, -1);
    std::vector<double> acc(Y.n_cols, 0.0);
    std::vector<int> cols;
    for (int i = 0; i < X.n_rows; ++i) {
        cols.clear();
        for (int p = X.rp[i]; p < X.rp[i + 1]; ++p) {
            const int k = X.col[p];
            const double x = X.val[p];
            for (int q = Y.rp[k]; q < Y.rp[k + 1]; ++q) {
                const int j = Y.col[q];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    cols.push_back(j);
                }
                acc[j] += x * Y.val[q];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int j : cols) {
            C.col.push_back(j);
            C.val.push_back(acc[j]);
        }
        C.rp[i + 1] = static_cast<int>(C.col.size());
    }
    return C;
}

HostCSR galerkin(const HostCSR& A, const HostCSR& P, const HostCSR& R) {
    return spgemm(R, spgemm(A, P));
}

void build_hierarchy(const HostCSR& A0, double theta, int max_levels, int max_coarse,
                     std::vector<HostLevel>& levels) {
    levels.clear();
    levels.emplace_back();
    levels.back().A = A0;
    while (static_cast<int>(levels.size()) < max_levels && levels.back().A.n_rows > max_coarse) {
        const HostCSR& A = levels.back().A;
        std::vector<int> split, S_rp, S_col;
        rs_split(A, theta, split, S_rp, S_col);
        long long nc = 0;
        for (int v : split) nc += v;
        if (nc == 0 || static_cast<double>(nc) > 0.9 * A.n_rows) break;
        HostLevel& L = levels.back();
        L.P = direct_interpolation(A, S_rp, S_col, split);
        L.R = transpose(L.P);
        HostCSR Ac = galerkin(L.A, L.P, L.R);
        levels.emplace_back();
        levels.back().A = std::move(Ac);
    }
}

double power_estimate(const HostCSR &A, int n_power) {
    const int n = A.n_rows;
    if (n <= 0) return 0.0;
    std::vector<double> dinv(n, 0.0), v(n), w(n);
    for (int i = 0; i < n; ++i)
        for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
            if (A.col[p] == i) dinv[i] += A.val[p];
    for (int i = 0; i < n; ++i) dinv[i] = 1.0 / dinv[i];
    double nv = 0.0;
    for (int i = 0; i < n; ++i) {
        const uint32_t h = static_cast<uint32_t>(static_cast<uint64_t>(i) * 2654435761ull);
        v[i] = static_cast<double>(h) / 4294967296.0 + 0.5;
        nv += v[i] * v[i];
    }
    nv = std::sqrt(nv);
    for (int i = 0; i < n; ++i) v[i] /= nv;
    double lam = 0.0;
    for (int it = 0; it < n_power; ++it) {
        double nw = 0.0;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) acc += A.val[p] * v[A.col[p]];
            w[i] = dinv[i] * acc;
            nw += w[i] * w[i];
        }
        lam = std::sqrt(nw);
        for (int i = 0; i < n; ++i) v[i] = w[i] / lam;
    }
    return lam;
}

}  // namespace amg
