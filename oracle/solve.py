"""AMG solve phase in plain FP64 (torch CPU ops, differentiable).

Test infrastructure only.  Every sparse product is written out as its
definition, y_i = sum_j m_ij x_j, with a gather and an index_add, so that
autograd can differentiate through the smoother's values (Sec. 3.3).

* Sec. 2.1: stationary correction u <- u + Q^-1 (f - A u).
* Sec. 2.3: relaxed Jacobi, Q^-1 = omega D^-1.
* Sec. 3.1: sparse pseudo-inverse smoother with A's pattern,
  q_ii^-1 = f_d(a_ii/s)/a_ii, q_ij^-1 = f_o(a_ij/s)/(a_ii + a_jj),
  s = max |A - D|, f_d(x) = c0 + c1 x + c2 x^2, f_o(x) = c3 x + c4 x^2
  (coefficient order (d0, d1, d2, o1, o2) is a reading; the paper fixes
  only "3 for f_d, 2 for f_o").
* Sec. 2.2: V-cycle: nu1 pre-sweeps, restriction of the residual with R,
  recursion with a zero initial guess, prolongation with P, nu2 post-sweeps;
  the coarsest level is solved by a dense Cholesky factorisation.
* Sec. 4: stop when ||f - A u||_2 / ||f||_2 <= tol (relative to ||f||: a
  reading) or after max_iter cycles; diverged when a norm is not finite or
  exceeds 1e3 times the initial one; stagnated when the smallest norm of
  the last 10 cycles is not 1% below the smallest of the 10 before them
  (a window of minima: a stationary V-cycle need not reduce the 2-norm
  monotonically, and from a warm start the first cycles can raise it).
* Sec. 3.3: the relative validation metric
  log10(||r_{n+1}|| / ||r^{omega-J}_{n+1}||) after one cycle from the same
  state.
* Chebyshev baseline smoother (not in the paper; the fixed-coefficient
  polynomial the learned smoother is compared with): one application of the
  degree-k Chebyshev polynomial in D^-1 A per smoothing phase, on the interval
  [rho/30, 1.1 rho] with rho from 20 power iterations on D^-1 A started from
  v_i = frac(i * 2654435761 / 2^32) + 0.5; the classical three-term
  recurrence theta = (hi + lo)/2, delta = (hi - lo)/2, sigma = theta/delta:
  d = D^-1 r / theta, then d <- rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r
  with rho_0 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1}), u <- u + d.
* Krylov outer loop (the Krylov form of the Sec. 2.1 correction): conjugate
  gradients on A u = f preconditioned by one V-cycle from a zero guess
  (symmetric for a symmetric smoother), with the flexible coefficient
  beta = z_k . (r_k - r_{k-1}) / (z_{k-1} . r_{k-1}), which equals the
  classical z_k . r_k / (z_{k-1} . r_{k-1}) for a fixed symmetric
  preconditioner and keeps a slightly non-symmetric one (an FP32 V-cycle)
  convergent.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from workloads import CSR

DT = torch.float64

OK, DIVERGED, STAGNATED, MAXITER = 0, -4, -5, -6


@dataclass
class TMat:
    """A sparse matrix as (row, col, val) triples in torch FP64."""
    n_rows: int
    n_cols: int
    row: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor

    @staticmethod
    def of(M: CSR) -> "TMat":
        row = torch.from_numpy(np.repeat(np.arange(M.n_rows), np.diff(M.row_ptr)).astype(np.int64))
        return TMat(M.n_rows, M.n_cols, row, torch.from_numpy(M.col.astype(np.int64)),
                    torch.from_numpy(M.val.astype(np.float64)))

    def diag(self) -> torch.Tensor:
        d = torch.zeros(self.n_rows, dtype=DT)
        on = self.row == self.col
        return d.index_add(0, self.row[on], self.val[on])


def matvec(row, col, val, x, n_rows) -> torch.Tensor:
    """y_i = sum_j m_ij x_j."""
    return torch.zeros(n_rows, dtype=DT).index_add(0, row, val * x[col])


def mv(M: TMat, x: torch.Tensor) -> torch.Tensor:
    return matvec(M.row, M.col, M.val, x, M.n_rows)


# ----------------------------------------------------------------------------
# smoothers (Sec. 2.3, Sec. 3.1)
# ----------------------------------------------------------------------------
def smoother_scale(A: TMat) -> float:
    """s = max |A - D| (largest off-diagonal magnitude)."""
    off = A.row != A.col
    return float(A.val[off].abs().max()) if bool(off.any()) else 1.0


def pseudo_inverse_values(A: TMat, c, s: float | None = None) -> torch.Tensor:
    """Values of Q^-1 on A's pattern for coefficients c = (d0, d1, d2, o1, o2)."""
    if s is None:
        s = smoother_scale(A)
    d = A.diag()
    x = A.val / s
    on = A.row == A.col
    f_d = c[0] + c[1] * x + c[2] * x * x
    f_o = c[3] * x + c[4] * x * x
    q_diag = f_d / d[A.row]
    q_off = f_o / (d[A.row] + d[A.col])
    return torch.where(on, q_diag, q_off)


def pseudo_inverse_values_nodes(A: TMat, C, s: float | None = None) -> torch.Tensor:
    """Q^-1 with one coefficient row per node, C (n x 5): the diagonal entry of
    row i uses node i's (d0, d1, d2); an off-diagonal entry (i, j) uses the
    mean of nodes i's and j's (o1, o2), so Q^-1 stays symmetric (reading: the
    paper's coefficients are per level; equal rows reduce to that form)."""
    if s is None:
        s = smoother_scale(A)
    C = torch.as_tensor(np.asarray(C, dtype=np.float64))
    d = A.diag()
    x = A.val / s
    on = A.row == A.col
    ci, cj = C[A.row], C[A.col]
    f_d = ci[:, 0] + ci[:, 1] * x + ci[:, 2] * x * x
    o1 = (ci[:, 3] + cj[:, 3]) / 2.0
    o2 = (ci[:, 4] + cj[:, 4]) / 2.0
    f_o = o1 * x + o2 * x * x
    return torch.where(on, f_d / d[A.row], f_o / (d[A.row] + d[A.col]))


def jacobi_values(A: TMat, omega: float) -> torch.Tensor:
    """Values of omega D^-1 on A's pattern (zero off the diagonal)."""
    d = A.diag()
    on = A.row == A.col
    return torch.where(on, torch.full_like(A.val, omega) / d[A.row], torch.zeros_like(A.val))


# ----------------------------------------------------------------------------
# coarsest level: dense Cholesky
# ----------------------------------------------------------------------------
def cholesky(Ad: np.ndarray) -> np.ndarray:
    """Lower-triangular L with L L^T = Ad, column by column."""
    n = Ad.shape[0]
    L = np.zeros_like(Ad)
    for j in range(n):
        djj = Ad[j, j] - L[j, :j] @ L[j, :j]
        if not djj > 0.0:
            raise np.linalg.LinAlgError("coarsest matrix is not positive definite")
        L[j, j] = math.sqrt(djj)
        L[j + 1:, j] = (Ad[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def cholesky_solve(L: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Solve L L^T x = b by forward then backward substitution."""
    n = L.shape[0]
    y = []
    for i in range(n):
        acc = b[i] - (L[i, :i] @ torch.stack(y) if i else 0.0)
        y.append(acc / L[i, i])
    y = torch.stack(y)
    x = [None] * n
    for i in reversed(range(n)):
        acc = y[i] - (L[i + 1:, i] @ torch.stack(x[i + 1:]) if i < n - 1 else 0.0)
        x[i] = acc / L[i, i]
    return torch.stack(x)


# ----------------------------------------------------------------------------
# hierarchy with smoothers
# ----------------------------------------------------------------------------
@dataclass
class OLevel:
    A: TMat
    P: TMat | None
    R: TMat | None
    M: torch.Tensor | None = None      # smoother values on A's pattern
    L: torch.Tensor | None = None      # Cholesky factor on the coarsest level
    s: float = 1.0
    cheb: tuple | None = None          # Chebyshev smoother: (theta, delta, degree, D^-1)


@dataclass
class OHierarchy:
    levels: list = field(default_factory=list)

    @staticmethod
    def of(setup_levels) -> "OHierarchy":
        h = OHierarchy()
        for k, lv in enumerate(setup_levels):
            A = TMat.of(lv.A)
            P = TMat.of(lv.P) if lv.P is not None else None
            R = TMat.of(lv.R) if lv.R is not None else None
            ol = OLevel(A, P, R, s=smoother_scale(A))
            if k == len(setup_levels) - 1:
                ol.L = torch.from_numpy(cholesky(lv.A.to_dense()))
            h.levels.append(ol)
        return h

    def set_jacobi(self, omega: float = 2.0 / 3.0):
        for lv in self.levels[:-1]:
            lv.M = jacobi_values(lv.A, omega)
            lv.cheb = None

    def set_pseudo_inverse(self, coeffs):
        """coeffs[l] = (d0, d1, d2, o1, o2) for level l (rows past the last smoothed level unused)."""
        for l, lv in enumerate(self.levels[:-1]):
            lv.M = pseudo_inverse_values(lv.A, coeffs[l], lv.s)
            lv.cheb = None

    def set_pseudo_inverse_nodes(self, node_coeffs):
        """node_coeffs[l] = (n_l x 5) per-node coefficients of level l."""
        for l, lv in enumerate(self.levels[:-1]):
            lv.M = pseudo_inverse_values_nodes(lv.A, node_coeffs[l], lv.s)
            lv.cheb = None

    def set_chebyshev(self, degree: int = 3, lo: float = 1.0 / 30.0, hi: float = 1.1, n_power: int = 20):
        for lv in self.levels[:-1]:
            rho = power_estimate(lv.A, n_power)
            dinv = 1.0 / diagonal(lv.A)
            a, b = lo * rho, hi * rho
            lv.cheb = ((b + a) / 2.0, (b - a) / 2.0, degree, dinv)
            lv.M = None


def diagonal(A: TMat) -> torch.Tensor:
    on = A.row == A.col
    return torch.zeros(A.n_rows, dtype=DT).index_add(0, A.row[on], A.val[on])


def power_start(n: int) -> torch.Tensor:
    """v_i = frac(i * 2654435761 / 2^32) + 0.5 (a fixed, RNG-free start vector)."""
    i = np.arange(n, dtype=np.uint64)
    return torch.from_numpy(((i * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.float64) / 2.0 ** 32 + 0.5)


def power_estimate(A: TMat, n_power: int = 20) -> float:
    """Largest eigenvalue of D^-1 A by n_power power iterations: v <- w / ||w||,
    w = D^-1 A v; the estimate is ||w|| of the last iteration."""
    dinv = 1.0 / diagonal(A)
    v = power_start(A.n_rows)
    v = v / torch.linalg.vector_norm(v)
    lam = 0.0
    for _ in range(n_power):
        w = dinv * mv(A, v)
        lam = float(torch.linalg.vector_norm(w))
        v = w / lam
    return lam


def cheb_smooth(lv: OLevel, b: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """One application of the degree-k Chebyshev polynomial smoother."""
    theta, delta, degree, dinv = lv.cheb
    sigma = theta / delta
    rho_prev = 1.0 / sigma
    r = b - mv(lv.A, u)
    d = dinv * r / theta
    u = u + d
    for _ in range(degree - 1):
        r = b - mv(lv.A, u)
        rho = 1.0 / (2.0 * sigma - rho_prev)
        d = (rho * rho_prev) * d + (2.0 * rho / delta) * (dinv * r)
        u = u + d
        rho_prev = rho
    return u


def sweep(lv: OLevel, b: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """One stationary smoothing step u + Q^-1 (b - A u)."""
    r = b - mv(lv.A, u)
    return u + matvec(lv.A.row, lv.A.col, lv.M, r, lv.A.n_rows)


def vcycle(h: OHierarchy, b: torch.Tensor, u: torch.Tensor, nu1: int = 2, nu2: int = 2, l: int = 0):
    """One V-cycle on level l for A_l u = b starting from u."""
    lv = h.levels[l]
    if l == len(h.levels) - 1:
        return cholesky_solve(lv.L, b)
    if lv.cheb is not None:
        u = cheb_smooth(lv, b, u)          # one polynomial application per phase
    else:
        for _ in range(nu1):
            u = sweep(lv, b, u)
    r = b - mv(lv.A, u)
    bc = mv(lv.R, r)
    ec = vcycle(h, bc, torch.zeros(lv.R.n_rows, dtype=DT), nu1, nu2, l + 1)
    u = u + mv(lv.P, ec)
    if lv.cheb is not None:
        u = cheb_smooth(lv, b, u)
    else:
        for _ in range(nu2):
            u = sweep(lv, b, u)
    return u


@dataclass
class SolveResult:
    x: np.ndarray
    history: list
    n_vcycles: int
    status: int


def solve(h: OHierarchy, f, tol: float = 1e-8, max_iter: int = 500, u0=None,
          nu1: int = 2, nu2: int = 2) -> SolveResult:
    """Stationary V-cycle iteration to ||f - A u|| / ||f|| <= tol."""
    f = torch.as_tensor(np.asarray(f, dtype=np.float64))
    A = h.levels[0].A
    u = torch.zeros(A.n_rows, dtype=DT) if u0 is None else torch.as_tensor(np.asarray(u0, dtype=np.float64)).clone()
    fnorm = float(torch.linalg.vector_norm(f))
    if fnorm == 0.0:
        fnorm = 1.0
    r0 = float(torch.linalg.vector_norm(f - mv(A, u)))
    hist = [r0 / fnorm]
    status = MAXITER
    if hist[0] <= tol:
        return SolveResult(u.numpy(), hist, 0, OK)
    k = 0
    with torch.no_grad():
        while k < max_iter:
            u = vcycle(h, f, u, nu1, nu2)
            k += 1
            rn = float(torch.linalg.vector_norm(f - mv(A, u)))
            hist.append(rn / fnorm)
            if not math.isfinite(rn) or rn > 1e3 * r0:
                status = DIVERGED
                break
            if hist[-1] <= tol:
                status = OK
                break
            if k >= 20 and min(hist[-10:]) > 0.99 * min(hist[-20:-10]):
                status = STAGNATED
                break
    return SolveResult(u.numpy(), hist, k, status)


def solve_pcg(h: OHierarchy, f, tol: float = 1e-8, max_iter: int = 500, u0=None, nu1: int = 2, nu2: int = 2,
              precond=None) -> SolveResult:
    """Preconditioned conjugate gradients to ||r|| / ||f|| <= tol (FP64).

    precond(r) -> z defaults to one V-cycle from a zero initial guess.  The
    history holds the recurrence residual r_{k+1} = r_k - alpha q_k relative
    to ||f||; statuses as in solve(), and DIVERGED also on a breakdown
    (z . r <= 0 or p . A p <= 0: the preconditioned operator is not SPD),
    which leaves the iterate and the history as they were.
    """
    f = torch.as_tensor(np.asarray(f, dtype=np.float64))
    A = h.levels[0].A
    if precond is None:
        def precond(r):
            with torch.no_grad():
                return vcycle(h, r, torch.zeros_like(r), nu1, nu2)
    u = torch.zeros(A.n_rows, dtype=DT) if u0 is None else torch.as_tensor(np.asarray(u0, dtype=np.float64)).clone()
    fnorm = float(torch.linalg.vector_norm(f))
    if fnorm == 0.0:
        fnorm = 1.0
    r = f - mv(A, u)
    r0 = float(torch.linalg.vector_norm(r))
    hist = [r0 / fnorm]
    if hist[0] <= tol:
        return SolveResult(u.numpy(), hist, 0, OK)
    status, k = MAXITER, 0
    p = r_prev = rho_prev = None
    with torch.no_grad():
        while k < max_iter:
            z = precond(r)
            rho = float(torch.dot(z, r))
            if p is None:
                p = z.clone()
            else:
                beta = float(torch.dot(z, r - r_prev)) / rho_prev
                p = z + beta * p
            q = mv(A, p)
            pq = float(torch.dot(p, q))
            if not (math.isfinite(rho) and math.isfinite(pq) and rho > 0.0 and pq > 0.0):
                status = DIVERGED          # breakdown: the iterate and history stay as they were
                break
            k += 1
            alpha = rho / pq
            u = u + alpha * p
            r_prev, rho_prev = r, rho
            r = r - alpha * q
            rn = float(torch.linalg.vector_norm(r))
            hist.append(rn / fnorm)
            if not math.isfinite(rn) or rn > 1e3 * r0:
                status = DIVERGED
                break
            if hist[-1] <= tol:
                status = OK
                break
            if k >= 20 and min(hist[-10:]) > 0.99 * min(hist[-20:-10]):
                status = STAGNATED
                break
    return SolveResult(u.numpy(), hist, k, status)


def vcycle_operator_apply(h: OHierarchy, r, nu1: int = 2, nu2: int = 2) -> np.ndarray:
    """B r: one V-cycle from a zero initial guess (the preconditioner's action)."""
    r = torch.as_tensor(np.asarray(r, dtype=np.float64))
    with torch.no_grad():
        return vcycle(h, r, torch.zeros_like(r), nu1, nu2).numpy()


def relative_metric(h_gnn: OHierarchy, h_jac: OHierarchy, f, u0=None, nu1=2, nu2=2, n_cycles: int = 1) -> float:
    """log10(||r_n|| / ||r^{omega-J}_n||) after n_cycles V-cycles from u0 (Sec. 3.3).

    The paper's metric compares the residuals after cycle n+1; n_cycles
    chooses that cycle.  A non-finite GNN residual gives +inf.
    """
    f = torch.as_tensor(np.asarray(f, dtype=np.float64))
    u = torch.zeros_like(f) if u0 is None else torch.as_tensor(np.asarray(u0, dtype=np.float64))
    with torch.no_grad():
        ug, uj = u.clone(), u.clone()
        for _ in range(n_cycles):
            ug = vcycle(h_gnn, f, ug, nu1, nu2)
            uj = vcycle(h_jac, f, uj, nu1, nu2)
        rg = torch.linalg.vector_norm(f - mv(h_gnn.levels[0].A, ug))
        rj = torch.linalg.vector_norm(f - mv(h_jac.levels[0].A, uj))
    if not bool(torch.isfinite(rg)):
        return math.inf
    return float(torch.log10(rg / rj))
