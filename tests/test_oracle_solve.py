"""Pins for the oracle's solve phase: SpMV, Jacobi, pseudo-inverse smoother,
Cholesky, V-cycle, stopping rule.  Closed forms (5-point eigenpairs),
hand-worked values (tests/golden), library routines (numpy LU) and algebraic
invariants (symmetry, linearity)."""
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import setup as S
from oracle import solve as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def eigvec(m, j, k):
    h = 1.0 / (m + 1)
    x = np.arange(1, m + 1) * h
    return np.outer(np.sin(j * np.pi * x), np.sin(k * np.pi * x)).ravel(), 4 - 2 * np.cos(j * np.pi * h) - 2 * np.cos(k * np.pi * h)


@pytest.mark.parametrize("j,k", [(1, 1), (3, 7), (32, 5), (64, 64)])
def test_spmv_5point_eigenpairs(j, k):
    m = 64
    A = O.TMat.of(W.poisson5(m))
    v, lam = eigvec(m, j, k)
    Av = O.mv(A, torch.from_numpy(v)).numpy()
    np.testing.assert_allclose(Av, lam * v, atol=1e-13)


@pytest.mark.parametrize("j,k", [(1, 1), (20, 40), (64, 64)])
def test_jacobi_damps_eigenvector_by_closed_form(j, k):
    # one relaxed-Jacobi step on A u = 0 multiplies an eigenvector by 1 - omega*lambda/4
    m, omega = 64, 2.0 / 3.0
    A = O.TMat.of(W.poisson5(m))
    lv = O.OLevel(A, None, None, M=O.jacobi_values(A, omega))
    v, lam = eigvec(m, j, k)
    u1 = O.sweep(lv, torch.zeros(m * m, dtype=torch.float64), torch.from_numpy(v)).numpy()
    np.testing.assert_allclose(u1, (1 - omega * lam / 4) * v, atol=1e-14)


def test_pseudo_inverse_hand_worked():
    A = W._coo_to_csr(3, 3, np.array([0, 0, 1, 1, 1, 2, 2]), np.array([0, 1, 0, 1, 2, 1, 2]),
                      np.array([2.0, -1, -1, 3, -2, -2, 4]))
    T = O.TMat.of(A)
    assert O.smoother_scale(T) == 2.0
    q = O.pseudo_inverse_values(T, [1.0, 0.5, 0.25, 0.3, 0.1]).numpy()
    rows = np.loadtxt(os.path.join(GOLDEN, "pinv_3x3.txt"), comments="#")
    got = {(int(r), int(c)): v for r, c, v in zip(T.row.numpy(), T.col.numpy(), q)}
    for r, c, v in rows:
        assert abs(got[(int(r), int(c))] - v) < 1e-15


def test_degree_one_coefficients_reproduce_jacobi():
    A = O.TMat.of(W.fv_mesh("graded", 3000, 1)[0])
    omega = 2.0 / 3.0
    np.testing.assert_array_equal(O.pseudo_inverse_values(A, [omega, 0, 0, 0, 0]).numpy(),
                                  O.jacobi_values(A, omega).numpy())


def test_pseudo_inverse_symmetric_and_pattern():
    Acsr = W.fv_mesh("band", 2000, 4, max_aspect=100.0)[0]
    A = O.TMat.of(Acsr)
    q = O.pseudo_inverse_values(A, [0.7, -0.1, 0.02, 0.3, -0.05])
    Q = W.CSR(Acsr.n_rows, Acsr.n_cols, Acsr.row_ptr, Acsr.col, q.numpy()).to_dense()
    np.testing.assert_allclose(Q, Q.T, rtol=0, atol=1e-15)
    # f_o(0) = 0: entries where a_ij = 0 stay zero
    Ad = Acsr.to_dense()
    assert np.all(Q[Ad == 0] == 0)


def test_node_coefficients_hand_worked():
    # tridiag(-1, 2, -1) on 3 points, s = 1: x_ii = 2, x_ij = -1.  Nodes carry
    # (d0, d1, d2, o1, o2) = (1,0,0,1,0), (0,1,0,3,0), (0,0,1,0,2):
    # q_00 = 1/2, q_11 = 2/2, q_22 = 4/2; q_01 = ((1+3)/2 * -1) / 4 = -1/2;
    # q_12 = ((3+0)/2 * -1 + (0+2)/2 * 1) / 4 = -1/8 (the same by symmetry)
    A = W._coo_to_csr(3, 3, np.array([0, 0, 1, 1, 1, 2, 2]), np.array([0, 1, 0, 1, 2, 1, 2]),
                      np.array([2.0, -1, -1, 2, -1, -1, 2]))
    T = O.TMat.of(A)
    C = [[1, 0, 0, 1, 0], [0, 1, 0, 3, 0], [0, 0, 1, 0, 2]]
    q = O.pseudo_inverse_values_nodes(T, C).numpy()
    expect = {(0, 0): 0.5, (0, 1): -0.5, (1, 0): -0.5, (1, 1): 1.0, (1, 2): -0.125, (2, 1): -0.125, (2, 2): 2.0}
    for r, c, v in zip(T.row.numpy(), T.col.numpy(), q):
        assert v == expect[(int(r), int(c))]


def test_node_coefficients_reduce_to_level_form_and_stay_symmetric():
    Acsr = W.fv_mesh("band", 2000, 4, max_aspect=100.0)[0]
    A = O.TMat.of(Acsr)
    c = [0.7, -0.1, 0.02, 0.3, -0.05]
    same = np.tile(c, (Acsr.n_rows, 1))
    assert torch.equal(O.pseudo_inverse_values_nodes(A, same), O.pseudo_inverse_values(A, c))
    C = same + 0.1 * W.uniform_pm1(5, 5 * Acsr.n_rows).reshape(-1, 5)
    q = O.pseudo_inverse_values_nodes(A, C)
    Q = W.CSR(Acsr.n_rows, Acsr.n_cols, Acsr.row_ptr, Acsr.col, q.numpy()).to_dense()
    np.testing.assert_allclose(Q, Q.T, rtol=0, atol=1e-15)
    assert not torch.equal(q, O.pseudo_inverse_values(A, c))


def test_cholesky_against_library_solve():
    A = W.fv_mesh("uniform", 200, 9)[0]
    Ad = A.to_dense()
    L = O.cholesky(Ad)
    np.testing.assert_allclose(L @ L.T, Ad, atol=1e-13 * np.abs(Ad).max())
    assert np.all(np.triu(L, 1) == 0)
    b = W.rhs_uniform(3, A.n_rows)
    x = O.cholesky_solve(torch.from_numpy(L), torch.from_numpy(b)).numpy()
    np.testing.assert_allclose(x, np.linalg.solve(Ad, b), rtol=1e-11, atol=1e-12)


def _hier(A, smoother="jacobi", coeffs=None, **kw):
    lv = S.build_hierarchy(A, **kw)
    h = O.OHierarchy.of(lv)
    if smoother == "jacobi":
        h.set_jacobi()
    else:
        h.set_pseudo_inverse([coeffs] * len(lv))
    return h


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_vcycle_operator_is_symmetric(smoother):
    # nu1 = nu2 with a symmetric smoother makes the V-cycle preconditioner B
    # symmetric: <B x, y> = <x, B y>.
    A = W.fv_mesh("graded", 3000, 2)[0]
    h = _hier(A, smoother, [0.6, 0.05, -0.01, 0.2, 0.03])
    x = W.rhs_uniform(1, A.n_rows)
    y = W.rhs_uniform(2, A.n_rows)
    Bx, By = O.vcycle_operator_apply(h, x), O.vcycle_operator_apply(h, y)
    lhs, rhs = Bx @ y, x @ By
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_vcycle_is_linear_in_b():
    A = W.poisson5(32)
    h = _hier(A, "pinv", [0.6, 0.05, -0.01, 0.2, 0.03])
    x, y = W.rhs_uniform(1, A.n_rows), W.rhs_uniform(2, A.n_rows)
    lhs = O.vcycle_operator_apply(h, 2.5 * x - 0.75 * y)
    rhs = 2.5 * O.vcycle_operator_apply(h, x) - 0.75 * O.vcycle_operator_apply(h, y)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(rhs).max())


@pytest.mark.parametrize("case", ["grid16", "delaunay300"])
def test_converged_solution_equals_dense_direct_solve(case):
    A = W.poisson5(16) if case == "grid16" else W.fv_mesh("graded", 300, 7)[0]
    h = _hier(A, max_coarse=8)
    assert len(h.levels) >= 3
    b = W.rhs_uniform(4, A.n_rows)
    res = O.solve(h, b, tol=1e-13, max_iter=200)
    assert res.status == O.OK
    np.testing.assert_allclose(res.x, np.linalg.solve(A.to_dense(), b), rtol=0,
                               atol=1e-11 * np.abs(np.linalg.solve(A.to_dense(), b)).max())


def test_single_level_vcycle_is_exact():
    A = W.poisson5(6)
    h = _hier(A)
    assert len(h.levels) == 1
    b = W.rhs_uniform(5, A.n_rows)
    res = O.solve(h, b, tol=1e-12)
    assert res.n_vcycles == 1 and res.history[-1] < 1e-14


def test_c1_jacobi_amg_converges_fast():
    # RS AMG with omega-Jacobi (2+2 sweeps) on the 5-point Laplacian is a
    # textbook fast solver: 1e-8 in well under 15 cycles.
    A = W.poisson5(64)
    h = _hier(A)
    res = O.solve(h, W.rhs_uniform(0, A.n_rows), tol=1e-8)
    assert res.status == O.OK and res.n_vcycles <= 12
    assert np.all(np.diff(res.history) < 0)


def test_status_codes():
    A = W.poisson5(32)
    b = W.rhs_uniform(0, A.n_rows)
    assert O.solve(_hier(A, "pinv", [5.0, 0, 0, 0, 0]), b).status == O.DIVERGED
    assert O.solve(_hier(A), b, max_iter=2).status == O.MAXITER
    assert O.solve(_hier(A, "pinv", [1e-6, 0, 0, 0, 0]), b).status == O.STAGNATED


def test_relative_metric_zero_for_identical_smoothers():
    A = W.poisson5(16)
    hg = _hier(A, "pinv", [2.0 / 3.0, 0, 0, 0, 0], max_coarse=8)
    hj = _hier(A, max_coarse=8)
    assert abs(O.relative_metric(hg, hj, W.rhs_uniform(1, A.n_rows))) < 1e-12


# ---------------------------------------------------------------------------
# Krylov outer loop (conjugate gradients preconditioned by one V-cycle)
# ---------------------------------------------------------------------------
def _iterates_scipy_cg(A, b, precond, k):
    """x_1 .. x_k of scipy's (classical) preconditioned CG."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    As = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n_rows, A.n_rows))
    M = sla.LinearOperator(As.shape, matvec=lambda r: precond(torch.from_numpy(np.asarray(r).ravel())).numpy())
    xs = []
    sla.cg(As, b, M=M, rtol=1e-300, atol=0.0, maxiter=k, callback=lambda x: xs.append(np.array(x)))
    return xs


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_pcg_iterates_equal_scipy_cg(smoother):
    """With a fixed symmetric preconditioner (FP64 V-cycle) the flexible
    coefficient reduces to the classical one: every iterate equals scipy's."""
    A = W.fv_mesh("graded", 1500, 3)[0]
    levels = S.build_hierarchy(A)
    h = O.OHierarchy.of(levels)
    if smoother == "jacobi":
        h.set_jacobi()
    else:
        h.set_pseudo_inverse([[0.62, 0.03, -0.01, -0.18, 0.02]] * len(levels))
    b = W.rhs_uniform(4, A.n_rows)
    pre = lambda r: O.vcycle(h, r, torch.zeros_like(r))
    ref = _iterates_scipy_cg(A, b, pre, 6)
    for k in range(1, 7):
        res = O.solve_pcg(h, b, tol=0.0, max_iter=k)
        assert res.n_vcycles == k
        assert np.abs(res.x - ref[k - 1]).max() <= 1e-10 * np.abs(ref[k - 1]).max()
        # the recurrence residual is the true residual in FP64
        rt = b - O.mv(h.levels[0].A, torch.from_numpy(res.x)).numpy()
        assert abs(np.linalg.norm(rt) / np.linalg.norm(b) - res.history[-1]) <= 1e-10


def test_pcg_exact_preconditioner_converges_in_one_step():
    A = W.poisson5(9)
    h = O.OHierarchy.of(S.build_hierarchy(A, max_coarse=4))
    Ad = A.to_dense()
    b = W.rhs_uniform(1, A.n_rows)
    res = O.solve_pcg(h, b, tol=1e-12, precond=lambda r: torch.from_numpy(np.linalg.solve(Ad, r.numpy())))
    assert res.status == O.OK and res.n_vcycles == 1
    assert np.abs(res.x - np.linalg.solve(Ad, b)).max() <= 1e-12 * np.abs(res.x).max()


def test_pcg_unpreconditioned_finishes_in_n_steps():
    """Plain CG on an n x n SPD matrix reaches the solution in at most n steps."""
    A = W.poisson5(4)              # n = 16, four distinct eigenvalue clusters by symmetry
    h = O.OHierarchy.of(S.build_hierarchy(A, max_coarse=4))
    b = W.rhs_uniform(2, A.n_rows)
    res = O.solve_pcg(h, b, tol=1e-13, precond=lambda r: r.clone())
    assert res.status == O.OK and res.n_vcycles <= A.n_rows
    assert np.abs(res.x - np.linalg.solve(A.to_dense(), b)).max() <= 1e-10


def test_pcg_beats_stationary_iteration():
    A = W.fv_mesh("band", 3000, 7, max_aspect=100.0)[0]
    h = O.OHierarchy.of(S.build_hierarchy(A))
    h.set_jacobi()
    b = W.rhs_zero_mean(3, A.n_rows)
    st = O.solve(h, b, tol=1e-8)
    kr = O.solve_pcg(h, b, tol=1e-8)
    assert st.status == kr.status == O.OK
    assert kr.n_vcycles < st.n_vcycles


def test_pcg_breakdown_on_indefinite_preconditioner():
    A = W.poisson5(8)
    h = O.OHierarchy.of(S.build_hierarchy(A, max_coarse=4))
    b = W.rhs_uniform(3, A.n_rows)
    res = O.solve_pcg(h, b, tol=1e-8, precond=lambda r: -r)
    assert res.status == O.DIVERGED and res.n_vcycles == 0 and len(res.history) == 1


# ---------------------------------------------------------------------------
# Chebyshev baseline smoother
# ---------------------------------------------------------------------------
def _lap1d(n):
    r = np.concatenate([np.arange(n), np.arange(n - 1), np.arange(1, n)])
    c = np.concatenate([np.arange(n), np.arange(1, n), np.arange(n - 1)])
    v = np.concatenate([np.full(n, 2.0), np.full(2 * (n - 1), -1.0)])
    return W._coo_to_csr(n, n, r, c, v)


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_error_propagation_closed_form(degree):
    """On the 1D Laplacian (D^-1 A eigenpairs 1 - cos(k pi/(n+1)), sin) the
    smoother maps an eigenvector e_k to T_d((theta - lam)/delta) / T_d(theta/delta) e_k."""
    n = 31
    A = _lap1d(n)
    lv = O.OLevel(O.TMat.of(A), None, None)
    theta, delta = 1.05, 0.95
    lv.cheb = (theta, delta, degree, torch.full((n,), 0.5, dtype=torch.float64))
    T = lambda x: np.cosh(degree * np.arccosh(x)) if abs(x) >= 1 else np.cos(degree * np.arccos(x))
    i = np.arange(1, n + 1)
    for k in (1, 5, 16, 30):
        lam = 1.0 - np.cos(k * np.pi / (n + 1))
        e = torch.from_numpy(np.sin(i * k * np.pi / (n + 1)))
        out = O.cheb_smooth(lv, torch.zeros(n, dtype=torch.float64), e).numpy()
        gain = T((theta - lam) / delta) / T(theta / delta)
        np.testing.assert_allclose(out, gain * e.numpy(), rtol=1e-12, atol=1e-13)


def test_power_estimate_brackets_the_spectrum():
    A = W.fv_mesh("graded", 800, 2)[0]
    Ad = A.to_dense()
    lam_max = np.linalg.eigvals(Ad / np.diag(Ad)[:, None]).real.max()
    rho = O.power_estimate(O.TMat.of(A), 20)
    assert 0.9 * lam_max <= rho <= lam_max * (1 + 1e-12)
    assert np.array_equal(O.power_start(5).numpy()[:2], [0.5, (2654435761 % 2 ** 32) / 2 ** 32 + 0.5])


def test_chebyshev_vcycle_converges_and_is_symmetric():
    A = W.fv_mesh("band", 2000, 4, max_aspect=100.0)[0]
    h = O.OHierarchy.of(S.build_hierarchy(A))
    h.set_chebyshev(3)
    b = W.rhs_zero_mean(2, A.n_rows)
    res = O.solve(h, b, tol=1e-8)
    assert res.status == O.OK
    n = A.n_rows
    x, y = W.rhs_uniform(7, n), W.rhs_uniform(8, n)
    assert abs(x @ O.vcycle_operator_apply(h, y) - y @ O.vcycle_operator_apply(h, x)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


def test_poisson7_closed_form_spectrum():
    """The 3D 7-point Laplacian: eigenvalues sum_d (2 - 2 cos(k_d pi/(m+1)))."""
    m = 6
    ev = np.sort(np.linalg.eigvalsh(W.poisson7(m).to_dense()))
    k = np.arange(1, m + 1)
    lam1 = 2 - 2 * np.cos(k * np.pi / (m + 1))
    ref = np.sort((lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]).ravel())
    np.testing.assert_allclose(ev, ref, rtol=1e-12, atol=1e-12)
    B = W.poisson7(8, body_ratio=1e-2).to_dense()
    assert np.allclose(B, B.T) and np.linalg.eigvalsh(B).min() > 0


def test_poisson5_body_workload():
    # conductivity 1 everywhere is the plain 5-point Laplacian; with a body the
    # operator stays symmetric positive definite, interior rows sum to zero,
    # and couplings across the body boundary are harmonic means
    A = W.poisson5(24)
    B = W.poisson5_body(24, 1.0)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    m, ratio = 40, 1e-2
    D = W.poisson5_body(m, ratio, 0.25).to_dense()
    np.testing.assert_array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    i, j = np.divmod(np.arange(m * m), m)
    interior = (i > 0) & (i < m - 1) & (j > 0) & (j < m - 1)
    np.testing.assert_allclose(D.sum(1)[interior], 0.0, atol=1e-13)
    assert np.isclose(-D.min(), 1.0) and np.isclose(np.sort(np.unique(-D[D < 0]))[1], 2 * ratio / (1 + ratio))
