"""GPU parity of the Chebyshev baseline smoother (degree-k polynomial in
D^-1 A on [rho/30, 1.1 rho], the fixed-coefficient comparison for the learned
smoother) against the FP64 oracle.

Bars: the power estimate within 1e-12 relative (same start vector, same
iteration, summation order only); FP64 smoothing and V-cycle within 1e-12;
FP64 solves with the same cycle count and history within 1e-10; FP32 V-cycle
solves within +-1 cycle.
"""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import CASES, ctx_from_oracle, ctx_setup, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, make in CASES.items():
        A = make()
        out[name] = (A, OS.build_hierarchy(A))
    return out


def cheb_hier(levels, degree=3):
    h = O.OHierarchy.of(levels)
    h.set_chebyshev(degree)
    return h


@pytest.mark.parametrize("name", list(CASES))
def test_interval_matches_oracle(cases, name):
    A, levels = cases[name]
    h = cheb_hier(levels)
    ctx = ctx_from_oracle(levels)
    try:
        P.amg_set_chebyshev(ctx, 3)
        for l in range(len(levels) - 1):
            rho, theta, delta = P.amg_get_chebyshev(ctx, l)
            assert abs(rho - O.power_estimate(h.levels[l].A, 20)) <= 1e-12 * rho
            assert abs(theta - h.levels[l].cheb[0]) <= 1e-12 * theta
            assert abs(delta - h.levels[l].cheb[1]) <= 1e-12 * delta
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("degree", [1, 3, 5])
@pytest.mark.parametrize("name", ["c1_64", "graded_5k", "band_4k"])
def test_smoothing_parity_fp64(cases, name, degree):
    A, levels = cases[name]
    h = cheb_hier(levels, degree)
    ctx = ctx_from_oracle(levels)
    try:
        P.amg_set_chebyshev(ctx, degree)
        for l in range(len(levels) - 1):
            b = W.rhs_uniform(20 + l, levels[l].A.n_rows)
            u0 = W.rhs_uniform(30 + l, levels[l].A.n_rows)
            db, du = torch.tensor(b, device="cuda"), torch.tensor(u0, device="cuda")
            P.amg_smooth_device(ctx, l, db, du, 2)
            torch.cuda.synchronize()
            u = torch.from_numpy(u0)
            for _ in range(2):
                u = O.cheb_smooth(h.levels[l], torch.from_numpy(b), u)
            assert rel_err(du.cpu().numpy(), u.numpy()) < 1e-12
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_and_solve_parity_fp64(cases, name):
    A, levels = cases[name]
    h = cheb_hier(levels)
    ctx = ctx_from_oracle(levels)
    try:
        P.amg_set_chebyshev(ctx, 3)
        r = W.rhs_uniform(5, A.n_rows)
        dr = torch.tensor(r, device="cuda")
        de = torch.empty_like(dr)
        P.amg_vcycle_device(ctx, dr, de)
        torch.cuda.synchronize()
        assert rel_err(de.cpu().numpy(), O.vcycle_operator_apply(h, r)) < 1e-12
        b = W.rhs_uniform(0, A.n_rows)
        ref = O.solve(h, b, tol=1e-8)
        st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
        assert st == ref.status == P.AMG_OK
        assert len(hist) - 1 == ref.n_vcycles
        assert rel_err(hist, ref.history) < 1e-10
        assert rel_err(x, ref.x) < 1e-11
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("outer", [P.AMG_OUTER_REFINE, P.AMG_OUTER_PCG])
@pytest.mark.parametrize("name", ["graded_5k", "band_4k"])
def test_mixed_precision_solve(cases, name, outer):
    A, levels = cases[name]
    h = cheb_hier(levels)
    b = W.rhs_zero_mean(1, A.n_rows)
    ref = (O.solve if outer == P.AMG_OUTER_REFINE else O.solve_pcg)(h, b, tol=1e-8)
    ctx = ctx_setup(A, P.AMG_FP32_IN_FP64, outer=outer)
    try:
        P.amg_set_chebyshev(ctx, 3)
        st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
        assert st == ref.status == P.AMG_OK
        assert abs((len(hist) - 1) - ref.n_vcycles) <= 1
        r = b - O.mv(O.TMat.of(A), torch.from_numpy(x)).numpy()
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.0001e-8
    finally:
        P.amg_destroy(ctx)


def test_switching_smoothers_keeps_graphs_apart(cases):
    A, levels = cases["band_4k"]
    b = W.rhs_uniform(9, A.n_rows)
    ctx = ctx_setup(A, P.AMG_FP64)
    try:
        counts = {}
        for name, select in (("jacobi", lambda: P.amg_set_jacobi(ctx)), ("cheb3", lambda: P.amg_set_chebyshev(ctx, 3)),
                             ("cheb1", lambda: P.amg_set_chebyshev(ctx, 1)), ("jacobi2", lambda: P.amg_set_jacobi(ctx))):
            select()
            st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
            assert st == P.AMG_OK
            counts[name] = len(hist) - 1
        assert counts["jacobi"] == counts["jacobi2"]
        lv = OS.build_hierarchy(A)
        assert counts["cheb1"] == O.solve(cheb_hier(lv, 1), b, tol=1e-8).n_vcycles
        assert counts["cheb3"] == O.solve(cheb_hier(lv, 3), b, tol=1e-8).n_vcycles
        with pytest.raises(P.AmgError):
            P.amg_set_chebyshev(ctx, 0)
    finally:
        P.amg_destroy(ctx)
