"""3D Cartesian finite-volume Poisson (7-point stencil, a low-conductivity
immersed sphere): the setup, the FP64 solve and the mixed-precision solve
against the FP64 oracle, and the 2D-trained smoother judged on a 3D mesh
(it must not cost more cycles than Jacobi once the judge has decided)."""
import os

import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import ctx_setup, library_levels, oracle_hier, rel_err

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300",
                       "weights", "gcin_c3.npy")
COEFFS = [0.6, 0.02, 0.0, -0.05, 0.01]   # a stable pseudo-inverse on this 3D stencil


@pytest.fixture(scope="module")
def cube():
    A = W.poisson7(16, body_ratio=1e-2)
    return A, OS.build_hierarchy(A)


def test_setup_matches_oracle(cube):
    A, levels = cube
    ctx = ctx_setup(A)
    try:
        lib = library_levels(ctx)
        assert len(lib) == len(levels)
        for (a, p), lv in zip(lib, levels):
            assert np.array_equal(a.row_ptr, lv.A.row_ptr) and np.array_equal(a.col, lv.A.col)
            assert rel_err(a.val, lv.A.val) < 1e-13
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_solves_match_oracle(cube, smoother):
    A, levels = cube
    coeffs = [COEFFS] * len(levels)
    b = W.rhs_uniform(3, A.n_rows)
    ref = O.solve(oracle_hier(levels, smoother, coeffs), b, tol=1e-8)
    for prec in (P.AMG_FP64, P.AMG_FP32_IN_FP64):
        ctx = ctx_setup(A, prec)
        try:
            if smoother == "pinv":
                P.amg_set_coeffs(ctx, coeffs)
            st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
            assert st == ref.status == P.AMG_OK
            if prec == P.AMG_FP64:
                assert len(hist) - 1 == ref.n_vcycles
                assert rel_err(x, ref.x) < 1e-11
            else:
                assert abs((len(hist) - 1) - ref.n_vcycles) <= 1
                r = b - O.mv(O.TMat.of(A), torch.from_numpy(x)).numpy()
                assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.0001e-8
        finally:
            P.amg_destroy(ctx)


def test_trained_smoother_judged_on_a_3d_mesh():
    A = W.poisson7(40, body_ratio=1e-2)
    b = W.rhs_zero_mean(4, A.n_rows)
    counts = {}
    for mode in ("gnn", "jacobi"):
        ctx = ctx_setup(A, P.AMG_FP32_IN_FP64)
        try:
            if mode == "gnn":
                P.gnn_load_params(ctx, np.load(WEIGHTS))
                P.gnn_predict_coeffs(ctx)
                P.amg_reroute(ctx, b, 30)
            st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
            assert st == P.AMG_OK
            counts[mode] = len(hist) - 1
        finally:
            P.amg_destroy(ctx)
    assert counts["gnn"] <= 1.05 * counts["jacobi"], counts
