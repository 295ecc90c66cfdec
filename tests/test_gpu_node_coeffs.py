"""GPU parity of the per-node coefficient form of the pseudo-inverse smoother
(a generalisation of Sec. 3.1's per-level coefficients: node i's row for the
diagonal, the mean of the two nodes' rows for an off-diagonal entry) against
the FP64 oracle.

Bars: equal rows give bit-for-bit the per-level smoother; Q^-1 values within
1e-12 of the oracle (a reciprocal multiply against its division); FP64 solves
with the same V-cycle count and x within 1e-10; mixed precision to the same
tolerance with the count within +-1.
"""
import numpy as np
import pytest

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import CASES, ctx_setup, rel_err

pytestmark = pytest.mark.gpu

COEFFS = [0.62, 0.03, -0.01, -0.18, 0.02]


def node_coeffs(levels, seed, spread=0.05):
    out = []
    for l, lv in enumerate(levels[:-1]):
        n = lv.A.n_rows
        out.append(np.tile(COEFFS, (n, 1)) * (1.0 + spread * W.uniform_pm1(seed + l, 5 * n).reshape(n, 5)))
    return out


@pytest.fixture(scope="module")
def cases():
    return {name: (A, OS.build_hierarchy(A)) for name, A in ((k, make()) for k, make in CASES.items())}


@pytest.mark.parametrize("name", list(CASES))
def test_equal_rows_reproduce_level_coefficients(cases, name):
    A, levels = cases[name]
    ctx = ctx_setup(A, P.AMG_FP64)
    try:
        P.amg_set_coeffs(ctx, [COEFFS] * len(levels))
        ref = [P.amg_get_smoother(ctx, l) for l in range(len(levels) - 1)]
        P.amg_set_node_coeffs(ctx, [np.tile(COEFFS, (lv.A.n_rows, 1)) for lv in levels[:-1]])
        for l in range(len(levels) - 1):
            assert np.array_equal(P.amg_get_smoother(ctx, l), ref[l])
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
def test_node_smoother_values_match_oracle(cases, name):
    A, levels = cases[name]
    C = node_coeffs(levels, 11)
    ctx = ctx_setup(A, P.AMG_FP64)
    try:
        P.amg_set_node_coeffs(ctx, C)
        for l, lv in enumerate(levels[:-1]):
            ref = O.pseudo_inverse_values_nodes(O.TMat.of(lv.A), C[l]).numpy()
            assert rel_err(P.amg_get_smoother(ctx, l), ref) < 1e-12
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("prec", [P.AMG_FP64, P.AMG_FP32_IN_FP64])
@pytest.mark.parametrize("name", ["c1_64", "graded_5k", "band_4k"])
def test_solve_with_node_coefficients_matches_oracle(cases, name, prec):
    A, levels = cases[name]
    C = node_coeffs(levels, 21)
    h = O.OHierarchy.of(levels)
    h.set_pseudo_inverse_nodes(C)
    b = W.rhs_uniform(4, A.n_rows)
    ref = O.solve(h, b, tol=1e-8)
    ctx = ctx_setup(A, prec)
    try:
        P.amg_set_node_coeffs(ctx, C)
        st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
        assert st == ref.status == P.AMG_OK
        if prec == P.AMG_FP64:
            assert len(hist) - 1 == ref.n_vcycles
            assert rel_err(x, ref.x) < 1e-10
        else:
            assert abs((len(hist) - 1) - ref.n_vcycles) <= 1
    finally:
        P.amg_destroy(ctx)


def test_node_coefficients_argument_checks(cases):
    A, levels = cases["c1_64"]
    ctx = ctx_setup(A, P.AMG_FP64)
    try:
        C = node_coeffs(levels, 1)
        with pytest.raises(P.AmgError) as e:
            P.amg_set_node_coeffs(ctx, C[:-1])
        assert e.value.code == P.AMG_ERR_ARG
        C[0][3, 2] = np.nan
        with pytest.raises(P.AmgError):
            P.amg_set_node_coeffs(ctx, C)
    finally:
        P.amg_destroy(ctx)
