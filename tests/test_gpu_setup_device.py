"""GPU parity of the device setup (every level built by CUDA kernels with the
block-local RS split or the PMIS split, optionally followed by the
round-parallel second pass; Sec. 2.2 with parallel forms of the
Ruge-Stueben passes) against the oracle's hierarchy of the same coarsening
drawn from the same random numbers.

Bars: integer work bit-exact (level count, sizes, the patterns of P and of
every A_l, hence the C/F splits); P_0 bit-exact (the same operations in the
same order on the same A_0); A_l values within 1e-13 (Galerkin sums in
another order) and P_l, l >= 1, within 1e-12 (its weights are ratios of
those A_l entries); solves on the device-built hierarchy equal the oracle's
solve on its own (FP64: same V-cycle count, x within 1e-10).
"""
import numpy as np
import pytest

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import CASES, library_levels, oracle_hier, rel_err

pytestmark = pytest.mark.gpu


MODES = {"pmis": 0, "pmis-h1": P.AMG_SPLIT_SECOND_PASS, "rs-blocks": P.AMG_SPLIT_RS_BLOCKS,
         "rs-blocks-h1": P.AMG_SPLIT_RS_BLOCKS | P.AMG_SPLIT_SECOND_PASS}


def device_ctx(A, seed, precision=P.AMG_FP64, mode="pmis-h1", **kw):
    ctx = P.amg_create(precision=precision, **kw)
    P.amg_setup_device(ctx, A, seed, MODES[mode])
    return ctx


def assert_same_hierarchy(ctx, levels):
    lib = library_levels(ctx)
    assert len(lib) == len(levels)
    for l, ((a, p), lv) in enumerate(zip(lib, levels)):
        assert a.n_rows == lv.A.n_rows
        assert np.array_equal(a.row_ptr, lv.A.row_ptr) and np.array_equal(a.col, lv.A.col)
        assert rel_err(a.val, lv.A.val) < 1e-13
        if lv.P is not None:
            assert p.n_cols == lv.P.n_cols
            assert np.array_equal(p.row_ptr, lv.P.row_ptr) and np.array_equal(p.col, lv.P.col)
            if l == 0:
                assert np.array_equal(p.val, lv.P.val)
            else:
                assert rel_err(p.val, lv.P.val) < 1e-12


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("seed", [0, 41])
@pytest.mark.parametrize("name", list(CASES))
def test_device_setup_matches_oracle(name, seed, mode):
    A = CASES[name]()
    levels = OS.build_hierarchy(A, coarsening=mode, seed=seed)
    ctx = device_ctx(A, seed, mode=mode)
    try:
        assert_same_hierarchy(ctx, levels)
        s = P.amg_get_scales(ctx)
        for l, lv in enumerate(levels):
            assert abs(s[l] - O.smoother_scale(O.TMat.of(lv.A))) <= 1e-13 * s[l]
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("make", [lambda: W.poisson7(14, 1e-2), lambda: W.c5_problem(3, n_rhs=1, n_surface=120, n_far=3000)[0]],
                         ids=["sphere_14", "airfoil_small"])
def test_device_setup_3d_and_airfoil(make):
    """The 3D stencil and the airfoil's wall layers (couplings over nine
    decades) through the same kernels, second pass on."""
    A = make()
    levels = OS.build_hierarchy(A, coarsening="pmis-h1", seed=4)
    ctx = device_ctx(A, 4)
    try:
        assert_same_hierarchy(ctx, levels)
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("mode", list(MODES))
def test_device_setup_full_size_c2(mode):
    A = W.c2_matrix(0)
    levels = OS.build_hierarchy(A, coarsening=mode, seed=7)
    ctx = device_ctx(A, 7, P.AMG_FP32_IN_FP64, mode=mode)
    try:
        assert_same_hierarchy(ctx, levels)
        st, x, hist = P.amg_solve(ctx, W.rhs_zero_mean(3, A.n_rows), rtol=1e-8)
        assert st == P.AMG_OK
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
@pytest.mark.parametrize("name", ["c1_64", "graded_5k", "band_4k"])
def test_solve_on_device_hierarchy_matches_oracle(name, smoother):
    A = CASES[name]()
    levels = OS.build_hierarchy(A, coarsening="pmis-h1", seed=3)
    coeffs = [[0.62, 0.03, -0.01, -0.18, 0.02]] * len(levels)
    b = W.rhs_uniform(8, A.n_rows)
    ref = O.solve(oracle_hier(levels, smoother, coeffs), b, tol=1e-8)
    ctx = device_ctx(A, 3)
    try:
        if smoother == "pinv":
            P.amg_set_coeffs(ctx, coeffs)
        st, x, hist = P.amg_solve(ctx, b, rtol=1e-8)
        assert st == ref.status
        assert len(hist) - 1 == ref.n_vcycles
        assert rel_err(x, ref.x) < 1e-10
    finally:
        P.amg_destroy(ctx)


def test_device_setup_is_deterministic_and_seeded():
    A = CASES["band_4k"]()
    outs = []
    for seed in (5, 5, 6):
        ctx = device_ctx(A, seed)
        try:
            outs.append(library_levels(ctx))
        finally:
            P.amg_destroy(ctx)
    for (a0, p0), (a1, p1) in zip(outs[0], outs[1]):
        assert np.array_equal(a0.col, a1.col) and np.array_equal(a0.val, a1.val)
        if p0 is not None:
            assert np.array_equal(p0.col, p1.col) and np.array_equal(p0.val, p1.val)
    assert not np.array_equal(outs[0][0][1].col, outs[2][0][1].col)


def test_device_setup_edge_cases():
    # a matrix at or below the coarse size is one level; a diagonal matrix has
    # no strong connections, so coarsening stops at the first level
    small = W.poisson5(8)
    ctx = device_ctx(small, 0)
    try:
        assert P.amg_num_levels(ctx) == 1
    finally:
        P.amg_destroy(ctx)
    n = 300
    D = W.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.linspace(1.0, 2.0, n))
    ctx = P.amg_create(precision=P.AMG_FP64, max_coarse=16)
    try:
        with pytest.raises(P.AmgError):      # a non-square matrix is refused
            P.amg_setup_device(ctx, W.CSR(n, n + 1, D.row_ptr, D.col, D.val), 0)
        P.amg_setup_device(ctx, D, 0)
        assert P.amg_num_levels(ctx) == 1
        st, x, hist = P.amg_solve(ctx, np.ones(n), rtol=1e-12)
        assert st == P.AMG_OK and rel_err(x, 1.0 / D.val) < 1e-14
    finally:
        P.amg_destroy(ctx)


def test_block_split_with_one_block_is_the_host_rs_setup():
    # n = 3600 rows and every level's strong pairs fit one block: the device
    # split is the classical first pass itself, so the hierarchy is amg_setup's
    A = W.poisson5(60)
    ref = OS.build_hierarchy(A, coarsening="rs")
    ctx = device_ctx(A, 0, mode="rs-blocks")
    host = P.amg_create(precision=P.AMG_FP64)
    try:
        assert_same_hierarchy(ctx, ref)
        P.amg_setup(host, A)
        for (a, p), (ah, ph) in zip(library_levels(ctx), library_levels(host)):
            assert np.array_equal(a.col, ah.col) and rel_err(a.val, ah.val) < 1e-13
            if p is not None:
                assert np.array_equal(p.col, ph.col)
    finally:
        P.amg_destroy(ctx)
        P.amg_destroy(host)


def test_block_split_small_blocks_on_a_dense_band():
    # a_ij = -1 for 0 < |i - j| <= 100: 200 strong pairs per row, so blocks
    # of 256 rows and more hold more than 32768 pairs (256 * 200 - 2 (100 +
    # 99 + ... + 1) = 41100) and the split runs on blocks of 128 rows (eight
    # CTAs on level 0)
    n, w = 1000, 100
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(max(0, i - w), min(n, i + w + 1)):
            rows.append(i)
            cols.append(j)
            vals.append(2.0 * w + 1.0 if i == j else -1.0)
    A = W._coo_to_csr(n, n, np.array(rows), np.array(cols), np.array(vals))
    Sg, _ = OS.strength(A, 0.25)
    assert OS.rs_block_size(n, Sg) == 128
    for mode in ("rs-blocks", "rs-blocks-h1"):
        levels = OS.build_hierarchy(A, coarsening=mode, seed=5)
        ctx = device_ctx(A, 5, mode=mode)
        try:
            assert_same_hierarchy(ctx, levels)
        finally:
            P.amg_destroy(ctx)


def test_unknown_split_refused():
    ctx = P.amg_create(precision=P.AMG_FP64)
    try:
        for bad in (-1, 4):
            with pytest.raises(P.AmgError):
                P.amg_setup_device(ctx, W.poisson5(20), 0, bad)
    finally:
        P.amg_destroy(ctx)


def test_host_routines_on_device_built_levels():
    """The device-built levels reach the host only on demand: the Chebyshev
    interval (a host power estimate) and the Jacobi smoother export read
    them, and must see the oracle's hierarchy of the same split."""
    A = CASES["graded_5k"]()
    levels = OS.build_hierarchy(A, coarsening="rs-blocks", seed=2)
    ctx = device_ctx(A, 2, mode="rs-blocks")
    try:
        P.amg_set_chebyshev(ctx, 3)
        for l in range(len(levels) - 1):
            rho, theta, delta = P.amg_get_chebyshev(ctx, l)
            ref = O.power_estimate(O.TMat.of(levels[l].A), 20)
            assert abs(rho - ref) <= 1e-11 * ref          # A_l within 1e-13 of the oracle's
        P.amg_set_jacobi(ctx)
        for l in range(len(levels) - 1):
            q = P.amg_get_smoother(ctx, l)
            ref = O.jacobi_values(O.TMat.of(levels[l].A), 2.0 / 3.0).numpy()
            assert rel_err(q, ref) < 1e-12
        # the host copies, once made, equal the oracle's levels
        assert_same_hierarchy(ctx, levels)
    finally:
        P.amg_destroy(ctx)
