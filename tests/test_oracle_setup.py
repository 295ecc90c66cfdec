"""Pins for the oracle's setup phase (Sec. 2.2): RS splitting, direct
interpolation, Galerkin product.  Each check comes from a closed form or an
independent computation, not from re-running the oracle's own formulas."""
import numpy as np
import pytest

import workloads as W
from oracle import setup as S
from workloads import CSR


def lap1d(n):
    """tridiag(-1, 2, -1), Dirichlet eliminated."""
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, v in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    return W._coo_to_csr(n, n, np.array(rows), np.array(cols), np.array(vals))


def test_1d_laplacian_closed_form():
    # RS on the 1-D Laplacian: first pick = lowest index of maximal measure
    # (index 1), then every other point; linear interpolation (weights 1/2) and
    # the Galerkin operator tridiag(-1/2, 1, -1/2).
    n = 15
    A = lap1d(n)
    Sg, ST = S.strength(A, 0.25)
    split = S.rs_split(n, Sg, ST)
    assert np.array_equal(np.nonzero(split)[0], np.arange(1, n, 2))
    P = S.direct_interpolation(A, Sg, split)
    Pd = P.to_dense()
    nc = (n - 1) // 2
    expect = np.zeros((n, nc))
    for I in range(nc):
        i = 2 * I + 1
        expect[i, I] = 1.0
        expect[i - 1, I] = 0.5
        expect[i + 1, I] = 0.5
    assert np.array_equal(Pd, expect)
    Ac = S.galerkin(A, P).to_dense()
    expect_c = np.diag(np.ones(nc)) - 0.5 * np.eye(nc, k=1) - 0.5 * np.eye(nc, k=-1)
    np.testing.assert_allclose(Ac, expect_c, atol=1e-15)


def test_5point_first_level_is_red_black():
    # 5-point stencil, theta = 0.25: all four neighbours are strong; the first
    # C point is (1,1) (lowest index with four strong dependents) and the
    # first pass produces the red-black split {(i, j): i + j even}.
    m = 64
    A = W.poisson5(m)
    Sg, ST = S.strength(A, 0.25)
    split = S.rs_split(A.n_rows, Sg, ST)
    i, j = np.divmod(np.arange(m * m), m)
    assert np.array_equal(split, ((i + j) % 2 == 0).astype(np.int64))


@pytest.mark.parametrize("kind", ["uniform", "graded", "band"])
def test_split_is_maximal_independent_set(kind):
    # For a symmetric strength graph the first pass leaves no two C points
    # strongly connected and every F point with a strong connection has a
    # strong C neighbour.
    A, _ = W.fv_mesh(kind, 1500, 5, max_aspect=100.0)
    Sg, ST = S.strength(A, 0.25)
    split = S.rs_split(A.n_rows, Sg, ST)
    sym = all(set(Sg[i]) == set(ST[i]) for i in range(A.n_rows))
    for i in range(A.n_rows):
        nb = set(Sg[i]) | set(ST[i])
        if split[i] == 1 and sym:
            assert not any(split[j] == 1 for j in nb)
        if split[i] == 0 and nb:
            assert any(split[j] == 1 for j in Sg[i]) or any(split[j] == 1 for j in ST[i])


@pytest.mark.parametrize("kind", ["uniform", "graded", "band"])
def test_galerkin_equals_dense_triple_product(kind):
    A, _ = W.fv_mesh(kind, 900, 2, max_aspect=100.0)
    levels = S.build_hierarchy(A, max_coarse=20)
    assert len(levels) >= 3
    for l in range(len(levels) - 1):
        Ad = levels[l].A.to_dense()
        Pd = levels[l].P.to_dense()
        Acd = levels[l + 1].A.to_dense()
        np.testing.assert_allclose(Acd, Pd.T @ Ad @ Pd, rtol=0, atol=1e-12 * np.abs(Ad).max())
        np.testing.assert_allclose(Acd, Acd.T, atol=1e-13 * np.abs(Acd).max())
        assert np.array_equal(levels[l].R.to_dense(), Pd.T)
        # C rows of P are the identity onto the coarse numbering
        c = np.nonzero(levels[l].split)[0]
        assert np.array_equal(Pd[c], np.eye(len(c)))


def test_direct_interpolation_preserves_constants_on_zero_row_sums():
    # Where a row of A sums to zero (interior Neumann rows) the direct weights
    # sum to one, so constants are interpolated exactly.
    A, _ = W.fv_mesh("graded", 2000, 3)
    Sg, ST = S.strength(A, 0.25)
    split = S.rs_split(A.n_rows, Sg, ST)
    P = S.direct_interpolation(A, Sg, split)
    Ad = A.to_dense()
    rowsum = Ad.sum(1)
    psum = P.to_dense().sum(1)
    zero_rows = np.abs(rowsum) < 1e-12 * np.abs(np.diag(Ad))
    has_row = np.diff(P.row_ptr) > 0
    sel = zero_rows & has_row & (split == 0)
    assert sel.sum() > 100
    np.testing.assert_allclose(psum[sel], 1.0, atol=1e-12)


def test_hierarchy_stopping_rules():
    A = W.poisson5(64)
    lv = S.build_hierarchy(A, max_coarse=64)
    assert lv[-1].A.n_rows <= 64 and all(l.A.n_rows > 64 for l in lv[:-1])
    lv2 = S.build_hierarchy(A, max_levels=3)
    assert len(lv2) == 3
    small = W.poisson5(8)
    assert len(S.build_hierarchy(small, max_coarse=64)) == 1
