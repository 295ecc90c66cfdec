"""GPU test of the allocation-free residual norm (amg_residual_norm_noalloc).

Some callers cannot call cudaMalloc (all device memory reserved up front in
their own pool, or a time-critical loop where an allocation may synchronise
the device or fail).  This entry point serves them: the caller passes every
input and output, and the only scratch is a fixed array of 2 x 1216 partial
sums compiled into the library.  The tests check it, through the C ABI:

* against the existing entry points on the same matrix (the relative
  residual that amg_solve reports before its first V-cycle, and b - A x from
  amg_spmv_device), on two calls in a row (the scratch keeps the previous
  call's contents);
* against the oracle's FP64 product on matrices large enough that the
  partial sums are capped at 1216 blocks and each block's grid-stride loop
  runs more than once, with one and with two lanes per row, with and
  without the residual output, and on an empty system.
"""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import solve as O

pytestmark = pytest.mark.gpu

SLOTS = 1216          # partial-sum slots of the library's scratch array
BLOCK = 256           # threads per block of its residual kernel


def _dev_csr(A):
    return (torch.tensor(A.row_ptr, dtype=torch.int32, device="cuda"),
            torch.tensor(A.col, dtype=torch.int32, device="cuda"),
            torch.tensor(A.val, dtype=torch.float64, device="cuda"))


def test_noalloc_residual_norm_matches_existing_entry_points():
    A = W.fv_mesh("graded", 20000, 11)[0]
    n = A.n_rows
    ctx = P.amg_create(precision=P.AMG_FP64, max_iter=0)
    try:
        P.amg_setup(ctx, A)
        d_rp, d_col, d_val = _dev_csr(A)
        for call, seed in enumerate((1, 2)):
            b = W.rhs_zero_mean(seed, n)
            x = 0.1 * W.rhs_uniform(seed + 10, n)
            d_b = torch.tensor(b, device="cuda")
            d_x = torch.tensor(x, device="cuda")
            d_r = torch.empty(n, dtype=torch.float64, device="cuda")
            d_out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            P.amg_residual_norm_noalloc(d_rp, d_col, d_val, d_b, d_x, d_out, d_r=d_r)
            torch.cuda.synchronize()
            out = d_out.cpu().numpy()
            # existing entry point 1: the solve's relative residual at x
            st, _, hist = P.amg_solve(ctx, b, x0=x, rtol=0.0)
            assert st == P.AMG_ERR_MAXITER and len(hist) == 1
            assert abs(out[0] / out[1] - hist[0]) <= 1e-12 * hist[0]
            # existing entry point 2: b - A x with the library's SpMV
            d_y = torch.empty_like(d_x)
            P.amg_spmv_device(ctx, 0, d_x, d_y)
            torch.cuda.synchronize()
            r_ref = b - d_y.cpu().numpy()
            r = d_r.cpu().numpy()
            assert np.abs(r - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
            assert abs(out[1] - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("name", ["grid700", "graded200k"])
def test_noalloc_grid_stride_against_oracle(name):
    # grid700: 2.45M entries -> one lane per row, 1914 row blocks;
    # graded200k: 1.4M entries -> two lanes per row, ~1560 row blocks;
    # both exceed the 1216 slots, so blocks loop over several row groups
    A = W.poisson5(700) if name == "grid700" else W.fv_mesh("graded", 200_000, 5)[0]
    n = A.n_rows
    tpr = 1 if name == "grid700" else 2
    assert (n * tpr + BLOCK - 1) // BLOCK > SLOTS
    M = O.TMat.of(A)
    d_rp, d_col, d_val = _dev_csr(A)
    for call, seed in enumerate((3, 4)):
        b = W.rhs_uniform(seed, n)
        x = W.rhs_uniform(seed + 20, n)
        r_ref = (torch.from_numpy(b) - O.mv(M, torch.from_numpy(x))).numpy()
        d_b = torch.tensor(b, device="cuda")
        d_x = torch.tensor(x, device="cuda")
        d_out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        d_r = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") if call == 0 else None
        P.amg_residual_norm_noalloc(d_rp, d_col, d_val, d_b, d_x, d_out, d_r=d_r)
        torch.cuda.synchronize()
        out = d_out.cpu().numpy()
        scale = np.abs(A.val).max() * np.abs(x).max() * np.diff(A.row_ptr).max()
        if d_r is not None:
            assert np.abs(d_r.cpu().numpy() - r_ref).max() <= 1e-13 * scale
        assert abs(out[0] - np.linalg.norm(r_ref)) <= 1e-12 * np.linalg.norm(r_ref)
        assert abs(out[1] - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_empty_system():
    d_rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_col = torch.zeros(0, dtype=torch.int32, device="cuda")
    d_val = torch.zeros(0, dtype=torch.float64, device="cuda")
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    d_out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    P.amg_residual_norm_noalloc(d_rp, d_col, d_val, e, e, d_out)
    torch.cuda.synchronize()
    assert d_out.cpu().tolist() == [0.0, 0.0]


def test_noalloc_rejects_oversized_problems():
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    zi = torch.zeros(2, dtype=torch.int32, device="cuda")
    L = P.api.lib()
    import ctypes as C
    p = C.c_void_p(z.data_ptr())
    pi = C.c_void_p(zi.data_ptr())
    rc = L.amg_residual_norm_noalloc(1 << 26, 1, pi, pi, p, p, p, None, p, None)
    assert rc == P.AMG_ERR_ARG
    assert "67108863" in P.amg_last_error(None)
