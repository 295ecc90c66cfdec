"""GPU test of the allocation-free residual norm (amg_residual_norm_noalloc).

Some callers cannot call cudaMalloc (all device memory reserved up front in
their own pool, or a time-critical loop where an allocation may synchronise
the device or fail).  This entry point serves them: the caller passes every
input and output, and the only scratch is a fixed array compiled into the
library.  The test checks it, through the C ABI, against the existing
entry points on the same matrix: the relative residual that amg_solve
reports before its first V-cycle, and b - A x from amg_spmv_device, on two
calls in a row (the scratch keeps the previous call's contents).
"""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_existing_entry_points():
    A = W.fv_mesh("graded", 20000, 11)[0]
    n = A.n_rows
    ctx = P.amg_create(precision=P.AMG_FP64, max_iter=0)
    try:
        P.amg_setup(ctx, A)
        d_rp = torch.tensor(A.row_ptr, dtype=torch.int32, device="cuda")
        d_col = torch.tensor(A.col, dtype=torch.int32, device="cuda")
        d_val = torch.tensor(A.val, dtype=torch.float64, device="cuda")
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
