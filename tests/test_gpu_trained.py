"""What the trained network gains over the method without it.

The committed parameters (paper_2606_19251_gb300/weights/gcin_c3.npy, made by
weights/make_weights.py on the 64-mesh training batch) are evaluated on
held-out meshes the training never saw: the 50k-point graded mesh and a
band mesh with a different seed.  With the predicted pseudo-inverse
smoothers the solve reaches 1e-8 in clearly fewer V-cycles than
omega-Jacobi on the same hierarchy, the one-cycle relative metric of
Sec. 3.3 is negative, and the final residual is verified in FP64 by the
oracle's own product.
"""
import os

import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import solve as O

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300",
                       "weights", "gcin_c3.npy")


def true_rel_residual(A, x, b):
    r = b - O.mv(O.TMat.of(A), torch.from_numpy(x)).numpy()
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("name", ["graded50k", "graded200k"])
def test_trained_gcin_beats_jacobi_on_held_out_meshes(name):
    theta = np.load(WEIGHTS)
    A = W.c2_matrix(0) if name == "graded50k" else W.fv_mesh("graded", 200000, 777)[0]
    b = W.rhs_zero_mean(5, A.n_rows)
    ctx = P.amg_create(precision=P.AMG_FP32_IN_FP64)
    try:
        P.amg_setup(ctx, A)
        st_j, x_j, h_j = P.amg_solve(ctx, b)
        P.gnn_load_params(ctx, theta)
        c = P.gnn_predict_coeffs(ctx)
        assert np.all(np.isfinite(c))
        st_g, x_g, h_g = P.amg_solve(ctx, b)
        metric = P.amg_judge(ctx, W.rhs_uniform(6, A.n_rows))
        diag = f"jacobi {st_j} {len(h_j) - 1} cycles; gnn {st_g} {len(h_g) - 1} cycles; judge {metric:.3f}; c0 {c[0]}"
        assert st_j == st_g == P.AMG_OK, diag
        assert true_rel_residual(A, x_g, b) <= 1e-8 and true_rel_residual(A, x_j, b) <= 1e-8
        assert len(h_g) - 1 <= 0.85 * (len(h_j) - 1), diag
        assert metric < -0.1, diag
    finally:
        P.amg_destroy(ctx)
