"""What the trained network gains over the method without it.

The committed parameters (paper_2606_19251_gb300/weights/gcin_c3.npy, made by
weights/make_weights.py on the 64-mesh training batch) are evaluated on
held-out meshes the training never saw: the 50k- and 200k-point graded
meshes and a 20k-point band mesh (aspect 100, the training batch's band
kind, another seed).  The widened parameters (gcin_wide.npy, trained with
band meshes of aspect up to 1000 added) are held to the same bars on a
200k-point band mesh of aspect 1000 with an unseen seed, the anisotropic
case of the generalisation workload.  With the predicted pseudo-inverse
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

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300", "weights")
# (weights, matrix, bar on the one-cycle relative metric of Sec. 3.3): on the
# anisotropic band meshes one cycle gains less (measured -0.04 / -0.07) while
# the solve still needs 20-24 % fewer V-cycles
CASES = {
    "graded50k": ("gcin_c3.npy", lambda: W.c2_matrix(0), -0.1),
    "graded200k": ("gcin_c3.npy", lambda: W.fv_mesh("graded", 200000, 777)[0], -0.1),
    "band20k-aspect100": ("gcin_c3.npy", lambda: W.fv_mesh("band", 20000, 777, max_aspect=100.0)[0], -0.02),
    "band200k-aspect1000": ("gcin_wide.npy", lambda: W.fv_mesh("band", 200000, 778, max_aspect=1000.0)[0], -0.02),
}


def true_rel_residual(A, x, b):
    r = b - O.mv(O.TMat.of(A), torch.from_numpy(x)).numpy()
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("name", list(CASES))
def test_trained_gcin_beats_jacobi_on_held_out_meshes(name):
    wfile, make, metric_bar = CASES[name]
    theta = np.load(os.path.join(WDIR, wfile))
    A = make()
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
        assert metric < metric_bar, diag
    finally:
        P.amg_destroy(ctx)
