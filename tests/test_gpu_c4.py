"""Full-size generalisation case: 2.5M-node graded Delaunay mesh with an
anisotropic band (aspect up to 1000), about 128x the training meshes.

The oracle cannot run the whole solve at this size, so the checks are
properties that hold at any size plus outputs it computes one by one:
sampled rows of A_l x on every level, sampled entries of the Galerkin
product P^T A P, the final residual of both solves recomputed in FP64 by
the oracle's own product, and the trained network's V-cycle reduction.
"""
import os

import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import solve as O

pytestmark = pytest.mark.gpu

WEIGHTS_WIDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300",
                            "weights", "gcin_wide.npy")
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300",
                       "weights", "gcin_c3.npy")


@pytest.fixture(scope="module")
def c4():
    A = W.c4_matrix(0)
    ctx = P.amg_create(precision=P.AMG_FP32_IN_FP64)
    P.amg_setup(ctx, A)
    yield A, ctx
    P.amg_destroy(ctx)


def test_c4_sampled_spmv_and_galerkin(c4):
    A, ctx = c4
    rng = np.random.default_rng(0)
    ctx64 = P.amg_create(precision=P.AMG_FP64)
    try:
        nl = P.amg_num_levels(ctx)
        levels = [P.amg_get_level(ctx, l) for l in range(nl)]
        A_l = [W.CSR(a["n"], a["n"], a["row_ptr"], a["col"], a["val"]) for a, _ in levels]
        P_l = [W.CSR(p["n"], p["nc"], p["row_ptr"], p["col"], p["val"]) for _, p in levels[:-1]]
        P.amg_load_hierarchy(ctx64, A_l, P_l)
        for l in range(nl):
            x = W.rhs_uniform(40 + l, A_l[l].n_rows)
            dx = torch.tensor(x, device="cuda")
            dy = torch.empty_like(dx)
            P.amg_spmv_device(ctx64, l, dx, dy)
            torch.cuda.synchronize()
            y = dy.cpu().numpy()
            M = A_l[l]
            for i in rng.integers(0, M.n_rows, 200):
                lo, hi = M.row_ptr[i], M.row_ptr[i + 1]
                ref = sum(M.val[p] * x[M.col[p]] for p in range(lo, hi))
                assert abs(y[i] - ref) <= 1e-13 * max(1.0, sum(abs(M.val[p] * x[M.col[p]]) for p in range(lo, hi)))
        # Galerkin entries (A_{l+1})_{IJ} = sum_{i,j} P_iI a_ij P_jJ, one by one
        for l in range(min(2, nl - 1)):
            M, Pm, C = A_l[l], P_l[l], A_l[l + 1]
            prow = np.repeat(np.arange(Pm.n_rows), np.diff(Pm.row_ptr))

            def p_entry(j, J):
                lo, hi = Pm.row_ptr[j], Pm.row_ptr[j + 1]
                k = np.nonzero(Pm.col[lo:hi] == J)[0]
                return Pm.val[lo + k[0]] if k.size else 0.0

            for I in rng.integers(0, C.n_rows, 10):
                sel = np.nonzero(Pm.col == I)[0]
                for p in range(C.row_ptr[I], C.row_ptr[I + 1]):
                    J = int(C.col[p])
                    ref = 0.0
                    for e in sel:
                        i, wi = int(prow[e]), Pm.val[e]
                        for q in range(M.row_ptr[i], M.row_ptr[i + 1]):
                            ref += wi * M.val[q] * p_entry(int(M.col[q]), J)
                    assert abs(C.val[p] - ref) <= 1e-12 * max(1.0, abs(M.val).max())
    finally:
        P.amg_destroy(ctx64)


def test_c4_trained_gcin_vs_jacobi_to_1e8(c4):
    # the trained smoother is judged over 30 cycles (Sec. 3.3 metric); where
    # it does not beat Jacobi the mesh is reported and rerouted, and the solve
    # still reaches 1e-8.
    A, ctx = c4
    b = W.rhs_zero_mean(3, A.n_rows)
    P.amg_set_jacobi(ctx)
    st_j, x_j, h_j = P.amg_solve(ctx, b)
    P.gnn_load_params(ctx, np.load(WEIGHTS))
    P.gnn_predict_coeffs(ctx)
    metric, sm = P.amg_reroute(ctx, W.rhs_uniform(8, A.n_rows), 30)
    st_g, x_g, h_g = P.amg_solve(ctx, b)
    rerouted = P.amg_last_solve_rerouted(ctx)
    P.amg_set_jacobi(ctx)
    diag = f"jacobi: {st_j}, {len(h_j) - 1} cycles; judged {metric:.3f} -> smoother {sm}; then {st_g}, {len(h_g) - 1} cycles"
    T = O.TMat.of(A)
    for st, x in ((st_j, x_j), (st_g, x_g)):
        assert st == P.AMG_OK, diag
        r = b - O.mv(T, torch.from_numpy(x)).numpy()
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8, diag
    diag += f"; rerouted in solve: {rerouted}"
    if sm == P.AMG_SMOOTHER_GNN and not rerouted:
        assert len(h_g) < len(h_j), diag
    elif sm != P.AMG_SMOOTHER_GNN:
        assert metric >= 0 and len(h_g) == len(h_j), diag
    print(diag)


def test_c4_widened_gcin_beats_jacobi_to_1e8(c4):
    """The network trained on the C3 batch plus band meshes of aspect ratio up
    to 1000 and small airfoils generalises to the 2.5M-node mesh: the judge
    keeps it and it needs clearly fewer V-cycles than Jacobi."""
    A, ctx = c4
    b = W.rhs_zero_mean(3, A.n_rows)
    P.amg_set_jacobi(ctx)
    st_j, x_j, h_j = P.amg_solve(ctx, b)
    P.gnn_load_params(ctx, np.load(WEIGHTS_WIDE))
    P.gnn_predict_coeffs(ctx)
    metric, sm = P.amg_reroute(ctx, W.rhs_uniform(8, A.n_rows), 30)
    st_g, x_g, h_g = P.amg_solve(ctx, b)
    P.amg_set_jacobi(ctx)
    diag = f"jacobi {len(h_j) - 1} cycles; judged {metric:.3f} -> {sm}; learned {len(h_g) - 1} cycles"
    assert st_j == st_g == P.AMG_OK, diag
    assert sm == P.AMG_SMOOTHER_GNN and metric < 0, diag
    assert len(h_g) < 0.9 * len(h_j), diag
    r = b - O.mv(O.TMat.of(A), torch.from_numpy(x_g)).numpy()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8, diag
    print(diag)

