"""The airfoil pressure sequence (C5): a NACA m412 section in a circular
farfield, wall-normal layers from 1e-5 chords (aspect ratios in the
hundreds), and 50 slowly varying right-hand sides solved one after another
from the previous solution, with the smoother's coefficients predicted once
(Sec. 4's time-dependent use of the learned smoother).

Small mesh: every solve of the sequence equals the FP64 oracle's solve from
the same warm start (same V-cycle count, x within 1e-10).  Full mesh
(254k unknowns): every solve reaches 1e-8 (checked in FP64 by the oracle's
matrix-vector product), and the judged smoother (the network trained with
the widened distribution, airfoils included) needs no more cycles than
Jacobi over the sequence.
"""
import os

import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import ctx_setup, oracle_hier, rel_err

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_19251_gb300",
                       "weights", "gcin_wide.npy")
COEFFS = [0.62, 0.03, -0.01, -0.18, 0.02]


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_small_airfoil_sequence_matches_oracle(smoother):
    A, fs, m = W.c5_problem(2, n_rhs=4, n_surface=120, n_far=3000)
    levels = OS.build_hierarchy(A)
    h = oracle_hier(levels, smoother, [COEFFS] * len(levels))
    ctx = ctx_setup(A, P.AMG_FP64)
    try:
        if smoother == "pinv":
            P.amg_set_coeffs(ctx, [COEFFS] * len(levels))
        x_gpu = x_ref = None
        for f in fs:
            ref = O.solve(h, f, tol=1e-8, u0=x_ref)
            st, x_gpu, hist = P.amg_solve(ctx, f, x0=x_gpu, rtol=1e-8)
            assert st == ref.status
            assert len(hist) - 1 == ref.n_vcycles
            assert rel_err(x_gpu, ref.x) < 1e-10
            x_ref = ref.x
    finally:
        P.amg_destroy(ctx)


@pytest.fixture(scope="module")
def c5():
    return W.c5_problem(0)


@pytest.mark.parametrize("outer", [P.AMG_OUTER_REFINE, P.AMG_OUTER_PCG])
def test_full_airfoil_sequence(c5, outer):
    A, fs, m = c5
    n = A.n_rows
    cycles = {}
    for mode in ("gnn", "jacobi"):
        ctx = ctx_setup(A, P.AMG_FP32_IN_FP64, outer=outer)
        try:
            if mode == "gnn":
                P.gnn_load_params(ctx, np.load(WEIGHTS))
                P.gnn_predict_coeffs(ctx)
                P.amg_reroute(ctx, fs[0], 30)
            else:
                P.amg_set_jacobi(ctx)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            total = 0
            for t, f in enumerate(fs):
                st, hist = P.amg_solve_device(ctx, torch.tensor(f, device="cuda"), x)
                torch.cuda.synchronize()
                assert st == P.AMG_OK, (mode, t, st)
                total += len(hist) - 1
                if t in (0, 25, 49):
                    r = f - O.mv(O.TMat.of(A), x.cpu()).numpy()
                    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1.0001e-8
            cycles[mode] = total
        finally:
            P.amg_destroy(ctx)
    assert cycles["gnn"] <= 1.05 * cycles["jacobi"], cycles
