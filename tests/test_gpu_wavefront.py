"""Wavefront smoothing chains (one kernel per smoothing phase on levels too
large for L2; Sec. 2.2 V-cycle, Sec. 2.3 Jacobi, Sec. 3.1 pseudo-inverse).

The chains must compute what the separate passes compute:
* FP64 (stored Q^-1 values, the same row arithmetic as the separate
  kernels): smoothing and V-cycles equal to the unfused path and to the
  oracle at the FP64 bars;
* FP32 (Q^-1 evaluated on the fly from A, s and c): smoothing within FP32
  rounding of the oracle's FP64 sweep, and mixed-precision solves reaching
  1e-8 (checked by the oracle's FP64 product) within one V-cycle of the
  unfused path.
Workloads: a 700 x 700 5-point grid (lexicographic order) and a 250k-point
band mesh numbered by reverse Cuthill-McKee.
"""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import setup as OS
from oracle import solve as O
from tests.gpu_helpers import library_levels, rel_err

pytestmark = pytest.mark.gpu

COEFFS = [0.62, 0.03, -0.01, -0.18, 0.02]


class _Lv:
    def __init__(self, A, Pm):
        self.A, self.P = A, Pm
        self.R = OS.transpose(Pm) if Pm is not None else None


def _mat(name):
    if name == "grid700":
        return W.poisson5(700)
    return W.renumber_rcm(W.fv_mesh("band", 250_000, 9, max_aspect=1000.0)[0])


@pytest.fixture(scope="module", params=["grid700", "band250k"])
def case(request):
    A = _mat(request.param)
    ctx0 = P.amg_create(precision=P.AMG_FP64)
    try:
        P.amg_setup(ctx0, A)
        levels = [_Lv(a, p) for a, p in library_levels(ctx0)]
    finally:
        P.amg_destroy(ctx0)
    return request.param, A, levels


def _ctx(levels, precision, fused):
    ctx = P.amg_create(precision=precision, fused_sweeps=fused)
    P.amg_load_hierarchy(ctx, [l.A for l in levels], [l.P for l in levels[:-1]], [l.R for l in levels[:-1]])
    return ctx


def _set(ctx, smoother, nlev):
    if smoother == "pinv":
        P.amg_set_coeffs(ctx, [COEFFS] * nlev)
    else:
        P.amg_set_jacobi(ctx)


def test_chains_run_on_the_large_levels(case):
    name, A, levels = case
    for fused in (1, 0):
        ctx = _ctx(levels, P.AMG_FP32_IN_FP64, fused)
        try:
            _set(ctx, "pinv", len(levels))
            if fused:
                P.amg_kernel_launch(ctx, P.AMG_K_WF_PRE, 0, 1)
                P.amg_kernel_launch(ctx, P.AMG_K_WF_POST, 0, 1)
                torch.cuda.synchronize()
            else:
                with pytest.raises(P.AmgError):
                    P.amg_kernel_launch(ctx, P.AMG_K_WF_PRE, 0, 1)
        finally:
            P.amg_destroy(ctx)


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
@pytest.mark.parametrize("nsweeps", [1, 2, 3])
def test_fp64_chain_smoothing_equals_separate_passes_and_oracle(case, smoother, nsweeps):
    name, A, levels = case
    h = O.OHierarchy.of(levels)
    if smoother == "pinv":
        h.set_pseudo_inverse([COEFFS] * len(levels))
    else:
        h.set_jacobi()
    outs = []
    for fused in (1, 0):
        ctx = _ctx(levels, P.AMG_FP64, fused)
        try:
            _set(ctx, smoother, len(levels))
            n = levels[0].A.n_rows
            b = W.rhs_uniform(20, n)
            u0 = W.rhs_uniform(30, n)
            db, du = torch.tensor(b, device="cuda"), torch.tensor(u0, device="cuda")
            P.amg_smooth_device(ctx, 0, db, du, nsweeps)
            torch.cuda.synchronize()
            outs.append(du.cpu().numpy())
        finally:
            P.amg_destroy(ctx)
    u = torch.from_numpy(u0)
    for _ in range(nsweeps):
        u = O.sweep(h.levels[0], torch.from_numpy(b), u)
    assert rel_err(outs[0], outs[1]) < 1e-15, rel_err(outs[0], outs[1])
    assert rel_err(outs[0], u.numpy()) < 1e-13


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_fp64_chain_vcycle(case, smoother):
    name, A, levels = case
    h = O.OHierarchy.of(levels)
    if smoother == "pinv":
        h.set_pseudo_inverse([COEFFS] * len(levels))
    else:
        h.set_jacobi()
    r = W.rhs_uniform(5, levels[0].A.n_rows)
    outs = []
    for fused in (1, 0):
        ctx = _ctx(levels, P.AMG_FP64, fused)
        try:
            _set(ctx, smoother, len(levels))
            dr = torch.tensor(r, device="cuda")
            de = torch.empty_like(dr)
            for _ in range(2):   # a second cycle re-runs every chain from its own state
                P.amg_vcycle_device(ctx, dr, de)
            torch.cuda.synchronize()
            outs.append(de.cpu().numpy())
        finally:
            P.amg_destroy(ctx)
    assert rel_err(outs[0], outs[1]) < 1e-13
    assert rel_err(outs[0], O.vcycle_operator_apply(h, r)) < 1e-12


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_fp32_chain_smoothing_within_fp32_of_oracle(case, smoother):
    name, A, levels = case
    h = O.OHierarchy.of(levels)
    if smoother == "pinv":
        h.set_pseudo_inverse([COEFFS] * len(levels))
    else:
        h.set_jacobi()
    ctx = _ctx(levels, P.AMG_FP32_IN_FP64, 1)
    try:
        _set(ctx, smoother, len(levels))
        for l in range(min(2, len(levels) - 1)):
            n = levels[l].A.n_rows
            b = W.rhs_uniform(40 + l, n)
            u0 = W.rhs_uniform(50 + l, n)
            db, du = torch.tensor(b, device="cuda"), torch.tensor(u0, device="cuda")
            P.amg_smooth_device(ctx, l, db, du, 2)
            torch.cuda.synchronize()
            u = torch.from_numpy(u0)
            for _ in range(2):
                u = O.sweep(h.levels[l], torch.from_numpy(b), u)
            err = rel_err(du.cpu().numpy(), u.numpy())
            assert err < 2e-5, (l, err)
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("smoother", ["jacobi", "pinv"])
def test_fp32_chain_solves_match_separate_passes(case, smoother):
    name, A, levels = case
    b = W.rhs_zero_mean(7, A.n_rows)
    res = []
    for fused in (1, 0):
        ctx = P.amg_create(precision=P.AMG_FP32_IN_FP64, fused_sweeps=fused)
        try:
            P.amg_setup(ctx, A)
            _set(ctx, smoother, P.amg_num_levels(ctx))
            res.append(P.amg_solve(ctx, b, rtol=1e-8))
        finally:
            P.amg_destroy(ctx)
    (st_f, x_f, h_f), (st_u, x_u, h_u) = res
    assert st_f == st_u == P.AMG_OK, (st_f, st_u)
    assert abs(len(h_f) - len(h_u)) <= 1, (len(h_f), len(h_u))
    r = b - O.mv(O.TMat.of(A), torch.from_numpy(x_f)).numpy()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
