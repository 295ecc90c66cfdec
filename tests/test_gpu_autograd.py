"""The autograd entry points (GcinCoefficients, GnnAmgLoss) compose into the
training objective of Sec. 3.3 / Algorithm 1: theta.grad from loss.backward()
equals the library's own training path (gcin_trainer_backward of the summed
amg_loss_grad) and the FP64 oracle's autograd gradient within the FP32 bar."""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import gcin as OG
from oracle import setup as OS
from oracle import solve as O
from oracle import train as OT
from paper_2606_19251_gb300.autograd import gcin_coefficients, gnn_amg_loss
from tests.gpu_helpers import ctx_setup

pytestmark = pytest.mark.gpu


def test_autograd_training_objective_matches_library_and_oracle():
    mats = [W.fv_mesh("uniform", 2000, 3)[0], W.fv_mesh("graded", 6000, 4)[0],
            W.fv_mesh("band", 8000, 5, max_aspect=100.0)[0]]
    fs = [W.rhs_uniform(100 + k, A.n_rows) for k, A in enumerate(mats)]
    theta0 = W.gcin_init_params(21)
    f32 = np.asarray(theta0, dtype=np.float32).astype(np.float64)
    ctxs = [ctx_setup(A, P.AMG_FP64) for A in mats]
    tr = P.gcin_trainer_create(theta0, precision=P.AMG_GNN_FP32)
    try:
        theta = torch.tensor(f32, requires_grad=True)
        c = gcin_coefficients(theta, tr, ctxs)
        rows, losses = 0, []
        for ctx, f in zip(ctxs, fs):
            nl = P.amg_num_levels(ctx)
            losses.append(gnn_amg_loss(c[rows:rows + nl], ctx, f))
            rows += nl
        L = torch.stack(losses).mean()
        L.backward()
        g = theta.grad.numpy()
        # the library's own path: per-problem dL/dc / M, one network backward
        c_np = P.gcin_trainer_forward(tr, ctxs)
        assert np.array_equal(c_np, c.detach().numpy())
        dc, row = np.zeros_like(c_np), 0
        for ctx, f in zip(ctxs, fs):
            nl = P.amg_num_levels(ctx)
            dc[row:row + nl] = P.amg_loss_grad(ctx, c_np[row:row + nl], f, 1)[1] / len(ctxs)
            row += nl
        g_lib = P.gcin_trainer_backward(tr, dc)
        assert np.linalg.norm(g - g_lib) <= 1e-6 * np.linalg.norm(g_lib)
        # the FP64 oracle (autograd through network and V-cycles)
        levels = [OS.build_hierarchy(A) for A in mats]
        Lref, gref = OT.batch_loss_and_grad(f32, [O.OHierarchy.of(lv) for lv in levels],
                                            [[OG.Graph(l.A) for l in lv] for lv in levels], fs)
        assert abs(L.item() - Lref) <= 1e-5 * abs(Lref)
        assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
        # a torch optimiser can drive it: one SGD step lowers the loss
        with torch.no_grad():
            theta -= 1e-3 * theta.grad / theta.grad.norm()
        c2 = gcin_coefficients(theta, tr, ctxs)
        rows, L2 = 0, 0.0
        for ctx, f in zip(ctxs, fs):
            nl = P.amg_num_levels(ctx)
            L2 += float(gnn_amg_loss(c2[rows:rows + nl], ctx, f)) / len(ctxs)
            rows += nl
        assert L2 < L.item()
    finally:
        P.gcin_trainer_destroy(tr)
        for ctx in ctxs:
            P.amg_destroy(ctx)
