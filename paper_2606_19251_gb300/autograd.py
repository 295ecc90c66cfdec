"""PyTorch autograd entry points over the library's training kernels (Sec. 3.3,
Algorithm 1).  Marshalling only: the V-cycles, their hand-written adjoint and
the network's forward and backward all run in libamggnn.so.

    c = gcin_coefficients(theta, trainer, problems)      # (sum_m L_m) x 5
    L = gnn_amg_loss(c[rows_m], problems[m], f_m, n_vc)  # per problem
    L.backward()                                          # theta.grad

so any torch optimiser can drive the training loop that train.Trainer runs
with the library's own clipping and Adam.
"""
from __future__ import annotations

import torch

from . import api as P


class GnnAmgLoss(torch.autograd.Function):
    """L(c) = sum_{n=1}^{n_vc} log10(||r_n|| / ||r_{n-1}||) for one problem
    (context `amg`, right-hand side f, u_0 = 0), c: (n_levels, 5); dL/dc from
    the V-cycle adjoint (amg_loss_grad)."""

    @staticmethod
    def forward(ctx, c, amg, f, n_vc=1):
        L, dc = P.amg_loss_grad(amg, c.detach().cpu().double().numpy(), f, n_vc)
        ctx.save_for_backward(torch.as_tensor(dc, dtype=c.dtype).to(c.device))
        return torch.tensor(L, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, g):
        (dc,) = ctx.saved_tensors
        return g * dc, None, None, None


class GcinCoefficients(torch.autograd.Function):
    """c = GCIN(theta) for every level of every problem (gcin_trainer_forward
    after loading theta into the trainer); the parameter gradient from the
    network's backward kernels (gcin_trainer_backward)."""

    @staticmethod
    def forward(ctx, theta, trainer, problems):
        P.gcin_trainer_set_params(trainer, theta.detach().cpu().numpy())
        c = P.gcin_trainer_forward(trainer, problems)
        ctx.trainer = trainer
        return torch.as_tensor(c, dtype=theta.dtype).to(theta.device)

    @staticmethod
    def backward(ctx, dc):
        g = P.gcin_trainer_backward(ctx.trainer, dc.detach().cpu().double().numpy())
        return torch.as_tensor(g, dtype=dc.dtype).to(dc.device), None, None


def gnn_amg_loss(c, amg, f, n_vc=1):
    return GnnAmgLoss.apply(c, amg, f, n_vc)


def gcin_coefficients(theta, trainer, problems):
    return GcinCoefficients.apply(theta, trainer, problems)
