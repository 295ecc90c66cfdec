"""Training of the GCIN coefficient network (Sec. 3.3, Algorithm 1, Table train_hyper).

Host-side loop only; every forward, adjoint and optimiser step runs in the
library's CUDA kernels:
  1. batched GCIN inference over every level of every problem of the
     mini-batch (gcin_trainer_forward; Algorithm 1 steps 1-6);
  2. per problem, N_vc V-cycles from u_0 = 0 with the predicted smoothers
     and the loss sum_{n=1}^{N_vc} log10(||r_n|| / ||r_{n-1}||) (it telescopes
     to log10(||r_{N_vc}|| / ||f||)), with its gradient dL/dc from the
     hand-written V-cycle adjoint (amg_loss_grad; steps 7-12; N_vc = 1 is the
     primary loss).  The training loss of a problem is that sum divided by
     N_vc: Sec. 3.3 describes the multi-V-cycle loss as averaging the
     reductions over the cycles (a reading of the equation's sum; it keeps
     the gradient scale of the N_vc = 1 loss, to which the clipping norm of
     1.0 applies).  The batch loss is the mean over the problems;
  3. backward through the network of the batch-mean loss, global-norm
     clipping to 1.0 and Adam with lr 1e-3 (gcin_trainer_backward /
     gcin_trainer_adam_step; step 13).
Validation uses the relative metric log10(||r^GNN|| / ||r^Jacobi||) after
`val_cycles` V-cycles (Sec. 3.3); the best-validation parameters are kept (early stopping,
App. B.1) and the learning rate follows ReduceLROnPlateau (factor 0.1,
patience 10; the factor and patience are readings).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import api as P


class Problem:
    """One matrix with its hierarchy on the device."""

    def __init__(self, A, precision=P.AMG_FP32_IN_FP64, device=0):
        self.A = A
        self.ctx = P.amg_create(precision=precision, device=device)
        P.amg_setup(self.ctx, A)
        self.n_levels = P.amg_num_levels(self.ctx)

    def close(self):
        if self.ctx is not None:
            P.amg_destroy(self.ctx)
            self.ctx = None


class Trainer:
    def __init__(self, theta0, device=0, lr=1e-3, max_norm=1.0, factor=0.1, patience=10, n_vc=1, val_cycles=10,
                 precision=P.AMG_GNN_FP32):
        self.tr = P.gcin_trainer_create(theta0, device, precision)
        self.n_vc, self.val_cycles = n_vc, val_cycles
        self.lr, self.max_norm = lr, max_norm
        self.factor, self.patience = factor, patience
        self.best_val, self.best_theta, self.bad_epochs = math.inf, None, 0
        self.history = []

    def step(self, problems, rhs):
        """One optimiser step on a mini-batch; returns the mean loss."""
        c = P.gcin_trainer_forward(self.tr, [p.ctx for p in problems])
        dc = np.zeros_like(c)
        losses, row = [], 0
        for p, f in zip(problems, rhs):
            L, g = P.amg_loss_grad(p.ctx, c[row:row + p.n_levels], f, self.n_vc)
            losses.append(L / self.n_vc)
            dc[row:row + p.n_levels] = g / (len(problems) * self.n_vc)
            row += p.n_levels
        if not np.all(np.isfinite(dc)):
            return float("nan")
        P.gcin_trainer_backward(self.tr, dc)
        P.gcin_trainer_adam_step(self.tr, self.lr, self.max_norm)
        return float(np.mean(losses))

    def params(self):
        return P.gcin_trainer_get_params(self.tr)

    def validate(self, problems, rhs):
        """Mean relative metric vs Jacobi (negative = better than Jacobi)."""
        theta = self.params()
        out = []
        for p, f in zip(problems, rhs):
            P.gnn_load_params(p.ctx, theta)
            P.gnn_predict_coeffs(p.ctx)
            out.append(P.amg_judge(p.ctx, f, self.val_cycles))
        return float(np.mean(out))

    def end_epoch(self, val):
        """Early stopping bookkeeping and ReduceLROnPlateau."""
        if val < self.best_val:
            self.best_val, self.best_theta, self.bad_epochs = val, self.params().copy(), 0
        else:
            self.bad_epochs += 1
            if self.bad_epochs > self.patience:
                self.lr *= self.factor
                self.bad_epochs = 0

    def close(self):
        if self.tr is not None:
            P.gcin_trainer_destroy(self.tr)
            self.tr = None


def train(train_mats, val_mats, theta0, epochs=30, batch=5, seed=0, log=print, device=0, n_vc=1, val_cycles=10,
          precision=P.AMG_GNN_FP32, factor=0.1, patience=10):
    """Train on `train_mats`, validate on `val_mats`; returns (best theta, log rows)."""
    import workloads as W
    probs = [Problem(A, device=device) for A in train_mats]
    vals = [Problem(A, device=device) for A in val_mats]
    val_rhs = [W.rhs_uniform(10_000 + k, p.A.n_rows) for k, p in enumerate(vals)]
    tr = Trainer(theta0, device=device, n_vc=n_vc, val_cycles=val_cycles, precision=precision, factor=factor,
                 patience=patience)
    rows = []
    try:
        val0 = tr.validate(vals, val_rhs)
        rows.append({"epoch": 0, "loss": None, "val": val0, "lr": tr.lr})
        log(rows[-1])
        tr.end_epoch(val0)
        step = 0
        for ep in range(1, epochs + 1):
            order = np.argsort(W.uniform01(seed * 7919 + ep, len(probs)))
            t0 = time.perf_counter()
            losses = []
            for s in range(0, len(order), batch):
                idx = order[s:s + batch]
                mb = [probs[i] for i in idx]
                rhs = [W.rhs_uniform(1_000_000 * (seed + 1) + step * 97 + k, p.A.n_rows) for k, p in enumerate(mb)]
                losses.append(tr.step(mb, rhs))
                step += 1
            val = tr.validate(vals, val_rhs)
            tr.end_epoch(val)
            rows.append({"epoch": ep, "loss": float(np.nanmean(losses)), "val": val, "lr": tr.lr,
                         "sec": time.perf_counter() - t0})
            log(rows[-1])
        best = tr.best_theta if tr.best_theta is not None else tr.params()
        return best, rows
    finally:
        tr.close()
        for p in probs + vals:
            p.close()
