"""Training objective and optimiser (Sec. 3.3, Algorithm 1, Table train_hyper).

Test infrastructure only.  FP64; gradients by autograd through the plain
V-cycle of ``oracle.solve`` and the network of ``oracle.gcin``.

* loss of one problem with u_0 = 0 (Sec. 3.3, multi-V-cycle form):
  L_m = sum_{n=1}^{N_vc} log10(||r_n||_2 / ||r_{n-1}||_2), r_n = f - A u_n,
  u_n = V-cycle(u_{n-1}, f); N_vc = 1 is the primary loss;
* batch loss = mean over problems (Algorithm 1 steps 7-12); with
  average_cycles, each L_m is divided by N_vc first (Sec. 3.3 describes the
  multi-V-cycle loss as averaging the reductions over the cycles; the
  training loop uses that form, amg_loss_grad returns the sum);
* global-norm clipping to 1.0 (Table train_hyper) as g * min(1, 1/(||g|| + 1e-6))
  (reading; the paper gives only the max norm);
* Adam with lr 1e-3 (Table train_hyper); beta1 = 0.9, beta2 = 0.999,
  eps = 1e-8 (reading: the paper names only Adam and its learning rate).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gcin
from .solve import DT, OHierarchy, mv, pseudo_inverse_values, vcycle

LOG10 = math.log(10.0)


def problem_loss(h: OHierarchy, coeffs: torch.Tensor, f, nu1: int = 2, nu2: int = 2, n_vc: int = 1) -> torch.Tensor:
    """L_m for one problem; coeffs (n_levels, 5) may require grad."""
    f = torch.as_tensor(np.asarray(f, dtype=np.float64))
    for l, lv in enumerate(h.levels[:-1]):
        lv.M = pseudo_inverse_values(lv.A, coeffs[l], lv.s)
    A = h.levels[0].A
    u = torch.zeros_like(f)
    r_prev = torch.linalg.vector_norm(f)
    L = 0.0
    for _ in range(n_vc):
        u = vcycle(h, f, u, nu1, nu2)
        r = torch.linalg.vector_norm(f - mv(A, u))
        L = L + torch.log10(r / r_prev)
        r_prev = r
    return L


def loss_and_coeff_grad(h: OHierarchy, coeffs, f, n_vc: int = 1):
    """(L_m, dL_m/dc) for one problem, c of shape (n_levels, 5)."""
    c = torch.as_tensor(np.asarray(coeffs, dtype=np.float64)).clone().requires_grad_(True)
    L = problem_loss(h, c, f, n_vc=n_vc)
    L.backward()
    return float(L.detach()), c.grad.numpy().copy()


def batch_loss(theta: torch.Tensor, hierarchies, graphs_per_problem, rhs, n_vc: int = 1,
               average_cycles: bool = False, bf16_linears: bool = False) -> torch.Tensor:
    """Algorithm 1: batched inference over all levels, then per-problem losses, mean."""
    all_graphs = [g for gs in graphs_per_problem for g in gs]
    c_all = gcin.forward(theta, all_graphs, bf16_linears=bf16_linears)
    total, off = 0.0, 0
    for h, gs, f in zip(hierarchies, graphs_per_problem, rhs):
        L_m = problem_loss(h, c_all[off:off + len(gs)], f, n_vc=n_vc)
        total = total + (L_m / n_vc if average_cycles else L_m)
        off += len(gs)
    return total / len(hierarchies)


def batch_loss_and_grad(theta, hierarchies, graphs_per_problem, rhs, n_vc: int = 1, average_cycles: bool = False,
                        bf16_linears: bool = False):
    t = torch.as_tensor(np.asarray(theta, dtype=np.float64)).clone().requires_grad_(True)
    L = batch_loss(t, hierarchies, graphs_per_problem, rhs, n_vc=n_vc, average_cycles=average_cycles,
                   bf16_linears=bf16_linears)
    L.backward()
    return float(L.detach()), t.grad.numpy().copy()


def clip_grad(g: np.ndarray, max_norm: float = 1.0) -> np.ndarray:
    norm = float(np.sqrt(np.sum(g * g)))
    return g * min(1.0, max_norm / (norm + 1e-6))


def adam_step(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
