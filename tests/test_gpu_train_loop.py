"""The training loop of the library (paper_2606_19251_gb300/train.py) on
GB300: one Trainer.step with the multi-V-cycle loss (N_vc = 2, averaged over
the cycles as Sec. 3.3 describes it) against the oracle's autograd of the
same batch loss followed by clipping and Adam, and a short run of train()
whose logged learning rates follow the ReduceLROnPlateau rule and whose
returned parameters are the best-validation ones (Sec. 3.3 early stopping)."""
import math

import numpy as np
import pytest

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import gcin as OG
from oracle import setup as OS
from oracle import solve as O
from oracle import train as OT
from paper_2606_19251_gb300 import train as T

pytestmark = pytest.mark.gpu


def _mats():
    return [W.fv_mesh("uniform", 2000, 3)[0], W.fv_mesh("graded", 3000, 4)[0],
            W.fv_mesh("band", 2500, 5, max_aspect=100.0)[0]]


def test_trainer_step_multi_cycle_matches_oracle():
    mats = _mats()
    theta = W.gcin_init_params(21)
    f32 = np.asarray(theta, dtype=np.float32).astype(np.float64)
    probs = [T.Problem(A, precision=P.AMG_FP64) for A in mats]
    rhs = [W.rhs_uniform(300 + k, A.n_rows) for k, A in enumerate(mats)]
    tr = T.Trainer(theta, n_vc=2, precision=P.AMG_GNN_FP32)
    try:
        loss = tr.step(probs, rhs)
        new = tr.params().astype(np.float64)
        levels = [OS.build_hierarchy(A) for A in mats]
        hs = [O.OHierarchy.of(lv) for lv in levels]
        gs = [[OG.Graph(l.A) for l in lv] for lv in levels]
        Lref, gref = OT.batch_loss_and_grad(f32, hs, gs, rhs, n_vc=2, average_cycles=True)
        assert abs(loss - Lref) <= 1e-5 * abs(Lref), (loss, Lref)
        ref, _, _ = OT.adam_step(f32, OT.clip_grad(gref, 1.0), np.zeros_like(gref), np.zeros_like(gref), 1)
        d = np.abs(new - ref)
        assert d.max() <= 2.1e-3
        assert np.mean(d < 1e-6) > 0.98
    finally:
        tr.close()
        for p in probs:
            p.close()


def test_train_loop_schedule_and_best_parameters():
    mats = _mats()
    val_mats = [W.fv_mesh("graded", 2200, 91)[0], W.fv_mesh("band", 2400, 92, max_aspect=100.0)[0]]
    theta0 = W.gcin_init_params(0)
    rows = []
    best, _ = T.train(mats, val_mats, theta0, epochs=4, batch=2, log=rows.append, n_vc=1, val_cycles=4,
                      patience=0, factor=0.5)
    assert len(rows) == 5 and rows[0]["epoch"] == 0
    # replay ReduceLROnPlateau (patience 0: every epoch without a new best halves lr)
    best_val, lr = math.inf, 1e-3
    for r in rows:
        if r["val"] < best_val:
            best_val = r["val"]
        else:
            lr *= 0.5
        assert r["lr"] == pytest.approx(lr, rel=1e-12), rows
    # the returned parameters reproduce the best validation value exactly
    vals = [T.Problem(A) for A in val_mats]
    tr = T.Trainer(best, val_cycles=4)
    try:
        val_rhs = [W.rhs_uniform(10_000 + k, p.A.n_rows) for k, p in enumerate(vals)]
        assert tr.validate(vals, val_rhs) == best_val
    finally:
        tr.close()
        for p in vals:
            p.close()
