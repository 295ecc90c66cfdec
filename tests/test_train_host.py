"""Host logic of the training loop (Sec. 3.3 validation metric as the early
stopping criterion; ReduceLROnPlateau): best-validation bookkeeping and the
learning-rate schedule, driven with a fake parameter source (no GPU)."""
import math

import numpy as np

from paper_2606_19251_gb300.train import Trainer


class _Fake(Trainer):
    def __init__(self, patience, factor=0.1, lr=1e-3):
        # the library trainer is not created: params() returns a counter
        self.tr = None
        self.n_vc, self.val_cycles = 1, 10
        self.lr, self.max_norm = lr, 1.0
        self.factor, self.patience = factor, patience
        self.best_val, self.best_theta, self.bad_epochs = math.inf, None, 0
        self.calls = 0

    def params(self):
        self.calls += 1
        return np.array([float(self.calls)])


def test_best_validation_parameters_are_kept():
    t = _Fake(patience=10)
    for v in (0.0, -0.3, -0.1, -0.5, -0.2):
        t.end_epoch(v)
    # the best value (-0.5) came at the 4th epoch, the 3rd improvement
    assert t.best_val == -0.5
    assert t.best_theta.tolist() == [3.0]


def test_learning_rate_drops_after_patience_epochs_without_improvement():
    t = _Fake(patience=2)
    lrs = []
    for v in (-0.1, -0.2, -0.2, -0.15, -0.19, -0.3, -0.3, -0.3, -0.3):
        t.end_epoch(v)
        lrs.append(t.lr)
    # epochs 3-5 do not improve: the third one (bad_epochs > patience) drops lr
    np.testing.assert_allclose(lrs, [1e-3, 1e-3, 1e-3, 1e-3, 1e-4, 1e-4, 1e-4, 1e-4, 1e-5], rtol=1e-12)
    assert t.best_val == -0.3
