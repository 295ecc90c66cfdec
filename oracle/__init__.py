"""Plain FP64 CPU oracle of the GNN-smoothed AMG solve phase.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import or run it; the library itself never does, and it shares no code
with the CUDA path (the only common module is ``workloads``, which generates
inputs and holds none of the method's arithmetic).

Modules
-------
setup   Sec. 2.2 setup phase: classical Ruge-Stueben C/F splitting with strength
        threshold theta (Sec. 4), direct interpolation P, R = P^T, Galerkin
        A_c = R A P, recursion to the coarsest level (Table train_hyper: at
        most 10 levels).
solve   Sec. 2.1 stationary correction, Sec. 2.3 relaxed Jacobi, Sec. 3.1
        sparse pseudo-inverse smoother, Sec. 2.2 V-cycle with a dense Cholesky
        solve on the coarsest level, the solve loop with the Sec. 4 stopping
        rule and divergence / stagnation detection, the Sec. 3.3 relative
        validation metric against Jacobi.
gcin    Sec. 3.2 + App. A.1 GCIN network (4 layers, hidden 64, instance norm,
        ReLU, mean/max jumping-knowledge readout, layer norm, sigmoid, MLP to
        5 coefficients); gradients come from autograd on this FP64 forward.
train   Sec. 3.3 residual-reduction loss through one V-cycle, Algorithm 1 batch
        loss, global-norm clipping and Adam (Table train_hyper).

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, library routines or brute force, except the quality of a trained
network, which no printed value of the paper pins.
"""
