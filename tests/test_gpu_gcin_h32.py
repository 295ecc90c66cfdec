"""GPU parity of the hidden-32 GCIN (the halved width of App. B.3) against the
FP64 oracle at width 32, through the same C ABI as the width-64 network: the
width follows from the length of the parameter vector.

Bars as for width 64: coefficients within 1e-5 relative (FP32 node linears)
or, for inference on the tensor cores (tcgen05 node linears, N = 32 MMAs,
activations stored in BF16), 2e-2 of the FP64 oracle on the vector's scale
(5e-2 per column) and 4e-3 of the oracle's BF16 inference mode; the
training forward 1e-3 of the BF16-operand oracle; network gradients within
1e-4 (FP32) and 1e-2 (BF16) in norm; the clipped Adam step as in the width-64 test.
"""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W
from oracle import gcin as OG
from oracle import setup as OS
from oracle import solve as O
from oracle import train as OT
from tests.gpu_helpers import ctx_setup

pytestmark = pytest.mark.gpu

H = 32


def f32(theta):
    return np.asarray(theta, dtype=np.float32).astype(np.float64)


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def rel_cols(a, b):
    """Largest relative error of the coefficient columns (d0, d1, d2, o1, o2),
    each against its own scale: a small column (d2 and o2 are often ~1e-2)
    is held to the same relative bar as the largest one."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, 5)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 5)
    return max(float(np.abs(a[:, k] - b[:, k]).max() / max(np.abs(b[:, k]).max(), 1e-30)) for k in range(5))


MATS = {
    "c1_64": lambda: W.poisson5(64),
    "poisson7_16": lambda: W.poisson7(16),
    "uniform_2k": lambda: W.fv_mesh("uniform", 2000, 3)[0],
    "graded_6k": lambda: W.fv_mesh("graded", 6000, 4)[0],
    "band_8k": lambda: W.fv_mesh("band", 8000, 5, max_aspect=100.0)[0],
}


def test_parameter_count():
    assert P.AMG_GCIN_NUM_PARAMS_H32 == OG.n_params(H) == W.gcin_init_params(0, hidden=H).size


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("seed", [0, 7])
def test_predict_coeffs_parity_fp32(name, seed):
    A = MATS[name]()
    theta = W.gcin_init_params(seed, last_scale=1.0, hidden=H)
    levels = OS.build_hierarchy(A)
    ref = OG.predict(f32(theta), [l.A for l in levels])
    ctx = ctx_setup(A, P.AMG_FP32_IN_FP64, gnn_precision=P.AMG_GNN_FP32)
    try:
        P.gnn_load_params(ctx, theta)
        c = P.gnn_predict_coeffs(ctx)
        assert c.shape == ref.shape
        assert rel_cols(c, ref) < 1e-5, rel_cols(c, ref)
        q = P.amg_get_smoother(ctx, 0)
        qref = O.pseudo_inverse_values(O.TMat.of(levels[0].A), c[0])
        assert rel(q, qref.numpy()) < 1e-12
    finally:
        P.amg_destroy(ctx)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("seed", [0, 7])
def test_predict_coeffs_parity_bf16(name, seed):
    A = MATS[name]()
    theta = W.gcin_init_params(seed, last_scale=1.0, hidden=H)
    levels = OS.build_hierarchy(A)
    ref = OG.predict(f32(theta), [l.A for l in levels])
    emu = OG.predict(f32(theta), [l.A for l in levels], bf16_linears=True, bf16_acts=True)
    ctx = ctx_setup(A, P.AMG_FP32_IN_FP64)
    try:
        P.gnn_load_params(ctx, theta)
        c = P.gnn_predict_coeffs(ctx)
        assert rel(c, ref) < 2e-2 and rel_cols(c, ref) < 5e-2, (rel(c, ref), rel_cols(c, ref))
        assert rel_cols(c, emu) < 4e-3, rel_cols(c, emu)
    finally:
        P.amg_destroy(ctx)


def test_predict_full_size_c2_bf16_and_width_switch():
    """Full-size mesh (ragged tiles in every graph); the same context then
    switches to a width-64 network and back, each matching its oracle."""
    A = W.c2_matrix(0)
    levels = OS.build_hierarchy(A)
    mats = [l.A for l in levels]
    t32 = W.gcin_init_params(3, last_scale=1.0, hidden=H)
    t64 = W.gcin_init_params(3, last_scale=1.0)
    ctx = ctx_setup(A, P.AMG_FP32_IN_FP64)
    try:
        for theta in (t32, t64, t32):
            P.gnn_load_params(ctx, theta)
            c = P.gnn_predict_coeffs(ctx)
            cf = OG.predict(f32(theta), mats)
            # BF16 against FP64: 2e-2 on the vector's scale, ~3 % per column at most
            assert rel(c, cf) < 2e-2 and rel_cols(c, cf) < 5e-2, (rel(c, cf), rel_cols(c, cf))
            assert rel_cols(c, OG.predict(f32(theta), mats, bf16_linears=True, bf16_acts=True)) < 4e-3
            assert np.array_equal(c, P.gnn_predict_coeffs(ctx))   # deterministic replay
    finally:
        P.amg_destroy(ctx)


def test_wrong_parameter_count_is_rejected():
    ctx = ctx_setup(W.poisson5(16), P.AMG_FP32_IN_FP64)
    try:
        with pytest.raises(P.AmgError) as e:
            P.gnn_load_params(ctx, np.zeros(OG.n_params(H) + 1, np.float32))
        assert e.value.code == P.AMG_ERR_ARG
    finally:
        P.amg_destroy(ctx)
    with pytest.raises(ValueError):
        P.gcin_trainer_create(np.zeros(1000, np.float32))


def _problems(names=("uniform_2k", "graded_6k", "band_8k")):
    out = []
    for k, nm in enumerate(names):
        A = MATS[nm]()
        out.append((A, OS.build_hierarchy(A), W.rhs_uniform(100 + k, A.n_rows)))
    return out


@pytest.mark.parametrize("prec", [P.AMG_GNN_FP32, P.AMG_GNN_BF16])
def test_network_backward_parity(prec):
    probs = _problems()
    theta = W.gcin_init_params(11, last_scale=1.0, hidden=H)
    ctxs = [ctx_setup(A, P.AMG_FP32_IN_FP64) for A, _, _ in probs]
    tr = P.gcin_trainer_create(theta, precision=prec)
    try:
        c = P.gcin_trainer_forward(tr, ctxs)
        dc = np.random.default_rng(0).standard_normal(c.shape)
        g = P.gcin_trainer_backward(tr, dc)
        assert g.size == OG.n_params(H)
        t = torch.tensor(f32(theta), requires_grad=True)
        graphs = [OG.Graph(l.A) for _, lv, _ in probs for l in lv]
        bf16 = prec == P.AMG_GNN_BF16
        cref = OG.forward(t, graphs, bf16_linears=bf16)
        (cref * torch.from_numpy(dc)).sum().backward()
        gref = t.grad.numpy()
        if not bf16:
            assert rel_cols(c, cref.detach().numpy()) < 1e-5
            assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
            off = 0
            for name, shape in OG.param_shapes(H):
                k = int(np.prod(shape))
                gs, rs = g[off:off + k], gref[off:off + k]
                off += k
                if name.startswith("conv") and name.endswith(".b"):   # exactly zero (instance norm)
                    assert np.abs(rs).max() <= 1e-8 * np.abs(gref).max()
                    continue
                assert np.linalg.norm(gs - rs) <= 1e-3 * max(np.linalg.norm(rs), 1e-6 * np.linalg.norm(gref)), name
        else:
            assert rel_cols(c, cref.detach().numpy()) < 1e-3
            assert np.linalg.norm(g - gref) <= 1e-2 * np.linalg.norm(gref)
    finally:
        P.gcin_trainer_destroy(tr)
        for c_ in ctxs:
            P.amg_destroy(c_)


def test_training_step_matches_oracle():
    probs = _problems()
    theta = W.gcin_init_params(21, hidden=H)
    ctxs = [ctx_setup(A, P.AMG_FP64) for A, _, _ in probs]
    tr = P.gcin_trainer_create(theta, precision=P.AMG_GNN_FP32)
    try:
        c = P.gcin_trainer_forward(tr, ctxs)
        dc, losses, row = np.zeros_like(c), [], 0
        for ctx, (A, lv, f) in zip(ctxs, probs):
            nl = P.amg_num_levels(ctx)
            L, g = P.amg_loss_grad(ctx, c[row:row + nl], f)
            losses.append(L)
            dc[row:row + nl] = g / len(probs)
            row += nl
        grad = P.gcin_trainer_backward(tr, dc)
        hs = [O.OHierarchy.of(lv) for _, lv, _ in probs]
        gs = [[OG.Graph(l.A) for l in lv] for _, lv, _ in probs]
        Lref, gref = OT.batch_loss_and_grad(f32(theta), hs, gs, [f for _, _, f in probs])
        assert abs(np.mean(losses) - Lref) <= 1e-5 * abs(Lref)
        assert np.linalg.norm(grad - gref) <= 1e-4 * np.linalg.norm(gref)
        P.gcin_trainer_adam_step(tr, 1e-3, 1.0)
        new = P.gcin_trainer_get_params(tr).astype(np.float64)
        assert new.size == OG.n_params(H)
        ref, _, _ = OT.adam_step(f32(theta), OT.clip_grad(gref, 1.0), np.zeros_like(gref), np.zeros_like(gref), 1)
        d = np.abs(new - ref)
        assert d.max() <= 2.1e-3
        assert np.mean(d < 1e-6) > 0.98
    finally:
        P.gcin_trainer_destroy(tr)
        for c_ in ctxs:
            P.amg_destroy(c_)
