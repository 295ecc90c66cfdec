"""Pins for the oracle's GCIN network (Sec. 3.2, App. A.1) and training
objective (Sec. 3.3).  The forward is checked against an independent build
from torch.nn.functional library layers on a dense adjacency; gradients are
checked against FP64 central finite differences; the optimiser against
torch.optim.Adam and torch.nn.utils.clip_grad_norm_."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import workloads as W
from oracle import gcin as G
from oracle import setup as S
from oracle import solve as O
from oracle import train as T


def test_parameter_count_matches_paper():
    assert G.n_params() == 55045          # App. A.1
    assert sum(s for s, _ in W.GCIN_PARAM_SIZES) == 55045
    # hidden 32 (App. B.3): conv 2*32+32 + 3*(32*32+32), IN 4*64, readout 4*(64*32+32),
    # LN 256 and the unchanged head 16512 + 8256 + 325
    assert G.n_params(32) == 96 + 3168 + 256 + 8320 + 256 + 16512 + 8256 + 325 == 37189
    assert sum(s for s, _ in W.gcin_param_sizes(32)) == 37189
    assert G.hidden_of(55045) == 64 and G.hidden_of(37189) == 32
    with pytest.raises(ValueError):
        G.hidden_of(55044)


def _pad_to_64(theta32):
    """Embed a hidden-32 parameter vector into the hidden-64 layout: the extra
    channels get zero weights in and out, zero bias and zero beta (their gamma
    is random), and the readout rows of their pooled features are random."""
    p32 = G.unpack(torch.from_numpy(theta32))
    rng = np.random.default_rng(7)
    out = []
    for name, shape in G.param_shapes(64):
        t = np.zeros(shape)
        src = p32[name].numpy()
        if name.startswith("conv"):
            t[tuple(slice(0, k) for k in src.shape)] = src
        elif name.endswith("gamma") and name.startswith("in"):
            t[:] = rng.uniform(0.5, 2.0, shape)
            t[:32] = src
        elif name.endswith("beta") and name.startswith("in"):
            t[:32] = src
        elif name.startswith("ro") and name.endswith(".W"):
            t[:] = rng.standard_normal(shape)       # multiplied by exact zeros
            t[0:32] = src[0:32]                     # mean of the 32 live channels
            t[64:96] = src[32:64]                   # max of the 32 live channels
        else:
            t[:] = src
        out.append(t.ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("kind", ["uniform", "band"])
def test_hidden32_equals_zero_padded_hidden64(kind):
    """A hidden-32 network is the hidden-64 network whose extra channels carry
    nothing: zero weights keep them at y = 0, the instance norm maps a constant
    channel to beta = 0 and the ReLU keeps 0, so every pooled feature of those
    channels is 0 and their readout rows add exact zeros."""
    A = W.fv_mesh(kind, 600, 3, max_aspect=100.0)[0]
    levels = S.build_hierarchy(A, max_coarse=20)
    theta32 = W.gcin_init_params(5, last_scale=1.0, hidden=32)
    mats = [l.A for l in levels]
    c32 = G.predict(theta32, mats)
    c64 = G.predict(_pad_to_64(theta32), mats)
    np.testing.assert_allclose(c32, c64, rtol=1e-12, atol=1e-13)
    # and the BF16 evaluation agrees the same way (zeros round to zeros)
    np.testing.assert_allclose(G.predict(theta32, mats, True), G.predict(_pad_to_64(theta32), mats, True),
                               rtol=1e-12, atol=1e-13)
    # the padding is not vacuous: a non-zero bias on an extra channel moves c
    bad = _pad_to_64(theta32)
    off = sum(int(np.prod(s)) for n, s in G.param_shapes(64)[:G.param_shapes(64).index(("in1.beta", (64,)))])
    bad[off + 40] = 0.5
    assert np.abs(G.predict(bad, mats) - c32).max() > 1e-6


def _rne_bf16_bits(t):
    """bfloat16 rounding done on the FP32 bit pattern (round to nearest, ties to
    even): keep the top 16 bits after adding 0x7FFF plus the lowest kept bit."""
    u = t.detach().numpy().astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return torch.from_numpy(u.astype(np.uint32).view(np.float32).astype(np.float64))


def _library_forward(theta, A, bf16=False, acts=False):
    """Same network from library layers: dense A_hat, F.linear, F.instance_norm,
    F.layer_norm (acts: the activations entering layers 2..4 rounded too)."""
    p = G.unpack(torch.from_numpy(theta))
    Ad = torch.from_numpy(A.to_dense())
    n = A.n_rows
    deg = torch.from_numpy((np.diff(A.row_ptr) - 1).astype(np.float64))
    x = torch.stack([torch.diagonal(Ad), deg], 1)
    pooled = []
    for l in range(1, 5):
        h, Wt = Ad @ (_rne_bf16_bits(x) if acts and l > 1 else x), p[f"conv{l}.W"].T
        if bf16 and l > 1:
            h, Wt = _rne_bf16_bits(h), _rne_bf16_bits(Wt)
        y = Fn.linear(h, Wt, p[f"conv{l}.b"])
        if acts:
            # statistics of y (as running statistics), the library's
            # normalisation applied to the BF16-rounded y
            y = Fn.instance_norm(_rne_bf16_bits(y).T.unsqueeze(0), running_mean=y.mean(0),
                                 running_var=y.var(0, unbiased=False), weight=p[f"in{l}.gamma"],
                                 bias=p[f"in{l}.beta"], use_input_stats=False, eps=1e-5)[0].T
        else:
            y = Fn.instance_norm(y.T.unsqueeze(0), weight=p[f"in{l}.gamma"], bias=p[f"in{l}.beta"], eps=1e-5)[0].T
        x = Fn.relu(y)
        g = torch.cat([x.mean(0), x.amax(0)])
        pooled.append(Fn.linear(g, p[f"ro{l}.W"].T, p[f"ro{l}.b"]))
    z = torch.sigmoid(Fn.layer_norm(torch.cat(pooled), (128,), p["ln.gamma"], p["ln.beta"], eps=1e-5))
    z = Fn.relu(Fn.linear(z, p["h1.W"].T, p["h1.b"]))
    z = Fn.relu(Fn.linear(z, p["h2.W"].T, p["h2.b"]))
    return Fn.linear(z, p["h3.W"].T, p["h3.b"])


@pytest.mark.parametrize("hidden", [64, 32])
@pytest.mark.parametrize("kind", ["uniform", "band"])
def test_forward_equals_library_layers(kind, hidden):
    A = W.fv_mesh(kind, 600, 3, max_aspect=100.0)[0]
    levels = S.build_hierarchy(A, max_coarse=20)
    theta = W.gcin_init_params(1, last_scale=1.0, hidden=hidden)
    c = G.predict(theta, [l.A for l in levels])
    for k, lv in enumerate(levels):
        ref = _library_forward(theta, lv.A).numpy()
        np.testing.assert_allclose(c[k], ref, rtol=1e-10, atol=1e-12)


def test_bf16_rounding_ties_to_even():
    v = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 1.0 + 2.0 ** -8 + 2.0 ** -20,
                      3.0e38, 1.0e-40, 0.0])
    r = G.bf16_round(v).numpy()
    assert r[0] == 1.0                       # tie, even neighbour below
    assert r[1] == 1.0 + 2.0 ** -6           # tie, even neighbour above
    assert r[2] == -1.0
    assert r[3] == 1.0 + 2.0 ** -7           # just above the tie
    x = torch.from_numpy(W.uniform_pm1(5, 4096) * 1e3)
    assert torch.equal(G.bf16_round(x), _rne_bf16_bits(x))


@pytest.mark.parametrize("kind", ["uniform", "band"])
def test_bf16_mode_equals_library_layers(kind):
    """BF16 mode rounds exactly the layer 2..4 linear operands."""
    A = W.fv_mesh(kind, 600, 3, max_aspect=100.0)[0]
    levels = S.build_hierarchy(A, max_coarse=20)
    theta = W.gcin_init_params(1, last_scale=1.0)
    c = G.predict(theta, [l.A for l in levels], bf16_linears=True)
    c64 = G.predict(theta, [l.A for l in levels])
    for k, lv in enumerate(levels):
        ref = _library_forward(theta, lv.A, bf16=True).numpy()
        np.testing.assert_allclose(c[k], ref, rtol=1e-10, atol=1e-12)
    # rounding 8-bit mantissas moves the coefficients, but within the BF16 bar
    d = np.abs(c - c64).max() / np.abs(c64).max()
    assert 1e-7 < d < 2e-2


def test_permutation_invariance():
    A = W.fv_mesh("graded", 800, 6)[0]
    perm = np.argsort(W.uniform01(99, A.n_rows))
    Ad = A.to_dense()[np.ix_(perm, perm)]
    r, c = np.nonzero(Ad != 0)
    Ap = W._coo_to_csr(A.n_rows, A.n_rows, r, c, Ad[r, c])
    theta = W.gcin_init_params(2, last_scale=1.0)
    np.testing.assert_allclose(G.predict(theta, [A])[0], G.predict(theta, [Ap])[0], rtol=1e-11, atol=1e-13)


def test_instance_norm_statistics():
    A = W.fv_mesh("uniform", 500, 8)[0]
    theta = W.gcin_init_params(3)
    p = G.unpack(torch.from_numpy(theta))
    keep = []
    with torch.no_grad():
        G.forward_graph(p, G.Graph(A), keep)
    for h, y, x in keep:
        z = (y - y.mean(0)) / torch.sqrt(y.var(0, unbiased=False) + 1e-5)
        np.testing.assert_allclose(z.mean(0).numpy(), 0, atol=1e-12)
        assert torch.all(x >= 0)


def _small_problem(seed, n_pts=400):
    A = W.fv_mesh(["uniform", "graded", "band"][seed % 3], n_pts, seed, max_aspect=100.0)[0]
    levels = S.build_hierarchy(A, max_coarse=16)
    return levels, O.OHierarchy.of(levels), W.rhs_uniform(seed, A.n_rows)


def test_coefficient_gradient_matches_finite_differences():
    levels, h, f = _small_problem(1)
    c = np.array([[0.6, 0.02, -0.01, 0.15, 0.02]] * len(levels))
    L, dc = T.loss_and_coeff_grad(h, c, f)
    eps = 1e-6
    for l in range(len(levels) - 1):
        for k in range(5):
            cp, cm = c.copy(), c.copy()
            cp[l, k] += eps
            cm[l, k] -= eps
            with torch.no_grad():
                fd = (float(T.problem_loss(h, torch.from_numpy(cp), f)) -
                      float(T.problem_loss(h, torch.from_numpy(cm), f))) / (2 * eps)
            assert abs(fd - dc[l, k]) <= 1e-6 * max(1.0, abs(fd)), (l, k, fd, dc[l, k])
    assert np.all(dc[-1] == 0)   # the coarsest level has no smoother


@pytest.mark.parametrize("hidden", [64, 32])
def test_network_gradient_matches_finite_differences(hidden):
    probs = [_small_problem(s) for s in (0, 2)]
    hs = [p[1] for p in probs]
    gs = [[G.Graph(l.A) for l in p[0]] for p in probs]
    fs = [p[2] for p in probs]
    theta = W.gcin_init_params(4, hidden=hidden)
    L, g = T.batch_loss_and_grad(theta, hs, gs, fs)
    rng = np.random.default_rng(0)
    for _ in range(4):
        d = rng.standard_normal(theta.size)
        d /= np.linalg.norm(d)
        eps = 1e-5
        with torch.no_grad():
            lp = float(T.batch_loss(torch.from_numpy(theta + eps * d), hs, gs, fs))
            lm = float(T.batch_loss(torch.from_numpy(theta - eps * d), hs, gs, fs))
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)


def test_adam_and_clip_match_library():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(50)
    t = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.standard_normal(50) * (10.0 if step % 2 else 0.1)
        t.grad = torch.tensor(g.copy())
        torch.nn.utils.clip_grad_norm_([t], 1.0)
        gc = T.clip_grad(g, 1.0)
        np.testing.assert_allclose(t.grad.numpy(), gc, rtol=1e-12)
        opt.step()
        theta, m, v = T.adam_step(theta, gc, m, v, step)
        np.testing.assert_allclose(t.detach().numpy(), theta, rtol=1e-12, atol=1e-15)


def test_jacobi_loss_equals_first_cycle_reduction():
    # with c = (omega, 0, 0, 0, 0) the loss is log10 of the first entry of the
    # Jacobi solve's relative residual history
    levels, h, f = _small_problem(5)
    c = np.array([[2.0 / 3.0, 0, 0, 0, 0]] * len(levels))
    L, _ = T.loss_and_coeff_grad(h, c, f)
    hj = O.OHierarchy.of(levels)
    hj.set_jacobi()
    res = O.solve(hj, f, tol=0.0, max_iter=1)
    assert abs(L - np.log10(res.history[1])) < 1e-12


def test_multi_cycle_loss_telescopes_and_matches_finite_differences():
    # Sec. 3.3: sum_n log10(||r_n|| / ||r_{n-1}||) = log10(||r_N|| / ||r_0||);
    # pinned against the solve's residual history and against FD.
    levels, h, f = _small_problem(4)
    c = np.array([[0.6, 0.02, -0.01, -0.12, 0.02]] * len(levels))
    L3, d3 = T.loss_and_coeff_grad(h, c, f, n_vc=3)
    hp = O.OHierarchy.of(levels)
    hp.set_pseudo_inverse(c)
    res = O.solve(hp, f, tol=0.0, max_iter=3)
    assert abs(L3 - np.log10(res.history[3])) < 1e-12
    eps = 1e-6
    for l, k in ((0, 0), (0, 3), (1, 1), (len(levels) - 2, 4)):
        cp, cm = c.copy(), c.copy()
        cp[l, k] += eps
        cm[l, k] -= eps
        with torch.no_grad():
            fd = (float(T.problem_loss(h, torch.from_numpy(cp), f, n_vc=3)) -
                  float(T.problem_loss(h, torch.from_numpy(cm), f, n_vc=3))) / (2 * eps)
        assert abs(fd - d3[l, k]) <= 1e-6 * max(1.0, abs(fd))


def test_relative_metric_after_n_cycles():
    levels, h, f = _small_problem(5)
    hj = O.OHierarchy.of(levels)
    hj.set_jacobi()
    hg = O.OHierarchy.of(levels)
    hg.set_pseudo_inverse([[2.0 / 3.0, 0, 0, 0, 0]] * len(levels))
    for n in (1, 4):
        assert abs(O.relative_metric(hg, hj, f, n_cycles=n)) < 1e-10
    hb = O.OHierarchy.of(levels)
    hb.set_pseudo_inverse([[3.0, 0, 0, 0, 0]] * len(levels))   # unstable smoother
    assert O.relative_metric(hb, hj, f, n_cycles=6) > 0.5


@pytest.mark.parametrize("kind", ["uniform", "band"])
def test_bf16_inference_mode_equals_library_layers(kind):
    """BF16 inference also rounds the linear outputs before the normalisation
    (statistics from the unrounded ones) and the activations entering layers
    2..4 (the pooling reads the unrounded ones)."""
    A = W.fv_mesh(kind, 600, 3, max_aspect=100.0)[0]
    levels = S.build_hierarchy(A, max_coarse=20)
    theta = W.gcin_init_params(1, last_scale=1.0)
    c = G.predict(theta, [l.A for l in levels], bf16_linears=True, bf16_acts=True)
    cl = G.predict(theta, [l.A for l in levels], bf16_linears=True)
    for k, lv in enumerate(levels):
        ref = _library_forward(theta, lv.A, bf16=True, acts=True).numpy()
        np.testing.assert_allclose(c[k], ref, rtol=1e-10, atol=1e-12)
    d = np.abs(c - cl).max() / np.abs(cl).max()
    assert 1e-7 < d < 2e-2
