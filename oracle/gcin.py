"""GCIN coefficient network (Sec. 3.2, App. A.1) in plain FP64 torch ops.

Test infrastructure only.  Gradients are taken by autograd on this forward.

Per level graph G = (V, E) of a matrix A (Sec. 3.2, Algorithm 1 steps 3-5):
node features x_i^(0) = [a_ii, deg(v_i)] with deg = number of off-diagonal
pattern entries of row i; edge weights w_ij = a_ij; the self-loop of
A_hat carries w_ii = a_ii (reading: A_hat = A).

Layer l = 1..4 (Eq. GCN + App. A.1):
    h_i = sum_{j in N(i) u {i}} w_ij x_j^(l-1)      (no GCN normalisation)
    y   = h Theta^(l) + b^(l)                         (MLP^(l) = one Linear)
    x^(l) = ReLU(InstanceNorm_graph(y))               (eps 1e-5, biased var, affine)
Readout (JK-like, Sec. 3.2 readout equations; App. A.1):
    g^(l) = Linear_{128->32}([mean_i x_i^(l), max_i x_i^(l)])   for l = 1..4
    z = sigmoid(LayerNorm_128(concat_l g^(l)))                  (eps 1e-5)
    c = Linear_{64->5}(ReLU(Linear_{128->64}(ReLU(Linear_{128->128}(z)))))
This layout has exactly 55,045 trainable parameters (App. A.1).

Hidden width H (App. B.3 halves it to 32 for structured meshes): every 64 above
that is the GCIN width becomes H (conv and instance-norm widths, readout
input 2H); the readout output (32 per layer), the 128-vector and the head
are unchanged (reading).  H = 32 has 37,189 parameters.  The width is
inferred from the length of the parameter vector.
Readings: no activation after the readout linears, linear output on the five
coefficients, max-pooling after the ReLU, readout over layers 1..L only.

BF16 mode (bf16_linears=True): the network evaluated with the operands of the
layer 2..4 node linears, h and Theta^(l), rounded to bfloat16 (round to
nearest, ties to even, from their FP32 values), everything else in FP64.  This
is the arithmetic of a tensor-core evaluation with BF16 operands and exact (or
FP32) accumulation; under autograd the rounding passes gradients straight
through.  BF16 inference (bf16_acts=True as well): the linear outputs y of
layers 1..4 are stored in bfloat16 (the instance-norm statistics come from the
unrounded y, the normalisation is applied to the rounded copy), and the
activations x that enter the aggregation of layers 2..4 are rounded to
bfloat16 too; the pooling of each layer reads the unrounded x.

Flat parameter order (weights stored [in][out], row-major; then bias):
conv1 W(2x64) b(64); conv2..4 W(64x64) b(64); IN1..4 gamma(64) beta(64);
readout1..4 W(128x32) b(32); LN gamma(128) beta(128);
head W(128x128) b(128), W(128x64) b(64), W(64x5) b(5).
"""
from __future__ import annotations

import numpy as np
import torch

from workloads import CSR

DT = torch.float64
HIDDEN = 64
WIDTHS = (64, 32)
N_LAYERS = 4
EPS = 1e-5


def param_shapes(hidden: int = HIDDEN):
    H = hidden
    shapes = [("conv1.W", (2, H)), ("conv1.b", (H,))]
    for l in range(2, N_LAYERS + 1):
        shapes += [(f"conv{l}.W", (H, H)), (f"conv{l}.b", (H,))]
    for l in range(1, N_LAYERS + 1):
        shapes += [(f"in{l}.gamma", (H,)), (f"in{l}.beta", (H,))]
    for l in range(1, N_LAYERS + 1):
        shapes += [(f"ro{l}.W", (2 * H, 32)), (f"ro{l}.b", (32,))]
    shapes += [("ln.gamma", (128,)), ("ln.beta", (128,))]
    shapes += [("h1.W", (128, 128)), ("h1.b", (128,)), ("h2.W", (128, 64)), ("h2.b", (64,)),
               ("h3.W", (64, 5)), ("h3.b", (5,))]
    return shapes


def n_params(hidden: int = HIDDEN) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(hidden))


def hidden_of(n: int) -> int:
    """GCIN width of a parameter vector of length n."""
    for H in WIDTHS:
        if n == n_params(H):
            return H
    raise ValueError(f"no GCIN width has {n} parameters")


def unpack(theta: torch.Tensor) -> dict:
    out, off = {}, 0
    for name, shape in param_shapes(hidden_of(theta.numel())):
        k = int(np.prod(shape))
        out[name] = theta[off:off + k].reshape(shape)
        off += k
    assert off == theta.numel(), (off, theta.numel())
    return out


class Graph:
    """One level's matrix as a graph (Algorithm 1 steps 3-4)."""

    def __init__(self, A: CSR):
        self.n = A.n_rows
        self.row = torch.from_numpy(np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr)).astype(np.int64))
        self.col = torch.from_numpy(A.col.astype(np.int64))
        self.w = torch.from_numpy(A.val.astype(np.float64))
        on = self.row == self.col
        self.diag = torch.zeros(self.n, dtype=DT).index_add(0, self.row[on], self.w[on])
        self.deg = torch.zeros(self.n, dtype=DT).index_add(0, self.row[~on], torch.ones(int((~on).sum()), dtype=DT))

    def features(self) -> torch.Tensor:
        return torch.stack([self.diag, self.deg], dim=1)

    def aggregate(self, x: torch.Tensor) -> torch.Tensor:
        """h_i = sum_j w_ij x_j over row i of A_hat (diagonal = self-loop)."""
        return torch.zeros(self.n, x.shape[1], dtype=DT).index_add(0, self.row, self.w[:, None] * x[self.col])


def instance_norm(y: torch.Tensor, gamma, beta, applied_to=None) -> torch.Tensor:
    """InstanceNorm with statistics of y, applied to y (or to `applied_to`, a
    rounded copy of y in BF16 inference)."""
    mu = y.mean(dim=0)
    var = ((y - mu) ** 2).mean(dim=0)
    v = y if applied_to is None else applied_to
    return (v - mu) / torch.sqrt(var + EPS) * gamma + beta


def layer_norm(z: torch.Tensor, gamma, beta) -> torch.Tensor:
    mu = z.mean()
    var = ((z - mu) ** 2).mean()
    return (z - mu) / torch.sqrt(var + EPS) * gamma + beta


def bf16_round(t: torch.Tensor) -> torch.Tensor:
    """Round to the nearest bfloat16 (ties to even) via FP32; returned in FP64."""
    return t.to(torch.float32).to(torch.bfloat16).to(DT)


def forward_graph(p: dict, g: Graph, keep=None, bf16_linears=False, bf16_acts=False) -> torch.Tensor:
    """Coefficients c (5,) for one graph."""
    x = g.features()
    pooled = []
    for l in range(1, N_LAYERS + 1):
        h = g.aggregate(bf16_round(x) if bf16_acts and l >= 2 else x)
        Wl = p[f"conv{l}.W"]
        if bf16_linears and l >= 2:
            h, Wl = bf16_round(h), bf16_round(Wl)
        y = h @ Wl + p[f"conv{l}.b"]
        x = torch.relu(instance_norm(y, p[f"in{l}.gamma"], p[f"in{l}.beta"],
                                     applied_to=bf16_round(y) if bf16_acts else None))
        if keep is not None:
            keep.append((h, y, x))
        gl = torch.cat([x.mean(dim=0), x.max(dim=0).values])
        pooled.append(gl @ p[f"ro{l}.W"] + p[f"ro{l}.b"])
    z = torch.sigmoid(layer_norm(torch.cat(pooled), p["ln.gamma"], p["ln.beta"]))
    z = torch.relu(z @ p["h1.W"] + p["h1.b"])
    z = torch.relu(z @ p["h2.W"] + p["h2.b"])
    return z @ p["h3.W"] + p["h3.b"]


def forward(theta, graphs, bf16_linears=False, bf16_acts=False) -> torch.Tensor:
    """Batched inference (Algorithm 1 step 6): c[g] for every graph, shape (G, 5)."""
    theta = torch.as_tensor(theta, dtype=DT) if not isinstance(theta, torch.Tensor) else theta
    p = unpack(theta)
    return torch.stack([forward_graph(p, g, bf16_linears=bf16_linears, bf16_acts=bf16_acts) for g in graphs])


def predict(theta, matrices, bf16_linears=False, bf16_acts=False) -> np.ndarray:
    """Coefficients for a list of CSR matrices (no gradient)."""
    with torch.no_grad():
        return forward(torch.as_tensor(np.asarray(theta, dtype=np.float64)), [Graph(A) for A in matrices],
                       bf16_linears, bf16_acts).numpy()
