"""The tensor-core GCIN layer kernel in isolation (identity graph, 128 nodes):
its tcgen05 product equals the BF16-rounded operands multiplied exactly (FP32
accumulation, 1e-5 relative), and its bounded mbarrier wait, made to run out
by issuing no MMA, raises the error flag and returns with the context still
usable (Sec. 3.2 layer; the error path has no counterpart in the paper)."""
import numpy as np
import pytest
import torch

import paper_2606_19251_gb300 as P
import workloads as W

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def operands(seed):
    x = W.uniform_pm1(seed, 128 * 64).reshape(128, 64) * 3.0
    Wm = W.uniform_pm1(seed + 1, 64 * 64).reshape(64, 64) * 0.2
    b = W.uniform_pm1(seed + 2, 64) * 0.1
    return x, Wm, b


@pytest.mark.parametrize("seed", [1, 2])
def test_tensor_core_product(seed):
    x, Wm, b = operands(seed)
    y, h, flag = P.gcin_tc_selftest(x, Wm, b)
    assert flag == 0
    assert np.array_equal(h, bf16(x).astype(np.float32))
    ref = bf16(x) @ bf16(Wm) + np.asarray(b, dtype=np.float32).astype(np.float64)
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()


def test_wait_timeout_sets_flag_and_returns():
    x, Wm, b = operands(3)
    _, _, flag = P.gcin_tc_selftest(x, Wm, b, no_commit=True)
    assert flag == 1
    # the device is still usable afterwards
    y, _, flag = P.gcin_tc_selftest(x, Wm, b)
    assert flag == 0
    ref = bf16(x) @ bf16(Wm) + np.asarray(b, dtype=np.float32).astype(np.float64)
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()
    t = torch.ones(4, device="cuda") * 2
    assert float(t.sum()) == 8.0
