"""Host-side helpers of bench.py (no GPU): the per-kernel source hash that keys
the committed DRAM-traffic counters finds each measured kernel's definition,
and the compulsory-byte formulas of the finest-level kernels."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_kernel_source_extraction():
    csrc = os.path.join(ROOT, "paper_2606_19251_gb300", "csrc")
    for key, (fname, name) in bench.TRAFFIC_KERNELS.items():
        if name is None:
            assert os.path.exists(os.path.join(csrc, fname))
        else:
            with open(os.path.join(csrc, fname)) as f:
                body = bench._kernel_source(f.read(), name)
            assert body.lstrip().startswith(("template", "__global__"))
            assert f"{name}(" in body and body.rstrip().endswith("}")
            assert body.count("{") == body.count("}")
        assert len(bench._kernel_sha(key)) == 16
    # different kernels hash differently
    assert bench._kernel_sha("k_ma_sweep") != bench._kernel_sha("k_resid")
    assert bench._kernel_sha("k_resid") != bench._kernel_sha("wf_post")


def test_chain_bytes_count_each_array_once():
    n, nnz, nnz_p, nc = 1000, 7000, 2000, 400
    mat = 4 * (n + 1) + 8 * nnz
    # separate residual pass: A, gathered u, b, r
    assert bench._chain_bytes("k_resid", True, n, nnz) == mat + 12 * n
    # pre chain (pseudo-inverse): A once, b and a_ii read, four vectors written
    assert bench._chain_bytes("wf_pre", True, n, nnz) == mat + 8 * n + 16 * n
    # post chain: A and P once, e, u, b, a_ii read, five vectors written
    assert bench._chain_bytes("wf_post", True, n, nnz, nnz_p, nc) == \
        mat + 4 * (n + 1) + 8 * nnz_p + 4 * nc + 12 * n + 20 * n
