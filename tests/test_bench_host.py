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
    for key, (fname, names) in bench.TRAFFIC_KERNELS.items():
        if names is None:
            assert os.path.exists(os.path.join(csrc, fname))
        else:
            with open(os.path.join(csrc, fname)) as f:
                text = f.read()
            for name in names:
                body = bench._kernel_source(text, name)
                assert body.lstrip().startswith(("template", "__global__"))
                assert f"{name}(" in body and body.rstrip().endswith("}")
                assert body.count("{") == body.count("}")
        assert len(bench._kernel_sha(key)) == 16
    # different kernels hash differently
    assert bench._kernel_sha("k_apply") != bench._kernel_sha("k_resid")
    assert bench._kernel_sha("gnn_sweep") != bench._kernel_sha("k_resid")
    assert bench._kernel_sha("k_resid") != bench._kernel_sha("wf_post")


def test_chain_bytes_count_each_array_once():
    n, nnz, nnz_p, nc = 1000, 7000, 2000, 400
    mat = 4 * (n + 1) + 8 * nnz
    # separate residual pass: A, gathered u, b, r; Q^-1 pass: Q, gathered r, u in and out
    assert bench._chain_bytes("k_resid", True, n, nnz) == mat + 12 * n
    assert bench._chain_bytes("k_apply", True, n, nnz) == mat + 12 * n
    # FP64 outer residual: 12 B per entry, x and b in FP64, r in FP32
    assert bench._chain_bytes("k_outer_resid", True, n, nnz) == 4 * (n + 1) + 12 * nnz + 20 * n
    # pre chain (pseudo-inverse): A once, b and a_ii read, four vectors written
    assert bench._chain_bytes("wf_pre", True, n, nnz) == mat + 8 * n + 16 * n
    # post chain: A and P once, e, u, b, a_ii read, five vectors written
    assert bench._chain_bytes("wf_post", True, n, nnz, nnz_p, nc) == \
        mat + 4 * (n + 1) + 8 * nnz_p + 4 * nc + 12 * n + 20 * n
