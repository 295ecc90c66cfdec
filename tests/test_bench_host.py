"""Host-side helpers of bench.py (no GPU): the per-kernel source hash that keys
the committed DRAM-traffic counters finds each measured kernel's definition."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_kernel_source_extraction():
    with open(os.path.join(ROOT, "paper_2606_19251_gb300", "csrc", "amg_solver.cu")) as f:
        text = f.read()
    for key, name in bench.TRAFFIC_KERNELS.items():
        body = bench._kernel_source(text, name)
        assert body.lstrip().startswith(("template", "__global__"))
        assert f"{name}(" in body and body.rstrip().endswith("}")
        assert body.count("{") == body.count("}")
        assert len(bench._kernel_sha(key)) == 16
    # the two kernels hash differently
    assert bench._kernel_sha("masweep") != bench._kernel_sha("residual")
