"""bench.py's host-side pieces without a GPU: the JSON configuration of the
workload and the bookkeeping that ties measured DRAM traffic to the kernel
sources it was measured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_measured_traffic_matches_the_current_kernel_sources():
    """The default roofline line reports ncu traffic only for the kernel
    sources it was taken on; this fails when those sources change until the
    launch list is taken again and recorded."""
    key = (bench.kernel_source_hash(), "fp32", 8192, "pair")
    assert key in bench.MEASURED_TRAFFIC, key
    t = bench.MEASURED_TRAFFIC[key]
    algorithmic = 72 * 8192 * 8192
    assert 0.95 * algorithmic < t < 1.05 * algorithmic


def test_workload_config_names_the_workload():
    class A:
        n, precision = 8192, "fp32"
    cfg = bench.workload_config(A)
    assert cfg["workload"].startswith("8192x8192 periodic D2Q9 spinodal decomposition")
    assert cfg["nx"] == cfg["ny"] == 8192 and "L2" in cfg["l2"]
