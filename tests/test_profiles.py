"""The committed ncu DRAM-traffic figure of the tensor-core bottom-node kernel
belongs to the current kernel source (bench.py reports it as the roofline's
traffic only while the source hash matches)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tc_heff_traffic_matches_kernel_source():
    sys.path.insert(0, ROOT)
    import bench
    t = bench.traffic_from_profile(os.path.join(ROOT, "paper_2011_10658_gb300", "csrc", "kernels_tc.cu"))
    assert t is not None and t > 0
