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


def test_class_table_and_roofline_inputs():
    """bench.py's per-class table from synthetic kernel timings: shares of the
    step, rates against each class's own peak and the tensor peak."""
    sys.path.insert(0, ROOT)
    import bench
    kt = {k: {"ms": 0.0, "launches": 0, "flops_alg": 0.0, "flops_exec": 0.0, "bytes_alg": 0.0}
          for k in bench.ALL_CLASSES}
    kt["tc_heff"].update(ms=300.0, launches=900, flops_alg=2.0e12)
    kt["heff_simt_upper"].update(ms=180.0, launches=870, flops_alg=4.5e11)
    kt["move_ops"].update(ms=200.0, launches=260, flops_alg=1.0e11)
    kt["lanczos"].update(ms=900.0)
    peaks = {"bf16": 1715.0, "tf32": 1060.0, "fp64": 1.1, "fp32_simt": 70.0}
    rows = bench.class_table(kt, 1340.0, peaks, "tf32x3")
    assert abs(rows["tc_heff"]["tflops_alg"] - 2.0e12 / 0.3 / 1e12) < 1e-9
    assert rows["tc_heff"]["tensor_peak"]["dtype"] == "tf32"
    assert abs(rows["lanczos_vectors"]["ms"] - (900.0 - 480.0)) < 1e-9
    assert abs(rows["move_ops"]["share_of_step"] - 200.0 / 1340.0) < 1e-12
