"""The measured-throughput entry point (the denominators of the pass kernels' roofline):
positive, FP32 well above FP64 (this GPU's FP64 rate is a small fraction of its FP32
rate), each covariance evaluation slower than one FP64 operation, and an FP64 tensor-core
rate."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def test_measure_peaks():
    h = vg.Handle(0)
    try:
        p = vg.vecchia_measure_peaks(h)
    finally:
        h.close()
    assert 100.0 < p["fp64_gflops"] < 1e4
    assert p["fp32_gflops"] > 10.0 * p["fp64_gflops"]
    for k in ("exp_pairs_per_s", "matern_pairs_per_s"):
        assert 0.0 < p[k] < p["fp64_gflops"] * 1e9
    assert 10.0 < p["fp64_tensor_gflops"] < 1e5
