"""Host-side pieces of bench.py (no GPU): the F-engine work count, the FP32
peak, and the rule that a DRAM-traffic capture applies only to the source and
the shape it was taken on."""
import hashlib
import json
import os

import bench


def test_fengine_flop_count():
    # 2 taps M (filter) + 2.5 M log2 M (half of one complex M-point FFT)
    assert bench.fe_flops_per_spectrum(1024, 4) == 2 * 4 * 2048 + 2.5 * 2048 * 11
    assert bench.fe_flops_per_spectrum(16, 1) == 2 * 32 + 2.5 * 32 * 5


def test_fp32_peak():
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def test_traffic_applies_only_to_its_source_and_shape(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel")
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"source": "k.cu", "source_sha256": hashlib.sha256(b"kernel").hexdigest(),
             "dram_bytes": 1000, "units": 10, "shape": {"n_inputs": 192}}
    (prof / "traffic.json").write_text(json.dumps({"k": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k", 20, n_inputs=192) == 2000
    assert bench.kernel_traffic("k", 20, n_inputs=32) is None      # another shape
    assert bench.kernel_traffic("k", 20) == 2000                    # no shape asked
    src.write_text("kernel changed")
    assert bench.kernel_traffic("k", 20, n_inputs=192) is None      # the source moved on
    assert bench.kernel_traffic("missing", 20) is None


def test_xengine_metric_names_the_input_count():
    assert bench.xe_metric(192) == bench.METRIC
    assert "at 32 inputs" in bench.xe_metric(32) and "192" not in bench.xe_metric(32)
