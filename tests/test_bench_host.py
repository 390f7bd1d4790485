"""Host logic of bench.py (no GPU): grouping of the per-class event times by kernel function and
the roofline fractions reported for each function."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "fp64_tflops": 1.0, "fp32_tflops": 80.0, "source": "test"}


def _cls(launches, total_ms, flops, nbytes):
    return {"launches": launches, "total_ms": total_ms, "flops_per_launch": flops, "bytes_per_launch": nbytes}


def test_axis_classes_of_one_kernel_are_summed():
    table = {"line_f64tc_x": _cls(10, 0.30, 1e8, 1e7), "line_f64tc_y": _cls(10, 0.25, 1e8, 1e7),
             "line_f64tc_z": _cls(10, 0.25, 1e8, 1e7), "hodge_block": _cls(10, 0.40, 2.5e7, 1.3e7)}
    kfr, dom = bench.kernel_rooflines(table, PEAKS)
    # the digit kernel is one function over three axis classes: 0.8 ms beats hodge_block's 0.4 ms
    assert dom["kernel"] == "mode_digit_kernel<7 digits>"
    assert dom["launches"] == 30
    assert sorted(dom["classes"]) == ["line_f64tc_x", "line_f64tc_y", "line_f64tc_z"]
    # 28 digit products x 1e8 flops per launch over 30 launches in 0.8 ms, against the BF16 peak
    assert dom["fracs"]["tensor"] == pytest.approx(28 * 1e8 * 30 / 0.8e-3 / 1e12 / 2000.0)
    assert dom["bound"] == "tensor"
    # 13.3 MB per launch in 26.7 us is a larger fraction of HBM: that roof binds first
    assert dom["binding"] == "hbm"
    assert sum(e["share"] for e in kfr) == pytest.approx(1.0)
    roof = bench.roofline_line(dom, PEAKS)
    assert roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])


def test_rated_roof_and_binding_roof():
    # a curl: 5 flop and 24 B per entry, 1e6 entries, 10 us -> 0.5 TFLOP/s (0.5 of FP64), 2.4 TB/s (0.4 of HBM)
    table = {"curl_primal": _cls(1, 0.010, 5e6, 24e6), "curl_dual": _cls(1, 0.010, 5e6, 24e6)}
    kfr, dom = bench.kernel_rooflines(table, PEAKS)
    assert dom["kernel"] == "curl_plane_kernel<double>" and dom["launches"] == 2
    assert dom["fracs"]["alu"] == pytest.approx(0.5)
    assert dom["fracs"]["hbm"] == pytest.approx(0.4)
    assert dom["bound"] == "hbm" and dom["frac"] == pytest.approx(0.4)   # rated against HBM
    assert dom["binding"] == "alu"                                       # the FP64 pipe binds first
    roof = bench.roofline_line(dom, PEAKS)
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["frac"] == pytest.approx(0.4)
    # an FP64 line kernel is rated against the FP64 pipe
    table = {"solve_y": _cls(1, 0.010, 7.5e6, 13.4e6)}
    _, dom = bench.kernel_rooflines(table, PEAKS)
    assert dom["bound"] == "alu" and dom["frac"] == pytest.approx(0.75)
    assert bench.roofline_line(dom, PEAKS)["unit"] == "TFLOP/s"


def test_peaks_fall_back_when_the_measured_file_is_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.load_peaks()
    assert p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0 and p["source"] == "of fallback"
    assert p["fp64_tflops"] == pytest.approx(1.2586, rel=1e-3)
