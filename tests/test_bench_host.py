"""Host-side logic of bench.py (no GPU): clock-sample parsing and the roofline of the top class."""
import bench


def test_clock_samples_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.parse_clock_samples(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3


def test_roofline_takes_the_class_with_the_largest_time():
    peaks = {"hbm_gbs": 6686.5, "bf16_tflops": 1921.8, "bf16_tflops_sustained": 1749.8}
    # ms, launches, flops, bytes per class
    prof = {"gemm": (100.0, 10, 2e12, 1e9), "permute": (300.0, 20, 0.0, 1.5e12), "tc_gemm": (50.0, 5, 9e13, 1e9)}
    r = bench._roofline(prof, "tf32x3", peaks, "measured")
    assert r["kernel"] == "permute" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 1.5e12 / 0.3 / 1e9) < 1e-6 and abs(r["frac"] - r["achieved"] / 6686.5) < 1e-12
    prof["tc_gemm"] = (400.0, 5, 9e14, 1e9)
    r = bench._roofline(prof, "tf32x3", peaks, "measured")
    assert r["kernel"] == "tc_gemm" and r["bound"] == "tensor" and abs(r["peak"] - 1749.8 / 2) < 1e-9
    prof["gemm_f64"] = (900.0, 7, 1e12, 1e9)
    r = bench._roofline(prof, "fp64", peaks, "measured")
    assert r["kernel"] == "gemm_f64" and r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS


def test_kept_per_pair_counts_values_above_the_cutoff():
    import numpy as np
    sp = np.array([[1.0, 0.5, 1e-7, 0.0], [2.0, 1e-5, 2.1e-6, 1e-9]])
    k = bench.kept_per_pair(sp, 3, 1e-6)
    assert k["min"] == 2 and k["max"] == 3 and k["chi"] == 3 and k["pairs"] == 2
