"""The roofline arithmetic of bench.py (no GPU): every roof's time is its
algorithmic work over its peak, the binding roof is the slowest, and the
reported fraction is that roof's time over the kernel's."""
import pytest

import bench

CELLS = 241_696_768          # the large level's valid cells
PEAKS = {"hbm_gbs": 6736.5}
ALU = {"fp32_tflops": 76.7, "fp64_tflops": 1.254}


def _check(r, kernel_ms, cells, peaks, alu):
    roofs = r["roofs"]
    for name, x in roofs.items():
        if name == "hbm":
            want = x["alg_per_zone"] * cells / (peaks["hbm_gbs"] * 1e9) * 1e3
        else:
            want = x["alg_per_zone"] * cells / (alu[f"{name}_tflops"] * 1e12) * 1e3
        assert x["roof_ms"] == pytest.approx(want, rel=1e-12)
        assert x["frac"] == pytest.approx(x["roof_ms"] / kernel_ms, rel=1e-12)
        assert x["achieved"] / x["peak"] == pytest.approx(x["frac"], rel=1e-12)
    bind = max(roofs, key=lambda k: roofs[k]["roof_ms"])
    assert r["bound"] == roofs[bind]["bound"]
    assert r["frac"] == roofs[bind]["frac"]
    assert r["kernel_ms"] == kernel_ms


def test_mixed_advance_is_bound_by_the_fp64_update():
    r = bench.roofline_of(118.0, CELLS, "mixed", PEAKS, "measured", ALU, "k_fused2")
    assert set(r["roofs"]) == {"hbm", "fp32", "fp64"}
    _check(r, 118.0, CELLS, PEAKS, ALU)
    assert r["bound"] == "fp64"
    # the FP64 update's 122 flop/zone at the measured rate: about 23.5 ms
    assert r["roofs"]["fp64"]["roof_ms"] == pytest.approx(23.5, abs=0.1)
    assert r["frac"] == pytest.approx(23.5 / 118.0, abs=1e-3)


def test_fp64_path_has_no_fp32_roof_and_hbm_can_bind():
    r = bench.roofline_of(7300.0, CELLS, "fp64", PEAKS, "measured", ALU, "k_fused<double>")
    assert set(r["roofs"]) == {"hbm", "fp64"}
    _check(r, 7300.0, CELLS, PEAKS, ALU)
    slow_hbm = {"hbm_gbs": 1.0}
    r2 = bench.roofline_of(7300.0, CELLS, "fp64", slow_hbm, "measured", ALU, "k_fused<double>")
    _check(r2, 7300.0, CELLS, slow_hbm, ALU)
    assert r2["bound"] == "hbm"
