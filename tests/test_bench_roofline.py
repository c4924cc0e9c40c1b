"""CPU checks of the arithmetic behind bench.py's `roofline` object: the dominant class is the one with the
most kernel time, achieved = its algorithmic flops / its summed kernel time, frac = achieved / peak of its
arithmetic, and the DRAM traffic is the ncu fraction of the class's algorithmic bytes times the algorithmic
bytes of its average launch."""
import pytest


def test_dominant_class_and_rates():
    import bench
    # (ms, launches, flops, bytes) per class, as lmvd_profile_read returns them
    prof = {"fft_x_inverse": (200.0, 10.0, 1.5e14, 9.0e10), "eval": (50.0, 5.0, 5e13, 1e10),
            "products": (20.0, 4.0, 1e12, 8e10)}
    r = bench.roofline_of(prof, 400.0, 0, (512, 513, 512))
    assert r["kernel"] == "fft_x_inverse" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1.5e14 / 0.2 / 1e12)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches"] == 10 and r["algorithmic_bytes_per_launch"] == pytest.approx(9.0e9)
    assert r["achieved_hbm_gbs"] == pytest.approx(9.0e10 / 0.2 / 1e9)
    assert r["share_of_step"] == pytest.approx(0.5)
    assert r["traffic"] == pytest.approx(bench.NCU_DRAM_FRACTION[(0, "fft_x_inverse", 768)] * 9.0e9)
    rd = bench.roofline_of(prof, 400.0, 1, (512, 513, 512))
    assert rd["peak"] == pytest.approx(152 * 128 * 2.07e9 / 10 / 1e12)
    assert rd["traffic"] == pytest.approx(bench.NCU_DRAM_FRACTION[(1, "fft_x_inverse", 768)] * 9.0e9)


def test_traffic_is_null_without_a_matching_capture():
    import bench
    prof = {"solve_mc": (100.0, 5.0, 1e13, 5e10)}
    assert bench.roofline_of(prof, 200.0, 0, (512, 513, 512))["traffic"] is None      # no capture of this class
    prof = {"fft_x_inverse": (100.0, 5.0, 1e13, 5e10)}
    assert bench.roofline_of(prof, 200.0, 0, (256, 257, 256))["traffic"] is None      # other transform length


def test_measured_rates_set_the_peaks():
    """With the probe's rates, the FP64 peak is 2 flop x the FP64 FMA rate and the double-float one the FP32
    FMA rate / 10 instructions per classic flop."""
    import bench
    prof = {"fft_x_inverse": (200.0, 10.0, 1.5e14, 9.0e10)}
    rates = {"fp64_fma": 6.0e11, "fp64_add": 5.0e11, "fp64_mul": 5.0e11, "fp32_fma": 4.0e13}
    r = bench.roofline_of(prof, 400.0, 0, (512, 513, 512), rates)
    assert r["peak"] == pytest.approx(1.2) and "measured" in r["peak_note"]
    rd = bench.roofline_of(prof, 400.0, 1, (512, 513, 512), rates)
    assert rd["peak"] == pytest.approx(4.0) and rd["frac"] == pytest.approx(rd["achieved"] / 4.0)


def test_class_table_rates():
    """Per-class table: ms and launches per step, algorithmic TFLOP/s and GB/s, fraction of the copy peak."""
    import bench
    prof = {"products": (20.0, 4.0, 1e12, 8e10), "idle": (0.0, 0.0, 0.0, 0.0)}
    t = bench.class_table(prof, 2)
    assert set(t) == {"products"}
    r = t["products"]
    assert r["ms_per_step"] == 10.0 and r["launches_per_step"] == 2.0
    assert r["tflops"] == pytest.approx(1e12 / 0.02 / 1e12)
    assert r["hbm_gbs"] == pytest.approx(8e10 / 0.02 / 1e9)
    assert r["hbm_frac"] == pytest.approx(r["hbm_gbs"] / bench.hbm_peak_gbs()[0])
