"""CPU check of bench.py's clock record: the nvidia-smi CSV lines sampled during the timed region are
reduced to the median SM clock under load, the maximum clock and power, and the throttle reasons seen
(a run with hw_slowdown or a thermal reason is rejected by the contract; sw_power_cap is kept and noted)."""


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_lines_reduce_to_median_max_and_reasons():
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = [
        "0, 2070, 2070, 612.30, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 640.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",     # unreadable sample
        "garbage",
    ]
    r = cs.stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["power_w_max"] == 1390.0
    assert r["reasons"] == ["sw_power_cap"]


def test_thermal_and_hw_reasons_are_reported():
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = ["0, 1500, 2070, 900, 0x48, Active, Not Active, Active, Not Active"]
    assert bench.ClockSampler.stop(cs)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_missing_nvidia_smi_is_reported():
    import bench
    cs = bench.ClockSampler(0)
    assert cs.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
