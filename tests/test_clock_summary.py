"""bench.py's summary of the nvidia-smi clock samples taken during the timed region: the median
SM clock under load, the maximum clock, and every throttle reason that was active in any sample
(a run that saw hw_slowdown or a thermal slowdown is rejected, sw_power_cap is kept and noted)."""
import bench

S = bench.ClockSampler.summarise


def test_median_max_and_reasons():
    lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active",
             "1995, 2070, Not Active, Not Active, Not Active, Active",
             "2032, 2070, Not Active, Not Active, Not Active, Not Active"]
    d = S(lines)
    assert d["sm_mhz"] == 2032.0 and d["sm_max_mhz"] == 2070.0 and d["samples"] == 3
    assert d["reasons"] == ["sw_power_cap"]


def test_every_reason_is_reported_once():
    lines = ["1500, 2070, Active, Not Active, Not Active, Not Active",
             "1400, 2070, Active, Active, Active, Not Active",
             "1450, 2070, Not Active, Not Active, Active, Active"]
    assert S(lines)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                                   "sw_thermal_slowdown"]


def test_unparsable_lines_are_skipped():
    lines = ["", "garbage", "[N/A], [N/A], Not Active, Not Active, Not Active, Not Active",
             "2070, [N/A], Active, Not Active, Not Active, Not Active",
             "2070, 2070, Not Active, Not Active, Not Active, Not Active"]
    d = S(lines)
    assert d["samples"] == 1 and d["sm_mhz"] == 2070.0 and d["reasons"] == []


def test_no_samples():
    d = S([])
    assert d["sm_mhz"] is None and d["sm_max_mhz"] is None and d["samples"] == 0
