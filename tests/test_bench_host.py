"""Host logic of the benchmark that runs without a GPU: the summary of the
clock samples taken during the timed region (median and maximum SM clock,
the throttle reasons seen active)."""
import bench


def line(sm, smax, hw="Not Active", hw_thermal="Not Active", sw_thermal="Not Active",
         power_cap="Not Active"):
    return f"0, {sm}, {smax}, 812.40, 0x0000000000000000, {hw}, {hw_thermal}, {sw_thermal}, " \
           f"{power_cap}"


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler.summarize([line(1980, 2070), line(2070, 2070), line(2070, 2070),
                                      line(1965, 2070, power_cap="Active")])
    assert s["sm_mhz"] == 2025.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_names_every_slowdown_once():
    lines = [line(1500, 2070, hw="Active"), line(1400, 2070, hw="Active", sw_thermal="Active"),
             line(1300, 2070, hw_thermal="Active")]
    s = bench.ClockSampler.summarize(lines)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1400.0


def test_clock_summary_skips_unreadable_lines():
    lines = ["", "0, [N/A], [N/A], 0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2070, 2070", line(2070, 2070)]
    s = bench.ClockSampler.summarize(lines)
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0 and s["reasons"] == []
    assert bench.ClockSampler.summarize([])["reasons"] == ["no samples"]
