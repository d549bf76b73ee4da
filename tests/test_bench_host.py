"""Host logic of the benchmark that runs without a GPU: the summary of the
clock samples taken during the timed region (median and maximum SM clock,
the throttle reasons seen active), and the reference arm (the oracle timed
on the host cores), whose JSON line is checked against the contract."""
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


def _reference_arm(env_extra):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], cwd=root, env=env,
                         capture_output=True, text=True, timeout=600, check=True).stdout
    return [json.loads(s) for s in out.splitlines() if s.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the keys of the GPU arm's contract."""
    lines = _reference_arm({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    line = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.UNIT and line["value"] > 0 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_other_ranks_print_nothing():
    assert _reference_arm({"RANK": "1", "WORLD_SIZE": "2"}) == []
