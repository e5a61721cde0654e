"""Host-side pieces of the benchmark, on the CPU: clock-record parsing, the
shared config object and the whole-job rate."""
import bench


def test_clock_summary_reports_median_max_and_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
        "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    c = bench.ClockSampler(0)
    c.proc, c.path = object(), str(path)
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_config_and_rate():
    cfg = bench.workload_config(6, world=2)
    assert cfg["cells"] == 3 ** 20 and cfg["tile_level"] == 6 and cfg["parallelism"] == "replicas"
    assert bench.job_value(cfg["cells"], 100, 5, 870.0, 2) == 2 * 3 ** 20 * 500 / 0.87
