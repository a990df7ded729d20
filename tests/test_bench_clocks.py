"""bench.py's clock record (no GPU): nvidia-smi samples taken during the timed
region become the JSON line's "clocks" object (median SM clock, the maximum
clock, the throttle reasons seen active)."""
import bench


def _summary(lines):
    c = bench.Clocks(0)
    c.f.write("\n".join(lines) + "\n")
    c.f.flush()
    return c.summary()


def test_median_clock_and_active_reasons():
    s = _summary([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_thermal_slowdown_is_reported_and_unreadable_fields_skipped():
    s = _summary([
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active",
        "0, 1800, 2070, 1000.0, 0x0, Active, Not Active, Not Active, Not Active",
    ])
    assert s["sm_mhz"] == 1800.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_no_samples_gives_none():
    assert _summary([]) is None
