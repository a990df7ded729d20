"""bench.py's child-process measurements (the batch_c5 sub-object of the default
line runs `bench.py --batch ...` in a child with a time limit): a child that
exits with an error, prints no JSON line or runs past its limit is reported
as unavailable instead of stopping the benchmark.  Host logic only."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_child_error_exit_is_reported():
    r = bench.extra_child(["--impl", "no-such-arm"], 120)
    assert set(r) == {"unavailable"} and "exit 2" in r["unavailable"]


def test_child_without_json_line_is_reported():
    r = bench.extra_child(["--help"], 120)
    assert r == {"unavailable": "--help: no JSON line"}


def test_child_past_its_limit_is_killed():
    # the oracle's reference arm runs far longer than a tenth of a second
    r = bench.extra_child(["--impl", "reference", "--steps", "1", "--warmup", "0"], 0.1)
    assert "did not finish within 0.1 s" in r["unavailable"]
