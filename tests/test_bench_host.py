"""CPU checks of the benchmark's host logic: the nvidia-smi clock samples it
parses, the rule that sends a timed region to be taken again (a hardware or
thermal slowdown, or clocks held low with no reason given), and the
algorithmic byte counts its roofline divides by."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def _row(sm, mx=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_parse_clock_csv():
    lines = [_row(2070), _row(2055, cap="Active"), "garbage\n", _row("[N/A]"), _row(2070)]
    c = bench.parse_clock_csv(lines)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.parse_clock_csv(["", "x, y\n"]) is None


def test_clocks_rejected_rule():
    ok = bench.parse_clock_csv([_row(2070)] * 5)
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)                      # no sampler: nothing to judge
    capped = bench.parse_clock_csv([_row(1600, cap="Active")] * 5)
    assert not bench.clocks_rejected(capped)                    # power cap: kept and noted
    for kw in ("hw", "hwt", "swt"):
        bad = bench.parse_clock_csv([_row(2070)] * 4 + [_row(1500, **{kw: "Active"})])
        assert bench.clocks_rejected(bad), kw
    locked = bench.parse_clock_csv([_row(1200)] * 5)            # low clocks, no reason: a left-over lock
    assert bench.clocks_rejected(locked)


def test_algorithmic_bytes_of_the_pair_kernels():
    g = (1024, 1024, 1024, 1024, 16, 16)
    R, Qh, P = 2047, 2048 // 2 + 1, 2048
    y = 16 * 16 * R * Qh * 8
    assert bench.algorithmic_bytes("pair_cols_f32", g) == (16 + 16) * Qh * P * 8 + y == 4834457600
    assert bench.algorithmic_bytes("pair_rows_f32", g) == y + R * R * 12
