"""bench.py's reading of the nvidia-smi clock samples taken during the timed
region: the median SM clock and every throttle reason that was active."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clean_run():
    b = _bench()
    text = "\n".join(f"0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
                     for mhz in (2070, 2055, 2070, 1980, 2070))
    r = b.parse_clock_samples(text)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_and_junk_lines():
    b = _bench()
    text = "\n".join([
        "0, 1800, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",  # unparsable clock: skipped
        "garbage",
        "0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active",
        "",
    ])
    r = b.parse_clock_samples(text)
    assert r["samples"] == 2 and r["sm_mhz"] == 1650.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_no_samples():
    b = _bench()
    assert b.parse_clock_samples("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
