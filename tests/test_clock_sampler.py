"""The bench's clock sampler on the CPU, against a stand-in for nvidia-smi that prints a
CSV line every 0.1 s (the query's nine fields)."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fake_smi(tmp_path, line: str) -> str:
    p = tmp_path / "nvidia-smi"
    p.write_text("#!/bin/sh\nwhile true; do echo '" + line + "'; sleep 0.1; done\n")
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


@pytest.fixture
def bench_mod():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_samples_inside_the_marked_region(tmp_path, monkeypatch, bench_mod):
    d = _fake_smi(tmp_path, "0, 2070, 2070, 812.5, 0x4, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    with bench_mod.ClockSampler(0) as clk:
        assert clk.lines, "sampling is live before the region starts"
        time.sleep(0.3)            # samples before the region are not counted
        n_before = len(clk.lines)
        clk.mark_start()
        time.sleep(0.45)
        clk.mark_end()
    s = clk.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert 3 <= s["samples"] <= 7
    assert s["samples"] < len(clk.lines) - n_before + 2


def test_short_region_still_has_a_sample(tmp_path, monkeypatch, bench_mod):
    d = _fake_smi(tmp_path, "0, 1980, 2070, 900.0, 0x0, Not Active, Active, Not Active, Not Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    with bench_mod.ClockSampler(0) as clk:
        clk.mark_start()
        time.sleep(0.01)
        clk.mark_end()
    s = clk.summary()
    assert s["samples"] >= 1
    assert s["sm_mhz"] == 1980.0
    assert s["reasons"] == ["hw_thermal_slowdown"]


def test_without_nvidia_smi(tmp_path, monkeypatch, bench_mod):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory
    with bench_mod.ClockSampler(0) as clk:
        clk.mark_start()
        clk.mark_end()
    assert clk.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
