"""The bench's clock sampler against a stand-in nvidia-smi (CPU only).

The sampler runs one nvidia-smi process that samples on its own (-lms), so
that no Python thread competes with the timed region; it must take a sample
just before the region, one after it, and report throttle reasons and the
median SM clock from them."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE = """#!/bin/sh
# prints one sample line every 50 ms until terminated
i=0
while true; do
  echo "0, $((2000 + i)), 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, CAP"
  i=$((i + 10))
  sleep 0.05
done
"""


def _fake_smi(tmp_path, power_cap):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    # the last field is sw_power_cap: "Active" or "Not Active"
    f.write_text(FAKE.replace("CAP", power_cap))
    f.chmod(f.stat().st_mode | stat.S_IEXEC)
    return str(d)


def test_sampler_brackets_the_region(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, "Not Active") + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as clk:
        assert len(clk.samples) == 1  # the sample taken just before the region
        time.sleep(0.01)
    s = clk.summary()
    assert s["samples"] >= 2
    assert s["sm_max_mhz"] == 2070.0
    assert 2000.0 <= s["sm_mhz"] <= 2070.0
    assert s["reasons"] == []


def test_sampler_reports_power_cap(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, "Active") + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as clk:
        pass
    assert clk.summary()["reasons"] == ["sw_power_cap"]


def test_sampler_without_nvidia_smi(monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    with bench.ClockSampler(0) as clk:
        pass
    assert clk.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
