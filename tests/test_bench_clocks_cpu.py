"""bench.py's clock sampler on the CPU, against a stand-in for nvidia-smi that
prints readings in the same CSV form: it waits for the first reading, takes
the median SM clock and the maximum, and reports the throttle reasons seen
(sw_power_cap here).  No GPU."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FAKE = """#!/bin/sh
# index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
sleep 0.2
i=0
while [ $i -lt 400 ]; do
  echo "0, 2040, 2070, 1210.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
  echo "0, 2070, 2070, 1180.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
  i=$((i + 1))
  sleep 0.02
done
"""


def test_sampler_with_a_stand_in(tmp_path, monkeypatch):
    import bench
    tool = tmp_path / "nvidia-smi"
    tool.write_text(FAKE)
    tool.chmod(tool.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0)
    t0 = time.monotonic()
    c.wait_first()
    assert time.monotonic() - t0 < 3.0
    assert os.path.getsize(c.path) > 0          # a reading exists before the timed work
    time.sleep(0.1)
    info = c.stop()
    assert info["samples"] >= 2
    assert 2040 <= info["sm_mhz"] <= 2070 and info["sm_max_mhz"] == 2070
    assert info["reasons"] == ["sw_power_cap"]


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))  # nothing to run
    c = bench.Clocks(0)
    c.wait_first(0.5)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
