"""bench.py samples the GPU clocks and throttle reasons with nvidia-smi during
the timed region and reports the median SM clock, the maximum and every
reason seen active.  The parsing is checked here against a stand-in
nvidia-smi on PATH that prints fixed samples; nothing reads or changes a GPU."""
import os
import stat
import time

import bench

FAKE = """#!/bin/sh
echo "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "0, [N/A], 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "garbage line"
exec sleep 30
"""


def test_clock_samples_are_summarised(tmp_path, monkeypatch):
    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE)
    smi.chmod(smi.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.Clocks(0)
    c.start()
    assert c.p is not None
    for _ in range(100):  # until the stand-in has printed its samples
        time.sleep(0.05)
        c.f.flush()
        if os.path.getsize(c.f.name) > 0 and open(c.f.name).read().count("\n") >= 5:
            break
    got = c.stop()
    assert got["samples"] == 4  # the line without nine fields is dropped
    assert got["sm_mhz"] == 2070.0  # median of the three numeric samples
    assert got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]


def test_no_sampler_gives_no_clocks(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi at all
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
