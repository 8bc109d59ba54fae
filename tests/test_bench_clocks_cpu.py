"""The clock record of bench.py on CPU, against a stand-in for nvidia-smi that
prints seeded samples: samples taken before the timed region starts are not
counted, the median SM clock and the maximum come from the rest, and a
throttle reason seen in any counted sample is reported."""

import os
import stat
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

# first line: an idle sample (printed before the timed region starts);
# then loaded samples, one with sw_power_cap active
_FAKE = """#!/bin/sh
echo "0, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"
sleep 0.4
echo "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
echo "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
echo "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"
exec sleep 30
"""


def _fake_smi(tmp_path, monkeypatch):
    path = tmp_path / "nvidia-smi"
    path.write_text(_FAKE)
    path.chmod(path.stat().st_mode | stat.S_IEXEC | stat.S_IXGRP | stat.S_IXOTH)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("TMPDIR", str(tmp_path))


def test_samples_before_the_timed_region_are_not_counted(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch)
    ck = bench.Clocks(0)
    ck.start()                      # returns once the first (idle) sample is out
    assert ck.skip == 1
    time.sleep(1.0)                 # the "timed region"
    rec = ck.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0  # median of 2070, 2055, 2070; the idle 345 is not in it
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_missing_nvidia_smi_gives_no_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.setenv("TMPDIR", str(tmp_path))
    ck = bench.Clocks(0)
    ck.start()
    assert ck.stop() is None
