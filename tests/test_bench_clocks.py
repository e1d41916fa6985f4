"""The bench's clock record (no GPU): the sampler parses nvidia-smi's CSV lines into the
median SM clock, the maximum clock and the active slowdown reasons, names its window,
and reports nvidia-smi's absence instead of failing.  A stand-in nvidia-smi script on
PATH prints fixed samples."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = """#!{py}
import sys, time
rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2050, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
for r in rows:
    print(r, flush=True)
    time.sleep(0.02)
time.sleep(60)
"""


def test_clock_record_from_samples(tmp_path, monkeypatch):
    import bench
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(py=sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0, window="warm-up and timed steps")
    c.start()
    time.sleep(0.3)
    rec = c.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2050.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["window"] == "warm-up and timed steps"


def test_clock_record_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))          # an empty directory: no nvidia-smi
    c = bench.Clocks(0)
    c.start()
    rec = c.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
