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
import os, sys, time
with open(os.environ["FAKE_SMI_ARGS"], "w") as f:
    f.write(" ".join(sys.argv[1:]))
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
    monkeypatch.setenv("FAKE_SMI_ARGS", str(tmp_path / "args.txt"))
    c = bench.Clocks("00000000:1B:00.0", window="warm-up and timed steps")
    c.start()
    time.sleep(0.3)
    rec = c.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2050.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["window"] == "warm-up and timed steps"
    # nvidia-smi was asked about the timed GPU by its bus id, and the record says which
    assert "--id=00000000:1B:00.0" in (tmp_path / "args.txt").read_text().split()
    assert rec["gpu_id"] == "00000000:1B:00.0"


class _Props:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def test_nvsmi_id_from_device_properties(monkeypatch):
    """nvidia-smi ignores CUDA_VISIBLE_DEVICES: the sampled GPU is named by its PCI bus id
    (domain:bus:device.function), else by its UUID, never by the CUDA ordinal."""
    import torch
    import bench
    props = {0: _Props(pci_domain_id=0, pci_bus_id=0x1B, pci_device_id=0, uuid="5a1e-77"),
             1: _Props(uuid="5a1e-78"),
             2: _Props(uuid="GPU-5a1e-79")}
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: props[i])
    assert bench.nvsmi_id(0) == "00000000:1B:00.0"
    assert bench.nvsmi_id(1) == "GPU-5a1e-78"
    assert bench.nvsmi_id(2) == "GPU-5a1e-79"


def test_clock_record_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))          # an empty directory: no nvidia-smi
    c = bench.Clocks(0)
    c.start()
    rec = c.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
