"""bench.py's clock record on the CPU: a fake nvidia-smi on PATH prints the sampled CSV.

The bench samples SM clocks and throttle reasons during its timed region; a run that saw a
hardware or thermal slowdown is to be rejected, so the parser must report every reason that
was active in any sample, the median SM clock and the maximum clock.
"""

import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SAMPLES = [
    "0, 2070, 2070, 810.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1200.7, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    "0, [N/A], 2070, 1200.7, 0x0, Not Active, Not Active, Not Active, Not Active",
    "garbage line",
]


def _fake_smi(tmp_path, lines):
    exe = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{ln}'" for ln in lines)
    exe.write_text(f"#!/bin/sh\n{body}\nexec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_reasons_median_and_max(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, SAMPLES) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0)
    cs.start()
    for _ in range(100):  # wait for the reader thread to see every line
        if len(cs.lines) >= len(SAMPLES):
            break
        time.sleep(0.05)
    rec = cs.stop()
    assert rec["samples"] == 3  # the unparsable lines are skipped
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
