"""Host logic of bench.py without a GPU: the clock sampler keeps the samples
of the marked region only and reports the throttle reasons it saw, read from
a stand-in for nvidia-smi that prints fixed query lines."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fake_smi(tmp_path, lines_before, lines_during):
    """A script named nvidia-smi that prints `lines_before` quickly, then
    `lines_during` every 20 ms until it is terminated."""
    script = tmp_path / "nvidia-smi"
    before = "\n".join("echo '%s'" % ln for ln in lines_before)
    during = "\n".join("echo '%s'; sleep 0.02" % ln for ln in lines_during)
    script.write_text("#!/bin/sh\n%s\nwhile true; do\n%s\ndone\n" % (before, during))
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_region_and_reasons(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    idle = "0, 345, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 1980, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, [idle], [busy]) + os.pathsep + os.environ["PATH"])
    clk = bench.ClockSampler(0)
    clk.start()
    time.sleep(0.05)  # lines printed before mark() are not part of the region
    clk.mark()
    time.sleep(0.2)
    out = clk.stop()
    assert out["samples"] >= 3
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))  # empty directory: no nvidia-smi
    clk = bench.ClockSampler(0)
    clk.start()
    clk.mark()
    out = clk.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_reported_only_for_the_captured_source(monkeypatch):
    """The ncu DRAM figure is attached to the roofline only while the stencil
    source hash recorded with it matches the current one."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    entry = rec["wilson_32x32x32x64_exp0.6"]["hop f16/f16-c12"]
    monkeypatch.setattr(bench, "source_hash", lambda: entry["source_hash"])
    assert bench.ncu_traffic("wilson_32x32x32x64_exp0.6", "hop f16/f16-c12") == entry["dram_bytes_per_launch_full"]
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("wilson_32x32x32x64_exp0.6", "hop f16/f16-c12") is None
    assert bench.ncu_traffic("no_such_workload", "hop f16/f16-c12") is None
