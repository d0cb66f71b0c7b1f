"""The bench's clock sampler against a stand-in nvidia-smi (host logic only, no GPU).

The bench samples SM clocks and throttle reasons with nvidia-smi during its timed region; a run that saw a
slowdown reason is rejected, so the sampler must be running before the region starts and must parse every line.
"""
import os
import stat
import sys
import time

import bench

FAKE = r'''#!{python}
import signal, sys, time
args = sys.argv[1:]
path = args[args.index("-f") + 1]
interval = int(args[args.index("-lms") + 1]) / 1000.0
time.sleep({delay})  # start-up latency of the real tool
signal.signal(signal.SIGTERM, lambda *_: sys.exit(0))
with open(path, "w") as f:
    i = 0
    while True:
        sm = 2070 if i % 3 else 1980
        cap = "Active" if i == 1 else "Not Active"
        f.write(f"0, {{sm}}, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, {{cap}}\n")
        f.flush()
        i += 1
        time.sleep(interval)
'''


def _install(tmp_path, monkeypatch, delay):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(python=sys.executable, delay=delay))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")


def test_sampler_waits_for_its_first_sample_and_parses_reasons(tmp_path, monkeypatch):
    _install(tmp_path, monkeypatch, delay=0.3)
    c = bench.ClockSampler(0)
    t0 = time.monotonic()
    c.start()
    # start() returned only once the (slow-starting) sampler had written a line
    assert time.monotonic() - t0 >= 0.25
    assert os.path.getsize(c.path) > 0
    time.sleep(0.3)  # a short timed region
    r = c.stop()
    assert r["samples"] >= 4  # 50 ms interval over about 0.3 s, plus the first sample
    assert r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] == 2070.0  # median: two of every three samples at the maximum
    assert r["reasons"] == ["sw_power_cap"]


def test_sampler_without_nvidia_smi_reports_it(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no nvidia-smi
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
