"""Host-side logic of bench.py that needs no GPU: the clock sampler, run
against a stand-in for nvidia-smi that prints the same CSV (timestamp first)
at the requested interval, line by line or in one burst at exit."""
import stat
import sys
import time

import bench

FAKE = r'''#!{python}
import datetime, signal, sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
buffered = {buffered}
out = []
def emit(line):
    if buffered:
        out.append(line)
    else:
        print(line, flush=True)
def bye(*_):
    if buffered:
        sys.stdout.write("\n".join(out) + "\n")
        sys.stdout.flush()
    sys.exit(0)
signal.signal(signal.SIGTERM, bye)
i = 0
while True:
    slow = "Active" if i == {slow_at} else "Not Active"
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    emit("%s, 0, %d, 2070, 500.0, 0x0, %s, Not Active, Not Active, Not Active" % (ts, 2070 - i, slow))
    i += 1
    time.sleep(ms / 1000.0)
'''


def _fake(tmp_path, slow_at=-1, buffered=False):
    p = tmp_path / "fake-smi"
    p.write_text(FAKE.replace("{python}", sys.executable).replace("{slow_at}", str(slow_at))
                 .replace("{buffered}", str(buffered)))
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(p)


def test_clock_sampler_window(tmp_path):
    s = bench.ClockSampler(0, interval_ms=20, exe=_fake(tmp_path))
    s.start()
    assert s.lines, "start() returns once the first sample arrived"
    time.sleep(0.1)
    s.begin()
    time.sleep(0.3)
    s.end()
    c = s.stop()
    # ~15 samples in 0.3 s at 20 ms, plus the first one after the region;
    # the samples before the region are left out
    assert c is not None and 8 <= c["samples"] <= 25
    assert c["sm_max_mhz"] == 2070 and c["sm_mhz"] < 2070 - 4 and c["reasons"] == []


def test_clock_sampler_places_burst_output_by_timestamp(tmp_path):
    # every line reaches the pipe at exit: only the embedded timestamps place
    # the samples inside the region
    s = bench.ClockSampler(0, interval_ms=20, exe=_fake(tmp_path, buffered=True))
    s.start(wait_s=0.1)
    time.sleep(0.2)
    s.begin()
    time.sleep(0.3)
    s.end()
    c = s.stop()
    assert c is not None and 8 <= c["samples"] <= 25
    assert c["sm_mhz"] < 2070 - 8     # the ~10 samples before the region are left out


def test_clock_sampler_reports_throttle_reasons(tmp_path):
    s = bench.ClockSampler(0, interval_ms=20, exe=_fake(tmp_path, slow_at=3))
    s.start()
    s.begin()
    time.sleep(0.25)
    s.end()
    c = s.stop()
    assert c is not None and "hw_slowdown" in c["reasons"]


def test_clock_sampler_without_nvidia_smi(tmp_path):
    s = bench.ClockSampler(0, interval_ms=20, exe=str(tmp_path / "missing"))
    s.start(wait_s=0.2)
    s.begin()
    s.end()
    assert s.stop() is None
