"""Host logic of bench.py's clock sampler, on CPU with a fake nvidia-smi: the
summary keeps the samples inside the timed region (all of them when none fell
there), reads the throttle reasons of those samples only, and skips malformed
lines; the start of a short timed region is placed so that a sample of the
periodic sampler falls in its middle."""

import datetime
import threading
import time

import pytest

import bench


def _line(t, sm, mx, reasons=()):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if nm in reasons else "Not Active" for nm in names]
    return ", ".join([ts, "0", str(sm), str(mx), "700.0", "0x0"] + flags) + "\n"


def _sampler(tmp_path, lines, t0, t1):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(lines))
    s = bench.ClockSampler(0)
    s.path = str(p)
    s.t_begin, s.t_end = t0, t1
    return s


def test_summary_keeps_the_region(tmp_path):
    base = time.time()
    lines = [_line(base + 0.0, 1200, 2032, ("hw_slowdown",)),  # before the region
             "garbage line\n",
             _line(base + 1.0, 2032, 2032),
             _line(base + 2.0, 1980, 2032, ("sw_power_cap",)),
             _line(base + 3.0, 2010, 2032),
             _line(base + 9.0, 900, 2032, ("hw_thermal_slowdown",))]  # after it
    s = _sampler(tmp_path, lines, base + 0.5, base + 3.5)
    r = s.summary()
    assert r["samples"] == 3 and r["samples_in_region"] == 3
    assert r["sm_mhz"] == 2010 and r["sm_max_mhz"] == 2032
    assert r["reasons"] == ["sw_power_cap"]
    assert r["region_s"] == pytest.approx(3.0, abs=1e-3)
    # offsets of the samples within 2 s of the region, relative to its start
    assert r["sample_offsets_s"] == pytest.approx([-0.5, 0.5, 1.5, 2.5], abs=2e-3)


def test_summary_without_samples_in_region_uses_all(tmp_path):
    base = time.time()
    lines = [_line(base, 2000, 2032), _line(base + 1.0, 1900, 2032, ("sw_thermal_slowdown",))]
    s = _sampler(tmp_path, lines, base + 0.2, base + 0.4)
    r = s.summary()
    assert r["samples_in_region"] == 0 and r["samples"] == 2
    assert r["sm_mhz"] == 1950
    assert r["reasons"] == ["sw_thermal_slowdown"]


def test_summary_of_nothing(tmp_path):
    s = _sampler(tmp_path, [], time.time(), time.time() + 1)
    r = s.summary()
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == []


class _FakeSmi:
    """Writes one CSV line every `period` seconds to the file it is given as
    stdout, like `nvidia-smi -lms`, from its own thread."""

    def __init__(self, period):
        self.period = period
        self.times = []
        self._stop = threading.Event()

    def popen(self, cmd, stdout=None, stderr=None):
        f = stdout
        t_first = time.time() + 0.05

        def run():
            k = 0
            while not self._stop.is_set():
                t = t_first + k * self.period
                d = t - time.time()
                if d > 0 and self._stop.wait(d):
                    break
                self.times.append(t)
                f.write(_line(t, 2032, 2032))
                f.flush()
                k += 1

        th = threading.Thread(target=run, daemon=True)
        th.start()
        fake = self

        class P:
            def terminate(self_inner):
                fake._stop.set()

            def wait(self_inner, timeout=None):
                th.join(timeout)

            def kill(self_inner):
                fake._stop.set()

        return P()


def _region_offset(monkeypatch, steps):
    """Runs one timed region of `steps` fake steps under the sampler; returns
    the distance from the region's middle to the nearest sample, and the
    region's half length."""
    period, step_s, warm_steps = 0.25, 0.004, 3
    smi = _FakeSmi(period)
    monkeypatch.setattr(bench.subprocess, "Popen", smi.popen)

    def warm():
        time.sleep(step_s * warm_steps)

    def pad():
        time.sleep(step_s)

    with bench.ClockSampler(0, warm, steps=steps, warm_steps=warm_steps, pad=pad, period_s=period) as clk:
        t0 = time.time()
        time.sleep(step_s * 10)
        t1 = time.time()
    assert clk.t_begin <= t0
    mid = (t0 + t1) / 2
    return min(abs(t - mid) for t in smi.times), (t1 - t0) / 2


def test_short_region_is_centred_on_a_sample(monkeypatch):
    # three regions, so that a sampler placing them at random (a quarter of
    # the period is within the tolerance) passes by chance about once in 60
    for _ in range(3):
        off, half = _region_offset(monkeypatch, steps=10)
        assert off < half + 0.01
