"""bench.py's clock record on CPU: nvidia-smi lines parsed by ClockSampler.stop(), with only the
samples stamped inside the timed region counted (median SM clock, maximum, throttle reasons)."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(ts, sm, smax, active, hw="Not Active", hwt="Not Active", swt="Not Active",
          cap="Not Active"):
    stamp = ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, 0, {sm}, {smax}, 900.5, {active}, {hw}, {hwt}, {swt}, {cap}"


def _sampler(lines, t0, t1):
    import bench
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = list(lines)
    c.t0, c.t1 = t0, t1
    return c


def test_only_samples_inside_the_timed_region_count():
    base = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    ms = lambda k: base + datetime.timedelta(milliseconds=k)
    lines = [
        _line(ms(0), 1200, 2070, "0x1", hwt="Active"),            # before the region
        _line(ms(40), 2070, 2070, "0x0"),
        _line(ms(60), 2055, 2070, "0x4", cap="Active"),
        _line(ms(80), 2070, 2070, "0x0"),
        "garbled line",
        _line(ms(200), 900, 2070, "0x8", hw="Active"),            # after the region
    ]
    out = _sampler(lines, ms(30), ms(100)).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_throttle_reasons_inside_the_region_are_reported():
    base = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    ms = lambda k: base + datetime.timedelta(milliseconds=k)
    lines = [_line(ms(10), 1800, 2070, "0x20", swt="Active"),
             _line(ms(30), 1700, 2070, "0x48", hw="Active", hwt="Active")]
    out = _sampler(lines, ms(0), ms(50)).stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 1750.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_no_nvidia_smi():
    import bench
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
