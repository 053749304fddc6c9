"""Host-side logic of the benchmark: the clock record keeps only the samples
taken inside the timed region and reports the throttle reasons seen there."""
import datetime
import time

import bench


def _line(sm, t, hw="Not Active", pcap="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return "0, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s, %s" % (sm, hw, pcap, ts)


def test_samples_outside_the_timed_region_are_dropped():
    t0 = time.time()
    c = bench.ClockSampler(0)
    lines = [_line(1000, t0 - 1.0, hw="Active")]  # before the region: ignored
    lines += [_line(2070 - k, t0 + 0.05 * (k + 1), pcap="Active" if k == 2 else "Not Active") for k in range(5)]
    lines += [_line(500, t0 + 5.0, hw="Active")]  # after the region: ignored
    c.out = "\n".join(lines)
    c.window = [t0, t0 + 0.3]
    s = c.summary()
    assert s["samples"] == 5
    assert s["sm_mhz"] == 2068
    assert s["reasons"] == ["sw_power_cap"]


def test_short_region_keeps_the_nearest_sample():
    t0 = time.time()
    c = bench.ClockSampler(0)
    c.out = "\n".join([_line(1900, t0), _line(2070, t0 + 0.2)])
    c.window = [t0 + 0.15, t0 + 0.16]
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070


def test_no_samples_reads_unavailable():
    c = bench.ClockSampler(0)
    c.out = ""
    assert c.summary()["reasons"] == ["unavailable"]
