"""Host logic of bench.py that needs no GPU: the clock samples kept for a timed region (the
samples stamped inside it, else the one nearest to it) and the throttle reasons they carry;
the dense-round traffic reference, which holds only while the dense-round source is the one
the ncu capture was taken on."""
import datetime
import os

import bench


def _line(t, mhz, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ", ".join("Active" if nm in reasons else "Not Active" for nm in names)
    return f"{t.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, {mhz}, 2070, 900.0, 0x0, {flags}"


def test_clock_samples_inside_the_timed_region():
    t0 = datetime.datetime(2026, 12, 4, 2, 0, 0)
    ms = datetime.timedelta(milliseconds=1)
    c = bench.Clocks(0)
    c.lines = [_line(t0 + k * 50 * ms, mhz, rs) for k, (mhz, rs) in
               enumerate([(1500, ("hw_slowdown",)), (2070, ()), (2000, ("sw_power_cap",)), (2070, ()),
                          (1200, ("hw_thermal_slowdown",))])]
    c.t_start, c.t_end = t0 + 40 * ms, t0 + 160 * ms  # samples 1, 2, 3
    got = c.summary()
    assert got["samples"] == 3 and got["window"] == "timed region"
    assert got["sm_mhz"] == 2070 and got["sm_max_mhz"] == 2070
    assert got["reasons"] == ["sw_power_cap"]  # the reasons outside the region are not counted


def test_short_region_takes_the_nearest_sample():
    t0 = datetime.datetime(2026, 12, 4, 2, 0, 0)
    ms = datetime.timedelta(milliseconds=1)
    c = bench.Clocks(0)
    c.lines = [_line(t0, 1800, ("sw_power_cap",)), _line(t0 + 100 * ms, 2070)]
    c.t_start, c.t_end = t0 + 80 * ms, t0 + 90 * ms
    got = c.summary()
    assert got == {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": [], "samples": 1, "window": "nearest sample"}


def test_unparsable_time_stamps_keep_every_sample():
    c = bench.Clocks(0)
    c.lines = ["n/a, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "n/a, 1900, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active", "garbage"]
    got = c.summary()
    assert got["samples"] == 2 and got["reasons"] == ["sw_power_cap"]
    assert got["window"].startswith("whole sampling")


def test_dense_traffic_reference_follows_the_dense_section(tmp_path, monkeypatch):
    traffic, note = bench._dense_traffic(bench.DENSE_TRAFFIC["algorithmic_bytes"] * 2)
    if traffic is not None:  # the committed source is the captured one: scaled by the byte ratio
        assert abs(traffic - 2 * bench.DENSE_TRAFFIC["bytes"]) < 1e-3 * traffic
    # a changed dense-round section voids the reference
    path = os.path.join(bench.ROOT, "paper_0912_2555_gb300", "csrc", "map_kernels.cuh")
    text = open(path, "rb").read()
    fake = tmp_path / "paper_0912_2555_gb300" / "csrc"
    fake.mkdir(parents=True)
    marker = b"// ------------------------------------------------------------ dense round --"
    (fake / "map_kernels.cuh").write_bytes(text.replace(marker, marker + b"\n// changed", 1))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, note = bench._dense_traffic(1.0)
    assert traffic is None and "changed" in note


def test_clock_queries_are_matched_to_the_steps_they_may_stall():
    t0 = datetime.datetime(2026, 12, 4, 2, 0, 0)
    ms = datetime.timedelta(milliseconds=1)
    c = bench.Clocks(0)
    c.lines = [_line(t0 + k * 500 * ms, 2070) for k in range(4)] + ["garbage line"]
    stamps = c.stamps()
    assert stamps == [t0 + k * 500 * ms for k in range(4)]
    # steps of 30 ms: one holds a sample, one starts 20 ms after a sample, one has none near it
    wins = [(t0 + 480 * ms, t0 + 510 * ms), (t0 + 1020 * ms, t0 + 1050 * ms), (t0 + 1200 * ms, t0 + 1230 * ms)]
    assert bench.queries_per_window(stamps, wins, lead_ms=50) == [1, 1, 0]
    assert bench.queries_per_window(stamps, wins, lead_ms=10) == [1, 0, 0]


def test_doubling_bytes():
    # one outer iteration of 12 rounds (the dense round and 11 doubling passes): 20n + 11 * 24n
    assert bench.doubling_bytes(1000, [12]) == 20 * 1000 + 11 * 24 * 1000
    # two outer iterations, the second with the dense round alone (no value: no pass at all)
    assert bench.doubling_bytes(10, [3, 1]) == 20 * 10 + 2 * 24 * 10
    assert bench.doubling_bytes(10, []) == 0
