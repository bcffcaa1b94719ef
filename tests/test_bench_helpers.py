"""bench.py's arithmetic and its clock log parsing, on CPU: the roofline objects of the JSON line against
hand-computed values, and the nvidia-smi sampler's summary (median clock under load, throttle reasons)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_rooflines_are_algorithmic_bytes_over_stage_time():
    stage = {"ms_sync": 1.0, "ms_inflate": 9.0, "ms_translate": 2.0, "ms_crc": 0.5}
    C, D, W, hbm = 3_000_000_000, 4_000_000_000, 100_000_000, 6000.0
    r1, r4, r5 = bench.rooflines(stage, C, D, W, hbm, traffic_per_out_byte=15.0)
    # pass 1: compressed bytes read + 2 bytes of symbol per output byte, over sync + inflate
    assert r1["algorithmic_bytes"] == C + 2 * D
    assert r1["achieved"] == pytest.approx((C + 2 * D) / 10e-3 / 1e9, abs=0.01)
    assert r1["frac"] == pytest.approx(r1["achieved"] / hbm, abs=1e-5)
    assert r1["traffic"] == 15 * D and r1["bound"] == "hbm" and r1["unit"] == "GB/s"
    # translation: symbols read (2 B), bytes written (1 B) and the windows read
    assert r4["bytes"] == 3 * D + W
    assert r4["achieved"] == pytest.approx((3 * D + W) / 2e-3 / 1e9, abs=0.1)
    # CRC: the output read once
    assert r5["bytes"] == D and r5["achieved"] == pytest.approx(D / 0.5e-3 / 1e9, abs=0.1)
    # no capture for the configuration: no traffic figure
    assert bench.rooflines(stage, C, D, W, hbm)[0]["traffic"] is None


def test_a_determined_tail_lowers_the_algorithmic_bytes():
    stage = {"ms_sync": 1.0, "ms_inflate": 1.0, "ms_translate": 1.0, "ms_crc": 1.0}
    r1, r4, _ = bench.rooflines(stage, 10, 100, 0, 1000.0, determined=40)
    assert r1["algorithmic_bytes"] == 10 + 2 * 100 - 40    # tail symbols are 1 byte, not 2
    assert r4["bytes"] == 3 * 100 - 40


def test_whole_job_throughput_counts_every_rank():
    assert bench.whole_job_gbs(1 << 30, 4, 100.0) == pytest.approx(4 * (1 << 30) / 0.1 / 1e9)


def _clock_log(lines):
    c = bench.Clocks(0)                  # not entered: no sampler runs, the log is written here
    c.f.write("\n".join(lines) + "\n")
    return c.summary()


def test_clock_summary_median_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    s = _clock_log([ok, ok, capped, "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    hot = "0, 1500, 2070, 1400.0, 0x28, Not Active, Active, Active, Not Active"
    s = _clock_log([hot, hot, ok])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    s = _clock_log([])
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
