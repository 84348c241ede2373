"""Host-side helpers of bench.py, without a GPU: the parsing of nvidia-smi
clock samples (throttle reasons, median clock), the peak lookup and the
lookup of the committed ncu traffic by kernel source hash."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""

    def kill(self):
        pass


def _clocks(text):
    c = bench.Clocks.__new__(bench.Clocks)
    c.p = _FakeSmi(text)
    return c.stop()


def test_clock_samples_and_reasons():
    text = "\n".join([
        "0, 2070, 2070, 800.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1900, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ])
    r = _clocks(text)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    r = _clocks("0, 1500, 2070, 900, 0x8, Active, Active, Not Active, Not Active")
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_no_sampler_gives_an_empty_record():
    c = bench.Clocks.__new__(bench.Clocks)
    c.p = None
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_peak_and_traffic_lookups():
    peak, kind = bench.measured_peak()
    assert peak > 0 and kind in ("measured", "fallback")
    for name in ("chung_lu_1m", "rmat_26"):
        traffic, h = bench.ncu_traffic(name)
        if h == bench.kernel_source_hash():
            assert traffic is not None and traffic > 1e8  # bytes of one pass of the dominant level
        else:
            assert traffic is None  # no summary, or one taken on other sources: not reported
    assert bench.ncu_traffic("no_such_workload") == (None, None)
