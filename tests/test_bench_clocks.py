"""bench.ClockSampler's reading of the nvidia-smi samples taken during the
timed region (no GPU: a finished child stands in for nvidia-smi and its CSV
is written by the test): the median SM clock under load, the maximum, and
which throttle reasons were ever active."""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _read(rows):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    c = bench.ClockSampler(0)
    c.proc, c.path = _Done(), path
    out = c.stop()
    assert not os.path.exists(path)
    return out


def _row(sm, active="0x0000000000000000", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), "2070", "900.00", active, hw, hwt, swt, cap]


def test_median_max_and_no_reasons():
    out = _read([_row(2070), _row(2055), _row(1980), _row(2070), _row(2070)])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 5


def test_reasons_collected_from_any_sample():
    out = _read([_row(2070), _row(1800, cap="Active"), _row(1500, hwt="Active"), _row(2000)])
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1900.0


def test_malformed_and_missing_samples():
    out = _read([["0", "[N/A]", "2070", "1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["garbage"], _row(2010)])
    assert out["sm_mhz"] == 2010.0 and out["samples"] == 2
    assert _read([])["reasons"] == ["no samples"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["unsampled"]
