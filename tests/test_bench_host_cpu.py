"""bench.py's host-side bookkeeping on CPU: the captured traffic file and the L2 report
built from it."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_file_has_the_headline_projection():
    t = bench.load_traffic()
    dram = t[f"{bench.WORKLOAD}:adjoint"]
    l2 = t[f"{bench.WORKLOAD}:adjoint:l2"]
    # L2 serves the staged boxes and the ray table, DRAM only what misses in L2
    assert 0 < dram < l2


def test_l2_report_arithmetic():
    t = {"w:adjoint:l2": 3.2e12}
    r = bench.l2_report(t, "w", "adjoint", ms=1000.0, l2_read_bps=16e12)
    assert r["achieved_GBps"] == pytest.approx(3200.0)
    assert r["peak_GBps"] == pytest.approx(16000.0)
    assert r["frac"] == pytest.approx(0.2)
    assert r["bytes_per_launch"] == 3.2e12
    assert bench.l2_report(t, "w", "forward", ms=1000.0, l2_read_bps=16e12) is None
    assert bench.l2_report(t, "w", "adjoint", ms=0.0, l2_read_bps=16e12) is None
    assert bench.l2_report({}, "w", "adjoint", ms=1.0, l2_read_bps=16e12) is None
