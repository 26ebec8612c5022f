"""Host-side arithmetic of bench.py (no GPU): the algorithmic byte counts the
roofline divides by, and the parsing of the sampled clocks."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1710_09421_gb300 import workloads as W  # noqa: E402
from helpers import box  # noqa: E402


def test_lb_bytes_per_node():
    """57 populations read and written at the storage width, the link word
    and the 8-byte potential per fluid node; the link word per wall node."""
    solid = np.zeros((6, 5, 4), np.uint8)
    solid[0] = 1
    wl = box(4, 5, 6, solid=solid)
    nf, ns = 4 * 5 * 5, 4 * 5
    for s, per_fluid in ((8, 924), (4, 468), (2, 240)):
        assert bench.lb_algorithmic_bytes(wl, s) == nf * per_fluid + ns * 4


def test_bench_pore_lb_bytes():
    """The figure behind the LB roofline of the benchmark pore (230.4 MB)."""
    wl = W.config_pore_fp32()
    assert bench.lb_algorithmic_bytes(wl, 4) == 230355456


def test_multigrid_bytes_per_iteration_and_solve():
    wl = box(4, 4, 4)
    nf = 64
    assert bench.mg_bytes_per_iter(4) == 172 and bench.mg_bytes_per_solve(4) == 68
    assert bench.mg_algorithmic_bytes(wl, 5) == nf * (5 * 172 + 68)
    # the split solve's 1-byte link array: 3 B less per lattice pass
    assert bench.mg_bytes_per_iter(1) == 172 - 3 * 5.5 - 3 * 3 and bench.mg_bytes_per_solve(1) == 68 - 9
    assert bench.mg_algorithmic_bytes(wl, 5, link_bytes=1) == nf * (5 * 146.5 + 59)


def test_clock_summary():
    c = bench.ClockSampler(0)
    c.rows = [["2070", "2070", "900", "Not Active", "Not Active", "Not Active", "Active"],
              ["2055", "2070", "910", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["2070", "2070", "905", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    c.rows = [["1500", "2070", "900", "Active", "Not Active", "Not Active", "Not Active"]]
    assert c.summary()["reasons"] == ["hw_slowdown"]
    c.rows = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_translocation_progress_step():
    """Samples every 10 steps (the first at step 10): the centre of mass
    falls 2 units below the first sample between the samples at steps 40
    (8.2) and 50 (7.5): step 40 + 10 * 0.2 / 0.7."""
    assert abs(bench.progress_step([10, 9.5, 9.0, 8.2, 7.5], 10) - (40 + 10 * 0.2 / 0.7)) < 0.01
    assert bench.progress_step([10, 9.9, 9.8], 10) is None
