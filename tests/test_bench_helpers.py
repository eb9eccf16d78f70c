"""Host-side pieces of the benchmark and of the golden fixture, on the CPU:
the oracle's per-sweep timing used beside the GPU measurements, and the
citations of the paper's printed values."""
import json
import os

import pytest


def test_oracle_sweep_timing_is_positive(orc):
    """The oracle's time per point and per z-line sweep (difference of one
    and two whole 32-sweep cycles) is positive and finite; the grid is large
    enough (131 k cells) that a cycle takes tens of milliseconds, well above
    timing noise."""
    import bench
    from paper_1511_07800_gb300 import inputs
    cfg = inputs.preset("les_channel", nx=64, ny=32, nz=64)
    for zline in (0, 1):
        us = bench.oracle_us_per_sweep(cfg, zline)
        assert 0.0 < us < 1e6, (zline, us)


def test_golden_values_carry_their_citations():
    """Every entry of the golden fixture names the section that prints it."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")
    with open(path) as f:
        g = json.load(f)
    entries = {k: v for k, v in g.items() if not k.startswith("_")}
    assert entries
    for k, v in entries.items():
        assert v.get("cite", "").startswith("Sec. "), k
        assert any(isinstance(x, float) for x in v.values()), k
