"""Host-side helpers of the bench's concurrent schedule (no GPU)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_in_threads_keeps_order_and_reraises():
    import bench
    assert bench.in_threads([lambda: 1, lambda: 2, lambda: 3]) == [1, 2, 3]

    def bad():
        raise ValueError("from a worker")
    with pytest.raises(ValueError, match="from a worker"):
        bench.in_threads([lambda: 1, bad])


def test_sweep_timing_per_launch_figures():
    import bench

    class Fake:
        def counters(self):
            return dict(launches=0, smooth_ms=2.0, smooth_launches=4, smooth_sweeps=4, smooth_cells=1000)
    t = bench.sweep_timing(Fake(), "fp64", 2)
    assert t["launches"] == 4 and abs(t["avg_s"] - 0.5e-3) < 1e-15
    assert t["bytes"] == 112.0 * 1000 and t["fp64_inst"] == 12.0 * 1000
    t3 = bench.sweep_timing(Fake(), "mixed", 3)
    assert t3["bytes"] == 64.0 * 1000
