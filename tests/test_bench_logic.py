"""Host-side rules of bench.py, without a GPU: the serving headline and
divergence point, the quantile helper, and the workload's name."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _pt(f, gbs, p99, kept):
    return {"offered_x_saturation": f, "GB/s": gbs, "p99_ms": p99, "kept_up": kept}


def test_serving_points_headline_divergence_and_peak():
    sweep = [_pt(0.1, 40, 0.1, True), _pt(0.5, 200, 0.4, True), _pt(1.0, 386, 4.9, True),
             _pt(1.1, 391, 12.0, False), _pt(1.25, 395, 21.0, False)]
    head, div, peak = bench.serving_points(sweep, bound_ms=5.0)
    assert head["offered_x_saturation"] == 1.0
    assert div["offered_x_saturation"] == 1.1
    assert peak["offered_x_saturation"] == 1.25
    head, _, _ = bench.serving_points(sweep, bound_ms=1.0)
    assert head["offered_x_saturation"] == 0.5


def test_serving_points_without_a_bounded_point_or_divergence():
    sweep = [_pt(0.5, 200, 9.0, True), _pt(1.0, 380, 7.0, True)]
    head, div, peak = bench.serving_points(sweep, bound_ms=5.0)
    assert head["p99_ms"] == 7.0  # lowest p99 when nothing is within the bound
    assert div is None
    assert peak["GB/s"] == 380


def test_quantile_and_workload_name():
    vals = [1.0, 2.0, 3.0, 4.0, 5.0]
    assert bench.quantile(vals, 0.0) == 1.0
    assert bench.quantile(vals, 1.0) == 5.0
    assert bench.quantile(vals, 0.5) == 3.0
    assert abs(bench.quantile(vals, 0.1) - 1.4) < 1e-12
    assert bench.quantile([], 0.5) is None
    assert "4096 MiB" in bench.workload_name(4 << 30) and "536870912 blocks" in bench.workload_name(4 << 30)
