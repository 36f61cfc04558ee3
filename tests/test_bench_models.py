"""The benchmark's algorithmic FLOP models, per route (they set the roofline figures).

Route codes are those of lmep_frozen_stats: m = 2 factorised row, m = 0 finite series in the
product type, m = 1 finite series in FP64 (FP32 form), m >= 3 the Pade degree.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def stats(*rows):
    return np.array(rows, dtype=np.int64)


def test_factorised_row_flops():
    n = 13
    f32, f64 = bench.flops_model(n, stats([2, 0, 0]), True)
    assert (f32, f64) == (2 * n * n + 6 * n + 2 * n, 0.0)
    f32, f64 = bench.flops_model(n, stats([2, 0, 0]), False)
    assert (f32, f64) == (0.0, 2 * n * n + 6 * n + 2 * n)


def test_series_rows_split_by_precision():
    n = 9
    ser = (n - 2) * 2 * n * n + (n - 1) * n
    assert bench.flops_model(n, stats([0, 0, 0]), True) == (ser + 2 * n, 0.0)
    assert bench.flops_model(n, stats([1, 0, 0]), True) == (2 * n, ser)   # FP64 sums in the FP32 form
    assert bench.flops_model(n, stats([0, 0, 0]), False) == (0.0, ser + 2 * n)


def test_pade_row_flops():
    n = 13
    d = float(n)
    f32, f64 = bench.flops_model(n, stats([13, 0, 0]), True)
    assert f32 == 6 * 2 * d ** 3 + 2 * d * d + 2 * d
    assert f64 == (2.0 / 3.0) * d ** 3 + 2 * d * d
    f32, f64 = bench.flops_model(n, stats([13, 2, 1]), True)
    assert f64 == (8.0 / 3.0) * d ** 3 + 2 * d ** 3 + 1 * 2 * d * d


def test_adjoint_flops_by_route():
    n = 9
    assert bench.adj_flops(n, [2], [0]) == 6 * n * n + 14 * n
    assert bench.adj_flops(n, [13], [1]) == 2.0 * n ** 3 * 37 + 12.0 * n ** 3 + 4.0 * n
    assert bench.adj_flops(n, [2, 13], [0, 1]) == 6 * n * n + 14 * n + 2.0 * n ** 3 * 37 + 12.0 * n ** 3 + 4.0 * n


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    """A captured DRAM figure stays in the bench line only while the kernel's sources are those captured."""
    import bench
    for key, (nbytes, sha, names) in bench.TRAFFIC.items():
        assert nbytes > 0 and len(sha) == 16 and names
        assert bench.traffic_of(key) in (nbytes, None)
    monkeypatch.setitem(bench.TRAFFIC, "probe", (123, "0" * 16, ("lmep_frozen_set.cu",)))
    assert bench.traffic_of("probe") is None
    sha = bench.sources_sha(("lmep_frozen_set.cu",))
    monkeypatch.setitem(bench.TRAFFIC, "probe", (123, sha, ("lmep_frozen_set.cu",)))
    assert bench.traffic_of("probe") == 123
    assert bench.traffic_of("never_captured") is None
