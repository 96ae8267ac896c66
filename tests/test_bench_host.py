"""Host-side pieces of the benchmark: the oracle's sector-parallel timing leg and
the roofline helpers (no GPU)."""
import numpy as np
import pytest

import bench
import oracle
import tpcsynth as ts


def test_sector_parallel_oracle_covers_the_frame():
    oracle.build()
    f = ts.generate(ts.continuous(0.2, 91))
    v, cores, sample = bench.cpu_oracle_rate_parallel(f, cores=2)
    assert cores == 2 and v > 0
    assert f"({f.n} clusters)" in sample  # every cluster went through a sector job


def test_sector_parallel_oracle_skips_empty_sectors():
    oracle.build()
    f = ts.generate(ts.c1())  # sector 0 only
    assert int(np.asarray(f.sector).max()) == 0
    v, _, sample = bench.cpu_oracle_rate_parallel(f, cores=2)
    assert v > 0 and "as 1 sector jobs" in sample


def test_fit_roofline_arithmetic():
    r = bench.fit_fp32(1_000_000, 0.5, 2000.0, 152)
    # 200 flop x 1e6 clusters in 0.5 ms = 0.4 TFLOP/s; peak 152 x 128 x 2 x 2 GHz = 77.824 TFLOP/s
    assert r["achieved"] == pytest.approx(0.4)
    assert r["peak"] == pytest.approx(77.824)
    assert bench.fit_fp32(1, None, 2000.0, 152) is None


def test_issue_roofline_arithmetic():
    r = bench.neighbours_issue("plain", 16765809, 1.0, 2000.0, 152)
    if r is None:  # the neighbour kernel changed since its capture
        pytest.skip("capture stale")
    assert r["peak"] == pytest.approx(4 * 152 * 2.0)  # G warp instructions/s
    assert r["achieved"] == pytest.approx(539628699 / 1e-3 / 1e9)
