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
    # warp instructions per cluster of the capture x clusters / 1 ms
    assert r["achieved"] == pytest.approx(bench.NB_INST["plain"] * 16765809 / 1e-3 / 1e9)


def test_reference_arm_line():
    """`bench.py --impl reference` prints one JSON line with the contract's keys and
    samples only non-empty sectors (the one-sector workload gives a rate > 0)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "clusters/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("c1: one sector") and "model" not in d["config"]
