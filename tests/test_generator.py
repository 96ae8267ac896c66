"""Pins of the synthetic input generator (helix geometry, drift, workload sizes).

The generator is not part of the method; these tests make sure the inputs have the
shapes and distributions stated for the synthetic workloads."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import tpcsynth as ts

K = 0.00149896229


def _local_xy_numeric(c, pl, sig):
    """Integrate the unit direction (cos, sin)(pl + c s) from 0 to sig."""
    x = integrate.quad(lambda s: math.cos(pl + c * s), 0.0, sig, epsabs=1e-13, epsrel=1e-13)[0]
    y = integrate.quad(lambda s: math.sin(pl + c * s), 0.0, sig, epsabs=1e-13, epsrel=1e-13)[0]
    return x, y


def test_crossing_matches_numeric_helix_and_is_first_root():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(400):
        qpt = rng.uniform(-10.0, 10.0)
        c = -K * qpt
        pl = rng.uniform(-0.6, 0.6)
        xr = rng.uniform(85.0, 245.0)
        res = ts.crossing(c, pl, xr)
        if res is None:
            continue
        sig, y, sp = res
        # position by numerical integration of the direction field
        xn, yn = _local_xy_numeric(c, pl, sig)
        assert abs(xn - xr) < 1e-9
        assert abs(yn - y) < 1e-9
        assert abs(math.sin(pl + c * sig) - sp) < 1e-12
        # first root: sample the arc before sig, x must stay below xr
        ss = np.linspace(0.0, sig, 2001)[:-1]
        xs = np.array([_local_xy_numeric(c, pl, s)[0] for s in ss[::100]])
        assert np.all(xs < xr + 1e-9)
        # bisection on [0, sig] for the crossing (x is increasing there)
        lo, hi = 0.0, sig
        f = lambda s: (math.sin(pl + c * s) - math.sin(pl)) / c - xr if abs(c) > 1e-12 else s * math.cos(pl) - xr
        if f(lo) < 0 < f(hi) + 1e-12:
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if f(mid) < 0:
                    lo = mid
                else:
                    hi = mid
            assert abs(0.5 * (lo + hi) - sig) < 1e-9
        checked += 1
    assert checked > 120


def test_no_crossing_beyond_reach():
    # pT = 0.1 GeV: R = 66.7 cm.  Starting along local x the track reaches x = R at most;
    # starting along local y it reaches x = 2R (after half a turn).
    c = -K * 10.0
    R = 1.0 / abs(c)
    assert ts.crossing(c, 0.0, R + 1.0) is None
    assert ts.crossing(c, 0.0, R - 1.0) is not None
    assert ts.crossing(c, np.pi / 2, 2 * R - 1.0) is not None
    assert ts.crossing(c, np.pi / 2, 2 * R + 1.0) is None


def test_drift_time_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(100):
        qpt = rng.uniform(-3, 3)
        phi0 = math.radians(10.0) + rng.uniform(-0.05, 0.05)
        eta = rng.uniform(-0.9, 0.9)
        sector = 0 if eta >= 0 else 18
        row = int(rng.integers(0, 152))
        t0 = rng.uniform(0, 1000)
        res = ts.truth_at(qpt, phi0, eta, t0, sector, row)
        if res is None:
            continue
        y, tb, sp, tz = res
        sig = ts.crossing(-K * qpt, phi0 - math.radians(10.0), 85.0 + row * 160.0 / 151.0)[0]
        z = sig * math.sinh(eta)
        assert abs((250.0 - 0.516 * (tb - t0)) - abs(z)) < 1e-9
        assert tz == pytest.approx(-abs(math.sinh(eta)))


def test_output_sorted_and_in_range():
    f = ts.generate(ts.c1())
    key = f.sector.astype(np.int64) * 152 + f.row
    assert np.all(np.diff(key) >= 0)
    same = np.diff(key) == 0
    assert np.all(np.diff(f.time)[same] >= 0)
    assert np.all(f.sector == 0)
    npads = 66 + (144 * f.row.astype(np.int64) + 151) // 302
    assert np.all(f.pad >= -0.5) and np.all(f.pad < npads - 0.5)
    assert np.all(f.time >= 0) and np.all(f.time < 500)
    nsig = int((f.label >= 0).sum())
    assert (f.label < 0).sum() == int(math.floor(0.05 * nsig + 0.5))


def test_deterministic_and_thread_independent():
    a = ts.c1(seed=7)
    b = ts.c1(seed=7)
    b.n_threads = 1
    fa, fb = ts.generate(a), ts.generate(b)
    for k in ("sector", "row", "pad", "time", "label"):
        assert np.array_equal(getattr(fa, k), getattr(fb, k))


@pytest.mark.slow
def test_c2_size_and_pt_distribution():
    f = ts.generate(ts.c2())
    # about 7M clusters (+-15 %) for a 2 ms frame at 50 kHz
    assert 7e6 * 0.85 <= f.n <= 7e6 * 1.15
    assert 80 <= f.n_collisions <= 120
    pt = 1.0 / np.abs(f.trk_qpt)
    assert pt.min() >= 0.1
    ks = stats.kstest(pt - 0.1, stats.expon(scale=0.5).cdf)
    assert ks.pvalue > 1e-3
    eta = f.trk_eta
    assert eta.min() >= -0.9 and eta.max() <= 0.9


def test_batched_instances():
    """Batched workload: one sector id per instance, each instance sorted, counts
    spread over the log-uniform range, the rate rescaled per instance."""
    b = ts.batched(30, seed=11, n_min=2e3, n_max=2e5, ms_min=0.2, ms_max=3.0)
    f, off = b.frame, b.offsets
    assert off[0] == 0 and off[-1] == f.n and np.all(np.diff(off) > 0)
    for k in range(30):
        a, e = off[k], off[k + 1]
        assert np.all(f.sector[a:e] == k)
        r, t = f.row[a:e].astype(np.int64), f.time[a:e]
        assert np.all(np.diff(r) >= 0)
        same_row = np.diff(r) == 0
        assert np.all(np.diff(t)[same_row] >= 0)
    sz = np.diff(off)
    assert sz.max() / sz.min() > 10
    # expected counts follow the rescaled rate: the median lies inside the drawn range
    assert 2e3 / 3 < np.median(sz) < 2e5 * 3
    # labels of different instances never collide
    lab = f.label[f.label >= 0]
    inst = f.sector[f.label >= 0]
    for k in range(29):
        assert lab[inst == k].max(initial=-1) < lab[inst == k + 1].min(initial=2**31 - 1)
