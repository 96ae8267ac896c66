"""Pins of the oracle's FP64 Kalman tracklet fit (A5).

The paper (Sec. 1) names Kalman-filter tracklet construction in native
coordinates, time standing in for z, and gives no formulas.  The fit's model
(helix in (x, y), straight line in (arc length, zeta)) is pinned against:
  * central finite differences of the transport (Jacobian);
  * noise-free helices, which the seed and the filter must reproduce exactly;
  * the batch weighted least-squares solution with the same prior (Gauss-Newton,
    Jacobians by finite differences), which a Kalman filter equals up to second
    order in the deviations;
  * pull statistics on smeared helices."""
import math

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts

K = 0.00149896229
X = 85.0 + np.arange(152) * (160.0 / 151.0)


def _npads(r):
    return 66 + (144 * r + 151) // 302


def _pitch_cm(r):
    return (4000 + (4000 * r + 151) // 302) * 1e-4


def _truth_chain(qpt, phi0, eta, rows=range(152), sector=0, sy=0.0, st=0.0, rng=None):
    rr, pads, times, truth = [], [], [], []
    for r in rows:
        res = ts.truth_at(qpt, phi0, eta, 0.0, sector, r)
        if res is None:
            break
        y, tb, sp, tz = res
        if rng is not None:
            y += sy * rng.standard_normal()
            tb += st * rng.standard_normal()
        pad = y / _pitch_cm(r) + 0.5 * (_npads(r) - 1)
        if not (-0.5 <= pad < _npads(r) - 0.5):
            break
        rr.append(r); pads.append(pad); times.append(tb); truth.append(res)
    return np.array(rr, np.int32), np.array(pads, np.float32), np.array(times, np.float32), truth


# ---------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("seed", range(9))
def test_jacobian_matches_central_differences(seed):
    """Forward transports (one row, 5 cm, 20 cm) and backward ones (towards smaller
    x, as the inward track follow uses them)."""
    rng = np.random.default_rng(seed)
    for _ in range(50):
        p = np.array([rng.uniform(-30, 30), rng.uniform(-50, 50), rng.uniform(-0.8, 0.8),
                      rng.uniform(-1.2, 1.2), rng.uniform(-8, 8)])
        dx = [160.0 / 151.0, 5.0, 20.0, -160.0 / 151.0, -5.0, -20.0, -150.0, 7.0, -60.0][seed]
        res = orc.propagate(p, dx)
        if res is None:
            continue
        _, F = res
        h = np.array([1e-4, 1e-4, 1e-6, 1e-6, 1e-5])
        for j in range(5):
            e = np.zeros(5)
            e[j] = h[j]
            a, b = orc.propagate(p + e, dx), orc.propagate(p - e, dx)
            if a is None or b is None:
                continue
            num = (a[0] - b[0]) / (2 * h[j])
            assert np.allclose(F[:, j], num, rtol=1e-6, atol=1e-7), (j, F[:, j], num)


@pytest.mark.parametrize("seed", range(4))
def test_transport_back_and_forth_is_the_identity(seed):
    """The helix through a point is the same curve in both directions: transport by
    dx then by -dx returns the state, and the two Jacobians are inverses."""
    rng = np.random.default_rng(100 + seed)
    done = 0
    for _ in range(50):
        p = np.array([rng.uniform(-30, 30), rng.uniform(-50, 50), rng.uniform(-0.8, 0.8),
                      rng.uniform(-1.2, 1.2), rng.uniform(-8, 8)])
        dx = rng.uniform(-160.0, 160.0)
        a = orc.propagate(p, dx)
        if a is None:
            continue
        b = orc.propagate(a[0], -dx)
        if b is None:
            continue
        assert np.allclose(b[0], p, rtol=0, atol=1e-9 * (1 + abs(dx))), (p, b[0])
        assert np.allclose(b[1] @ a[1], np.eye(5), atol=1e-7)
        done += 1
    assert done > 20


def test_backward_transport_of_a_helix_reproduces_its_clusters():
    """From the truth at the outermost row, transport back to every row: (y, zeta)
    equal the generator's crossings (zeta relative to the outer row)."""
    rows, pads, times, truth = _truth_chain(-0.8, math.radians(9.0), 0.3)
    yl, tl, sl, tzl = truth[-1]
    p_out = np.array([yl, 0.0, sl, tzl, -0.8])
    for r, tr in zip(rows[::7], truth[::7]):
        res = orc.propagate(p_out, X[r] - X[rows[-1]])
        assert res is not None
        assert res[0][0] == pytest.approx(tr[0], abs=1e-9)
        assert res[0][1] == pytest.approx(0.516 * (tr[1] - tl), abs=1e-9)


def test_propagation_stops_at_sin_phi_limit():
    p = np.array([0.0, 0.0, 0.998, 0.1, -5.0])   # c = +0.0075: s grows
    assert orc.propagate(p, 1.0) is None
    p[4] = 5.0
    assert orc.propagate(p, 1.0) is not None


# ---------------------------------------------------------------- noise free
@pytest.mark.parametrize("qpt,eta", [(2.0, 0.3), (-1.5, 0.8), (0.4, 0.05), (-6.0, 0.5), (0.0, 0.6)])
def test_noise_free_helix_is_reproduced(qpt, eta):
    # aim so that the track is at the sector centre at radius 100 cm
    phi0 = math.radians(10.0) - math.asin(-K * qpt * 50.0)
    rows, pads, times, truth = _truth_chain(qpt, phi0, eta)
    L = len(rows)
    assert L >= 20
    p0, st = orc.seed_chain(rows, pads, times)
    assert st == 0
    y0, t0, s0, tz0 = truth[0]
    assert abs(p0[2] - s0) < 2e-6
    assert abs(p0[3] - tz0) < 2e-6
    assert abs(p0[4] - qpt) < 2e-4
    rec = orc.fit_chain(0, rows, pads, times)
    y, tl, sl, tzl = truth[-1]
    assert rec["status"] == 0 and rec["nhits"] == L and rec["ndf"] == 2 * L - 5
    assert rec["x"] == pytest.approx(X[rows[-1]], abs=1e-12)
    assert abs(rec["p"][0] - y) < 2e-5
    assert abs(rec["p"][1] - 0.516 * (tl - float(times[0]))) < 1e-4
    assert abs(rec["p"][2] - sl) < 1e-6
    assert abs(rec["p"][3] - tzl) < 1e-6
    assert abs(rec["p"][4] - qpt) < 2e-5
    assert rec["chi2"] < 1e-4
    # covariance is symmetric positive definite
    C = np.zeros((5, 5))
    C[np.tril_indices(5)] = rec["C"]
    C = C + np.tril(C, -1).T
    assert np.all(np.linalg.eigvalsh(C) > 0)


# ---------------------------------------------------------------- batch LSQ
def _transport(p0, rows):
    """state at every row of the chain by repeated transport from the first row"""
    out = [p0.copy()]
    p = p0.copy()
    for a, b in zip(rows[:-1], rows[1:]):
        r = orc.propagate(p, X[b] - X[a])
        assert r is not None
        p = r[0]
        out.append(p.copy())
    return np.array(out)


GAPPED_ROWS = [r for r in range(0, 75) if r not in (9, 10, 31, 47, 48, 49, 60)]


@pytest.mark.parametrize("rows_sel", ["consecutive", "gapped"])
@pytest.mark.parametrize("noise,tol,ctol", [(0.0, 1e-11, 1e-6), (2e-5, 2e-9, 5e-6), (2e-3, 2e-5, 5e-4)])
def test_kalman_equals_batch_least_squares(noise, tol, ctol, rows_sel):
    """The filter linearises at its running estimate, the batch solution at the
    final one: states agree to second order in the deviations (which scale with the
    noise), covariances to first order.  Float rounding of the inputs is the only
    noise in the first case.  The gapped chain (rows missing, as in tracks that the
    follower extended or joined) uses the same filter across the gaps."""
    rng = np.random.default_rng(4)
    sel = range(0, 60) if rows_sel == "consecutive" else GAPPED_ROWS
    rows, pads, times, truth = _truth_chain(1.3, math.radians(11.0), 0.4, rows=sel,
                                            sy=noise, st=2 * noise, rng=rng)
    L = len(rows)
    ym = (pads.astype(np.float64) - 0.5 * (np.array([_npads(r) for r in rows]) - 1)) * \
        np.array([_pitch_cm(r) for r in rows])
    zm = 0.516 * (times.astype(np.float64) - float(times[0]))
    pseed, _ = orc.seed_chain(rows, pads, times)
    C0inv = np.diag(1.0 / np.array([0.06 ** 2, 0.0516 ** 2, 0.01, 0.01, 0.01]))
    Winv = np.array([1.0 / 0.06 ** 2, 1.0 / 0.0516 ** 2])
    p = pseed.copy()
    h = np.array([1e-6, 1e-6, 1e-8, 1e-8, 1e-7])
    for _ in range(8):
        S = _transport(p, rows)
        J = np.zeros((L, 2, 5))
        for j in range(5):
            e = np.zeros(5)
            e[j] = h[j]
            J[:, :, j] = ((_transport(p + e, rows) - _transport(p - e, rows)) / (2 * h[j]))[:, :2]
        r = np.stack([ym - S[:, 0], zm - S[:, 1]], axis=1)
        A = C0inv.copy()
        g = -C0inv @ (p - pseed)
        for k in range(1, L):
            A += J[k].T @ np.diag(Winv) @ J[k]
            g += J[k].T @ (Winv * r[k])
        p = p + np.linalg.solve(A, g)
    S = _transport(p, rows)
    r = np.stack([ym - S[:, 0], zm - S[:, 1]], axis=1)
    objective = (p - pseed) @ C0inv @ (p - pseed) + sum((Winv * r[k] ** 2).sum() for k in range(1, L))
    P0 = np.linalg.inv(A)
    # transport of the batch covariance to the last row
    G = np.zeros((5, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = h[j]
        G[:, j] = (_transport(p + e, rows)[-1] - _transport(p - e, rows)[-1]) / (2 * h[j])
    PL = G @ P0 @ G.T
    rec = orc.fit_chain(0, rows, pads, times)
    scale = np.array([1.0, 1.0, 1e-2, 1e-2, 1e-1])
    assert np.all(np.abs(rec["p"] - S[-1]) < tol * scale), (rec["p"], S[-1])
    C = np.zeros((5, 5))
    C[np.tril_indices(5)] = rec["C"]
    C = C + np.tril(C, -1).T
    assert np.all(np.abs(C - PL) < ctol * np.sqrt(np.outer(np.diag(PL), np.diag(PL)))), (C, PL)
    # sum of normalised innovations = minimum of the batch objective (prior included)
    assert rec["chi2"] == pytest.approx(objective, rel=max(ctol, 1e-6), abs=1e-9)


# ---------------------------------------------------------------- pulls
@pytest.mark.slow
def test_pulls_on_smeared_helices():
    cfg = ts.c1(seed=77)
    cfg.n_tracks = 14000
    cfg.noise_frac = 0.0
    cfg.pt_min = 1.0
    cfg.phi_min, cfg.phi_max = math.radians(6.0), math.radians(14.0)
    f = ts.generate(cfg)
    lab = f.label
    order = np.argsort(lab, kind="stable")
    bounds = np.searchsorted(lab[order], np.arange(len(f.trk_qpt) + 1))
    pulls = []
    for t in range(len(f.trk_qpt)):
        idx = order[bounds[t]:bounds[t + 1]]
        if len(idx) < 100:
            continue
        idx = idx[np.argsort(f.row[idx], kind="stable")]
        rows = f.row[idx].astype(np.int32)
        if np.any(np.diff(rows) != 1):
            continue
        rec = orc.fit_chain(0, rows, f.pad[idx], f.time[idx])
        if rec["status"]:
            continue
        y, tb, sp, tz = ts.truth_at(f.trk_qpt[t], f.trk_phi0[t], f.trk_eta[t], 0.0, 0, int(rows[-1]))
        truth = np.array([y, 0.516 * (tb - float(f.time[idx[0]])), sp, tz, f.trk_qpt[t]])
        C = rec["C"]
        var = np.array([C[0], C[2], C[5], C[9], C[14]])
        pulls.append((rec["p"] - truth) / np.sqrt(var))
        if len(pulls) >= 10000:
            break
    pulls = np.array(pulls)
    assert len(pulls) >= 10000
    mu, rms = pulls.mean(axis=0), pulls.std(axis=0)
    assert np.all(np.abs(mu) < 0.05), mu
    assert np.all((rms > 0.95) & (rms < 1.05)), rms
