"""Pins of the oracle's track following and joining (oracle/follow.c), on the CPU.

  * exact recovery: noise-free, well-separated helices with rows taken out break
    into chains and free fragments; following must give one track per helix
    holding every cluster of it (the generator's truth, not the oracle, decides);
  * a join needs a consistent continuation: a straight line that leaves the
    extrapolation of another with a kink is not joined (but is with a one-cluster
    check);
  * invariants on a dense slice of the 2 ms frame (every chain ends up in exactly
    one track, rows strictly increase, pick-ups take only free clusters, record
    fields agree with the membership);
  * quality: clones fall several-fold at equal efficiency."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts


def _npads(r):
    return 66 + (144 * r + 151) // 302


def _pitch_cm(r):
    return (4000 + (4000 * r + 151) // 302) * 1e-4


def _helices(n_tracks, drop, seed=21):
    """Separated noise-free helices in sector 0 (as the chain-recovery test), without
    the clusters of the rows in `drop`."""
    rng = np.random.default_rng(seed)
    sec, row, pad, tim, lab = [], [], [], [], []
    for t in range(n_tracks):
        sh = 0.05 + 0.08 * t
        eta = float(np.arcsinh(sh))
        pt = rng.uniform(0.5, 3.0)
        q = 1 if rng.uniform() < 0.5 else -1
        phi0 = np.radians(3.0 + 14.0 * t / max(1, n_tracks - 1))
        for r in range(152):
            if r in drop:
                continue
            res = ts.truth_at(q / pt, phi0, eta, 0.0, 0, r)
            if res is None:
                continue
            y, tb, _, _ = res
            p = y / _pitch_cm(r) + 0.5 * (_npads(r) - 1)
            if not (-0.5 <= p < _npads(r) - 0.5) or not (0 <= tb < 500):
                continue
            sec.append(0); row.append(r); pad.append(p); tim.append(tb); lab.append(t)
    return (np.array(sec, np.uint16), np.array(row, np.uint16), np.array(pad, np.float32),
            np.array(tim, np.float32), np.array(lab))


@pytest.mark.parametrize("drop", [(70,), (6,), (145,), (40, 41), (30, 90)])
def test_broken_helices_are_followed_and_joined(drop):
    sec, row, pad, tim, lab = _helices(8, drop)
    chains = orc.track(sec, row, pad, tim)
    res = orc.track_follow(sec, row, pad, tim)
    ct = res["cluster_track"]
    full = tracked = 0
    for t in range(8):
        mine = np.where(lab == t)[0]
        if mine.size < 40 and (ct[mine] < 0).all():
            continue  # a short arc that leaves the sector early
        ids = np.unique(ct[mine])
        assert len(ids) == 1 and ids[0] >= 0, (t, ids)
        assert np.array_equal(np.where(ct == ids[0])[0], mine)
        tracked += 1
        full += mine.size >= 40
    assert full >= 6 and res["n_tracks"] == tracked
    # the chains alone did not get there: broken helices gave several tracks or free clusters
    assert chains["n_tracks"] > res["n_tracks"] or (chains["cluster_track"] < 0).sum() > (ct < 0).sum()
    # the refit of a joined track runs over all its clusters
    for k in range(res["n_tracks"]):
        rec = res["tracks"][k]
        rows_k = np.sort(row[ct == k].astype(int))
        assert rec["nhits"] == rows_k.size and rec["row_first"] == rows_k[0] and rec["row_last"] == rows_k[-1]
        assert rec["ndf"] == 2 * rows_k.size - 5 and rec["status"] == 0


def _polyline(rows, slope_before, slope_after, x_kink):
    """y and time along a straight line through (x_0, 0) that turns at x_kink."""
    X = 85.0 + np.asarray(rows) * (160.0 / 151.0)
    X0 = 85.0
    y = np.where(X <= x_kink, slope_before * (X - X0),
                 slope_before * (x_kink - X0) + slope_after * (X - x_kink))
    tb = 100.0 + 0.5 * (X - X0)
    pad = np.array([y[i] / _pitch_cm(r) + 0.5 * (_npads(r) - 1) for i, r in enumerate(rows)])
    return pad.astype(np.float32), tb.astype(np.float32)


def test_join_needs_a_consistent_continuation():
    """A: rows 0..69 of a straight line.  B: rows 72..151; its clusters of rows 72
    and 73 lie on A's line, after row 73 it turns (slope 0.10 -> 0.45).  B's chain
    starts at row 73 (row 72 has no link below), so A's follow picks up row 69 and
    row 72 and meets B's first cluster on its extrapolation; B's next clusters fail
    the gate, so there is no join unless a single cluster is checked."""
    X = 85.0 + np.arange(152) * (160.0 / 151.0)
    rows = np.concatenate([np.arange(0, 70), np.arange(72, 152)])
    row = rows.astype(np.uint16)
    sec = np.zeros(row.size, np.uint16)
    pad, tim = _polyline(rows, 0.10, 0.45, X[73])
    chains = orc.track(sec, row, pad, tim)
    assert chains["n_tracks"] == 2
    res = orc.track_follow(sec, row, pad, tim)
    assert res["n_tracks"] == 2 and res["stats"][2] == 0
    one = orc.track_follow(sec, row, pad, tim, fp=orc.follow_params(join_check=1))
    assert one["n_tracks"] == 1 and one["stats"][2] == 1
    # without the turn the default rule joins them into one track of every cluster
    pad2, tim2 = _polyline(rows, 0.10, 0.10, X[73])
    res2 = orc.track_follow(sec, row, pad2, tim2)
    assert res2["n_tracks"] == 1 and (res2["cluster_track"] == 0).all()


@pytest.fixture(scope="module")
def c2_slice():
    f = ts.generate(ts.c2())
    m = f.sector < 3
    return f, m


def test_invariants_dense_slice(c2_slice):
    f, m = c2_slice
    s, r, p, t = f.sector[m], f.row[m], f.pad[m], f.time[m]
    a = orc.track(s, r, p, t)
    b = orc.track_follow(s, r, p, t)
    cta, ctb = a["cluster_track"], b["cluster_track"]
    o2n = b["old_to_new"]
    assert b["n_chains"] == a["n_tracks"] and o2n.size == a["n_tracks"]
    # every chain lies in exactly one final track, and assigned clusters stay assigned
    assert np.all(ctb[cta >= 0] == o2n[cta[cta >= 0]])
    # pick-ups are clusters that no chain held
    picked = (cta < 0) & (ctb >= 0)
    assert picked.sum() == b["stats"][1]
    assert b["n_tracks"] == a["n_tracks"] - b["stats"][2]
    assert np.array_equal(np.sort(np.unique(o2n)), np.arange(b["n_tracks"]))
    # per track: one sector, strictly increasing rows, records agree
    order = np.lexsort((r, ctb))
    ct_sorted, r_sorted, s_sorted = ctb[order], r[order].astype(int), s[order].astype(int)
    sel = ct_sorted >= 0
    ct_sorted, r_sorted, s_sorted = ct_sorted[sel], r_sorted[sel], s_sorted[sel]
    same = ct_sorted[1:] == ct_sorted[:-1]
    assert np.all(r_sorted[1:][same] > r_sorted[:-1][same])
    assert np.all(s_sorted[1:][same] == s_sorted[:-1][same])
    nh = np.bincount(ctb[ctb >= 0], minlength=b["n_tracks"])
    tr = b["tracks"]
    assert np.array_equal(tr["nhits"], nh)
    first = np.full(b["n_tracks"], 10 ** 9)
    np.minimum.at(first, ctb[ctb >= 0], r[ctb >= 0].astype(np.int64))
    assert np.array_equal(tr["row_first"], first)
    assert np.all(r[tr["first_cluster"]] == tr["row_first"])
    assert np.all(ctb[tr["first_cluster"]] == np.arange(b["n_tracks"]))
    assert np.all(np.isfinite(tr["p"])) and np.all(b["margin"] > 0)


def test_following_cuts_clones_at_equal_efficiency(c2_slice):
    f, m = c2_slice
    s, r, p, t, lab = f.sector[m], f.row[m], f.pad[m], f.time[m], f.label[m]
    a = orc.track(s, r, p, t)
    b = orc.track_follow(s, r, p, t)
    ea = orc.evaluate(lab, s, a["cluster_track"], a["n_tracks"], f.trk_qpt.shape[0])
    eb = orc.evaluate(lab, s, b["cluster_track"], b["n_tracks"], f.trk_qpt.shape[0])
    assert eb["efficiency"] >= ea["efficiency"] - 5e-4
    assert eb["clone_rate"] < ea["clone_rate"] / 4
    assert eb["fake_rate"] < 3e-3


def test_empty_and_no_tracks():
    e = np.zeros(0)
    res = orc.track_follow(e.astype(np.uint16), e.astype(np.uint16), e.astype(np.float32), e.astype(np.float32))
    assert res["n_tracks"] == 0
    sec, row, pad, tim, _ = _helices(1, drop=set(range(5, 152, 6)))  # no chain of 10 survives
    res = orc.track_follow(sec, row, pad, tim)
    assert res["n_tracks"] == 0 and (res["cluster_track"] < 0).all()


# ---------------------------------------------------------------- cross-sector links
X = 85.0 + np.arange(152) * (160.0 / 151.0)
BETA = np.radians(20.0)


@pytest.mark.parametrize("seed", range(4))
def test_rotation_jacobian_matches_finite_differences(seed):
    """The rotation's Jacobian (new parameters at fixed x') against rotating a
    perturbed state exactly and transporting it back to the nominal x'."""
    rng = np.random.default_rng(300 + seed)
    done = 0
    for _ in range(40):
        x = rng.uniform(90.0, 240.0)
        p = np.array([rng.uniform(0.8, 1.0) * x * np.tan(np.radians(10.0)), rng.uniform(-20, 20),
                      rng.uniform(-0.5, 0.5), rng.uniform(-1.0, 1.0), rng.uniform(-3, 3)])
        beta = BETA if rng.uniform() < 0.5 else -BETA
        res = orc.rotate(p, x, beta)
        if res is None:
            continue
        q0, x0, J = res
        h = np.array([1e-5, 1e-5, 1e-7, 1e-7, 1e-6])
        num = np.zeros((5, 5))
        ok = True
        for j in range(5):
            cols = []
            for sgn in (1, -1):
                e = np.zeros(5)
                e[j] = sgn * h[j]
                r = orc.rotate(p + e, x, beta)
                back = orc.propagate(r[0], x0 - r[1]) if r is not None else None
                if back is None:
                    ok = False
                    break
                cols.append(back[0])
            if not ok:
                break
            num[:, j] = (cols[0] - cols[1]) / (2 * h[j])
        if not ok:
            continue
        assert np.allclose(J, num, rtol=1e-5, atol=1e-6), (J, num)
        done += 1
    assert done > 20


def test_rotation_then_transport_reproduces_the_neighbouring_sector():
    """A generator helix seen in sector 0 at row r, rotated into sector 1's frame and
    transported to a row there, equals the generator's own crossing in sector 1."""
    checked = 0
    for qpt, phi0, eta in ((1.0, 17.0, 0.3), (-0.7, 21.0, 0.5), (2.5, 19.0, 0.1), (-1.5, 15.0, 0.7)):
        phi0 = np.radians(phi0)
        for r in (20, 60, 100):
            a = ts.truth_at(qpt, phi0, eta, 0.0, 0, r)
            if a is None:
                continue
            y, tb, sp, tz = a
            res = orc.rotate(np.array([y, 0.0, sp, tz, qpt]), X[r], BETA)
            if res is None:
                continue
            q, xq, _ = res
            for r2 in range(152):
                if X[r2] < xq:
                    continue
                b = ts.truth_at(qpt, phi0, eta, 0.0, 1, r2)
                if b is None:
                    continue
                out = orc.propagate(q, X[r2] - xq)
                if out is None:
                    continue
                assert out[0][0] == pytest.approx(b[0], abs=1e-8)
                assert out[0][2] == pytest.approx(b[2], abs=1e-10)
                assert out[0][1] == pytest.approx(0.516 * (b[1] - tb), abs=1e-8)
                checked += 1
                break
    assert checked >= 6


def _crossing_helices(n_tracks, seed=5):
    """Noise-free helices of one collision that cross from sector 0 into sector 1
    (or back), clusters in both sectors wherever they fall on the pad plane."""
    rng = np.random.default_rng(seed)
    sec, row, pad, tim, lab = [], [], [], [], []
    for t in range(n_tracks):
        eta = 0.05 + 0.8 * t / n_tracks
        pt = rng.uniform(0.5, 2.0)
        q = 1 if t % 2 else -1
        # the position's azimuth at radius rho is phi0 -/+ asin(|c| rho / 2) for q = +/-1:
        # cross the sector boundary (20 deg) at a radius between 115 and 215 cm
        rho = rng.uniform(115.0, 215.0)
        d = np.arcsin(0.00149896229 / pt * rho / 2.0)
        phi0 = np.radians(20.0) + (d if q > 0 else -d)
        for s in (0, 1):
            for r in range(152):
                res = ts.truth_at(q / pt, phi0, eta, 0.0, s, r)
                if res is None:
                    continue
                y, tb, _, _ = res
                p = y / _pitch_cm(r) + 0.5 * (_npads(r) - 1)
                if not (-0.5 <= p < _npads(r) - 0.5) or not (0 <= tb < 500):
                    continue
                sec.append(s); row.append(r); pad.append(p); tim.append(tb); lab.append(t)
    return (np.array(sec, np.uint16), np.array(row, np.uint16), np.array(pad, np.float32),
            np.array(tim, np.float32), np.array(lab))


def _labels(ct, lab, nt):
    out = np.full(nt, -2)
    for k in range(nt):
        v, c = np.unique(lab[ct == k], return_counts=True)
        out[k] = v[np.argmax(c)]
    return out


def test_crossing_helices_are_linked_across_the_boundary():
    s, r, p, t, lab = _crossing_helices(10)
    res = orc.track_follow(s, r, p, t, fp=orc.follow_params(links=1))
    nt = res["n_tracks"]
    labs = _labels(res["cluster_track"], lab, nt)
    sec = res["tracks"]["sector"]
    nxt = res["next"]
    pairs = 0
    for L in np.unique(labs):
        ks = np.nonzero(labs == L)[0]
        if len(ks) != 2 or sec[ks[0]] == sec[ks[1]]:
            continue
        pairs += 1
        a, b = ks
        assert nxt[a] == b or nxt[b] == a, (L, a, b, nxt[a], nxt[b])
    linked = np.nonzero(nxt >= 0)[0]
    assert pairs >= 5 and linked.size == pairs
    assert np.all(labs[linked] == labs[nxt[linked]])
    # without links nothing is reported
    off = orc.track_follow(s, r, p, t)
    assert np.all(off["next"] == -1)


def test_links_on_a_dense_slice_are_pure(c2_slice):
    f, _ = c2_slice
    m = f.sector < 4
    s, r, p, t, lab = f.sector[m], f.row[m], f.pad[m], f.time[m], f.label[m]
    res = orc.track_follow(s, r, p, t, fp=orc.follow_params(links=1))
    nt = res["n_tracks"]
    nxt = res["next"]
    linked = np.nonzero(nxt >= 0)[0]
    sec = res["tracks"]["sector"].astype(int)
    # a link goes to the neighbouring sector of the same side; each track has one predecessor at most
    d = (sec[nxt[linked]] % 18 - sec[linked] % 18) % 18
    assert np.all((d == 1) | (d == 17)) and np.all(sec[nxt[linked]] // 18 == sec[linked] // 18)
    assert np.unique(nxt[linked]).size == linked.size
    assert np.all(res["tracks"]["status"][linked] == 0)
    labs = _labels(res["cluster_track"], lab, nt)
    pure = np.mean(labs[linked] == labs[nxt[linked]])
    assert linked.size > 500 and pure > 0.995
