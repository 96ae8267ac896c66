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
