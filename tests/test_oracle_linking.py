"""Pins of the oracle's integer linking (A1 neighbour finding, A2 cleaning, A3
start hits, A4 chains) against hand-worked values, brute force and invariants.
The seeding rule follows the CA tracker the paper builds on (Sec. 1: seeding in
native coordinates, time in place of z)."""
import os

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "a1_worked_example.txt")


# ---------------------------------------------------------------- geometry
def test_geometry_tables():
    x, npads, pitch = orc.geometry()
    assert x[0] == 85.0 and abs(x[151] - 245.0) < 1e-12
    assert np.allclose(np.diff(x), 160.0 / 151.0)
    assert npads[0] == 66 and npads[151] == 138
    assert pitch[0] == 4000 and pitch[151] == 6000
    assert np.all(np.diff(npads) >= 0) and np.all(np.diff(pitch) >= 0)
    # the pad plane fits inside the 20-degree sector at every row
    assert np.all(npads * pitch * 1e-4 < 2.0 * x * np.tan(np.radians(10.0)))
    # round-half-up reading at an exact half: 72*r/151 never hits .5 exactly, but
    # the integer formula must agree with the real-valued rounding everywhere
    r = np.arange(152)
    assert np.array_equal(npads, 66 + np.floor(72.0 * r / 151.0 + 0.5).astype(int))
    assert np.array_equal(pitch, 4000 + np.floor(2000.0 * r / 151.0 + 0.5).astype(int))


# ---------------------------------------------------------------- quantisation
def test_quantisation_closed_forms():
    rows = np.array([0, 0, 0, 0, 151, 151], np.uint16)
    pads = np.array([32.5, 1.0 / 128, 3.0 / 128, -5.0 / 128, 68.5, 0.0], np.float32)
    times = np.array([0.5 / 64, 1.5 / 64, 2.5 / 64, 100.0, 7.0, 1e4], np.float32)
    pq, tq, yq, zq = orc.quantize(rows, pads, times)
    # round half to even: 0.5 -> 0, 1.5 -> 2, 2.5 -> 2, -2.5 -> -2
    assert list(pq[:4]) == [2080, 0, 2, -2]
    assert list(tq[:3]) == [0, 2, 2]
    assert yq[0] == 0                      # pad centre of row 0: (66-1)/2 = 32.5
    assert yq[4] == 0                      # pad centre of row 151: (138-1)/2 = 68.5
    assert yq[5] == (0 - 32 * 137) * 6000
    assert zq[3] == 6400 * 5160 and zq[5] == 640000 * 5160


# ---------------------------------------------------------------- golden example
def _read_golden():
    cases, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = cases.setdefault(tok[1], {"cl": [], "expect": []})
        elif tok[0] == "expect":
            cur["expect"].append(tok[1:])
        else:
            cur["cl"].append((tok[0], int(tok[1]), int(tok[2]), float(tok[3]), float(tok[4])))
    return cases


@pytest.mark.parametrize("name", ["full", "tie"])
def test_golden_worked_example(name):
    case = _read_golden()[name]
    ids = [c[0] for c in case["cl"]]
    sec = np.array([c[1] for c in case["cl"]], np.uint16)
    row = np.array([c[2] for c in case["cl"]], np.uint16)
    pad = np.array([c[3] for c in case["cl"]], np.float32)
    tim = np.array([c[4] for c in case["cl"]], np.float32)
    order = orc.sort_order(sec, row, pad, tim)
    d, u, _ = orc.neighbours_sorted(sec[order], row[order], pad[order], tim[order])
    bd, bu = orc.bruteforce_neighbours(sec, row, pad, tim)
    name_of = lambda ci: "-" if ci < 0 else ids[ci]
    for cid, ed, eu in case["expect"]:
        ci = ids.index(cid)
        p = int(np.where(order == ci)[0][0])
        got_d = name_of(order[d[p]] if d[p] >= 0 else -1)
        got_u = name_of(order[u[p]] if u[p] >= 0 else -1)
        assert (got_d, got_u) == (ed, eu)
        assert (name_of(bd[ci]), name_of(bu[ci])) == (ed, eu)


# ---------------------------------------------------------------- brute force
def _random_tiny(rng, n_rows, n_per_row, dense=True, ties=False):
    rows, pads, times, secs = [], [], [], []
    r0 = int(rng.integers(1, 140))
    for s in range(int(rng.integers(1, 3))):
        for r in range(r0, r0 + n_rows):
            m = int(rng.integers(0, n_per_row + 1))
            npads = 66 + (144 * r + 151) // 302
            for _ in range(m):
                if dense:
                    pads.append(rng.uniform(20, 26))
                    times.append(rng.uniform(100, 115))
                else:
                    pads.append(rng.uniform(-0.5, npads - 0.5))
                    times.append(rng.uniform(0, 400))
                rows.append(r)
                secs.append(s)
    n = len(rows)
    pads = np.array(pads, np.float32)
    times = np.array(times, np.float32)
    if ties and n > 4:
        # snap to a coarse grid so equal costs and equal (time, pad) keys occur
        pads = (np.round(pads * 4) / 4).astype(np.float32)
        times = (np.round(times * 2) / 2).astype(np.float32)
    perm = rng.permutation(n)
    return (np.array(secs, np.uint16)[perm], np.array(rows, np.uint16)[perm], pads[perm], times[perm])


@pytest.mark.parametrize("seed", range(40))
def test_neighbours_match_bruteforce(seed):
    rng = np.random.default_rng(1000 + seed)
    sec, row, pad, tim = _random_tiny(rng, n_rows=int(rng.integers(3, 6)), n_per_row=int(rng.integers(3, 14)),
                                      dense=seed % 3 != 2, ties=seed % 2 == 1)
    if sec.shape[0] == 0:
        return
    order = orc.sort_order(sec, row, pad, tim)
    d, u, cost = orc.neighbours_sorted(sec[order], row[order], pad[order], tim[order])
    bd, bu = orc.bruteforce_neighbours(sec, row, pad, tim)
    # map oracle (sorted positions) to caller indices
    od = np.where(d >= 0, order[np.maximum(d, 0)], -1)
    ou = np.where(u >= 0, order[np.maximum(u, 0)], -1)
    assert np.array_equal(od, bd[order])
    assert np.array_equal(ou, bu[order])


def test_bruteforce_notices_a_dropped_term():
    """A neighbour rule without the time term would pick a different pair here;
    the oracle must not (guards against a dropped d2z term)."""
    sec = np.zeros(4, np.uint16)
    row = np.array([0, 1, 2, 2], np.uint16)
    pad = np.array([30.0, 30.0, 30.0, 30.05], np.float32)
    tim = np.array([100.0, 101.0, 105.0, 102.0], np.float32)
    order = orc.sort_order(sec, row, pad, tim)
    d, u, _ = orc.neighbours_sorted(sec[order], row[order], pad[order], tim[order])
    p = int(np.where(order == 1)[0][0])
    assert order[u[p]] == 3   # straight in time, 0.05 pad off in y


# ---------------------------------------------------------------- invariants
def _check_invariants(f, res, n_min=10):
    n = f.n
    order = res["order"]
    srow = f.row[order].astype(np.int64)
    ssec = f.sector[order]
    mup, mdown = res["mup"], res["mdown"]
    a = np.where(mup >= 0)[0]
    assert np.array_equal(mdown[mup[a]], a)                       # mutual both ways
    b = np.where(mdown >= 0)[0]
    assert np.array_equal(mup[mdown[b]], b)
    assert np.all(srow[mup[a]] == srow[a] + 1)                    # vertical paths
    assert np.all(ssec[mup[a]] == ssec[a])
    assert len(np.unique(mup[a])) == len(a)                       # <= 1 mutual down per cluster
    starts = np.where(res["is_start"])[0]
    assert np.all(mdown[starts] < 0) and np.all(mup[starts] >= 0)
    ct = res["cluster_track"]
    tr = res["tracks"]
    nt = res["n_tracks"]
    assert ct.max() == nt - 1 if nt else ct.max() < 0
    counts = np.bincount(ct[ct >= 0], minlength=nt)
    assert np.array_equal(counts, tr["nhits"])                    # sum of nhits = assigned
    assert np.all(tr["nhits"] >= n_min)
    # track ids follow the order of their start cluster
    first_sorted = np.argsort(order)[tr["first_cluster"]]
    assert np.all(np.diff(first_sorted) > 0)
    # every member of a track lies in one sector and consecutive rows
    for t in range(min(nt, 200)):
        idx = np.where(ct == t)[0]
        assert len(np.unique(f.sector[idx])) == 1
        rr = np.sort(f.row[idx].astype(int))
        assert np.all(np.diff(rr) == 1)
        assert rr[0] == tr["row_first"][t] and rr[-1] == tr["row_last"][t]


def test_invariants_c1():
    f = ts.generate(ts.c1())
    res = orc.track(f.sector, f.row, f.pad, f.time)
    assert res["n_tracks"] > 50
    _check_invariants(f, res)


def test_invariants_dense_pileup_slice():
    """One sector of a 2 ms continuous frame (pile-up of ~100 collisions)."""
    cfg = ts.c2()
    cfg.sector_only = 3
    f = ts.generate(cfg)
    res = orc.track(f.sector, f.row, f.pad, f.time)
    _check_invariants(f, res)
    ev = orc.evaluate(f.label, f.sector, res["cluster_track"], res["n_tracks"], len(f.trk_qpt))
    assert ev["efficiency"] > 0.97 and ev["fake_rate"] < 0.02


def test_input_order_does_not_change_result():
    f = ts.generate(ts.c1())
    a = orc.track(f.sector, f.row, f.pad, f.time)
    perm = np.random.default_rng(3).permutation(f.n)
    b = orc.track(f.sector[perm], f.row[perm], f.pad[perm], f.time[perm])
    assert a["n_tracks"] == b["n_tracks"]
    assert np.array_equal(b["cluster_track"], a["cluster_track"][perm])
    assert np.array_equal(perm[b["order"]], a["order"])


def test_empty_input():
    e = np.zeros(0)
    res = orc.track(e.astype(np.uint16), e.astype(np.uint16), e.astype(np.float32), e.astype(np.float32))
    assert res["n_tracks"] == 0


# ---------------------------------------------------------------- exact recovery
def test_exact_recovery_of_separated_noise_free_helices():
    rng = np.random.default_rng(21)
    allsec, allrow, allpad, alltime, alllab = [], [], [], [], []
    for t in range(10):
        sh = 0.05 + 0.08 * t
        eta = float(np.arcsinh(sh))
        pt = rng.uniform(0.3, 3.0)
        q = 1 if rng.uniform() < 0.5 else -1
        phi0 = np.radians(rng.uniform(3.0, 17.0))
        for r in range(152):
            res = ts.truth_at(q / pt, phi0, eta, 0.0, 0, r)
            if res is None:
                continue
            y, tb, _, _ = res
            npads = 66 + (144 * r + 151) // 302
            pitch = (4000 + (4000 * r + 151) // 302) * 1e-4
            pad = y / pitch + 0.5 * (npads - 1)
            if not (-0.5 <= pad < npads - 0.5) or not (0 <= tb < 500):
                continue
            allsec.append(0); allrow.append(r); allpad.append(pad); alltime.append(tb); alllab.append(t)
    sec = np.array(allsec, np.uint16); row = np.array(allrow, np.uint16)
    pad = np.array(allpad, np.float32); tim = np.array(alltime, np.float32); lab = np.array(alllab)
    res = orc.track(sec, row, pad, tim)
    ct = res["cluster_track"]
    found = 0
    for t in range(10):
        rows_t = np.sort(row[lab == t].astype(int))
        if rows_t.size == 0:
            continue
        # split into runs of consecutive rows (segments)
        segs = np.split(rows_t, np.where(np.diff(rows_t) != 1)[0] + 1)
        for sgm in segs:
            a, b = sgm[0], sgm[-1]
            a2 = a if a == 0 else a + 1          # inner end attaches only at row 0
            b2 = b if b == 151 else b - 1        # outer end attaches only at row 151
            members = np.where((lab == t) & (row >= a2) & (row <= b2))[0]
            if b2 - a2 + 1 < 10:
                continue
            ids = np.unique(ct[members])
            assert len(ids) == 1 and ids[0] >= 0
            assert np.array_equal(np.sort(np.where(ct == ids[0])[0]), np.sort(members))
            found += 1
    assert found == res["n_tracks"] and found >= 8


# ---------------------------------------------------------------- A2 edge-row claims
GOLDEN_A2 = os.path.join(os.path.dirname(__file__), "golden", "a2_edge_claims.txt")


def _read_golden_a2():
    cases, cur = {}, None
    for line in open(GOLDEN_A2):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = cases.setdefault(tok[1], {"cl": [], "expect": [], "mutual": []})
        elif tok[0] in ("expect", "mutual"):
            cur[tok[0]].append(tok[1:])
        else:
            cur["cl"].append((tok[0], int(tok[1]), int(tok[2]), float(tok[3]), float(tok[4])))
    return cases


@pytest.mark.parametrize("name", ["bottom", "bottom_tie", "top_tie"])
def test_golden_edge_claims(name):
    """Hand-worked claims: several claimants of different cost per edge cluster,
    a cost tie at equal time (pad decides the row-local order) and a tie between
    clusters at different times."""
    case = _read_golden_a2()[name]
    ids = [c[0] for c in case["cl"]]
    sec = np.array([c[1] for c in case["cl"]], np.uint16)
    row = np.array([c[2] for c in case["cl"]], np.uint16)
    pad = np.array([c[3] for c in case["cl"]], np.float32)
    tim = np.array([c[4] for c in case["cl"]], np.float32)
    res = orc.track(sec, row, pad, tim)
    order = res["order"]
    pos = {ids[order[p]]: p for p in range(len(ids))}
    nm = lambda p: "-" if p < 0 else ids[order[p]]
    bd, bu = orc.bruteforce_links(sec, row, pad, tim)
    nmc = lambda c: "-" if c < 0 else ids[c]
    for cid, ed, eu in case["expect"]:
        p = pos[cid]
        assert (nm(res["down"][p]), nm(res["up"][p])) == (ed, eu), cid
        assert (nmc(bd[ids.index(cid)]), nmc(bu[ids.index(cid)])) == (ed, eu), cid
    for cid, ed, eu in case["mutual"]:
        p = pos[cid]
        assert (nm(res["mdown"][p]), nm(res["mup"][p])) == (ed, eu), cid


def _random_edge_tiny(rng, ties):
    """Tiny frames around the first or last pad rows: few edge clusters, crowded
    claimant rows, so that edge clusters have several claimants (and, with
    `ties`, equal costs from coordinates snapped to a coarse grid)."""
    secs, rows, pads, times = [], [], [], []
    for s in range(int(rng.integers(1, 3))):
        top = bool(rng.integers(0, 2))
        edge_rows = [151, 150, 149, 148] if top else [0, 1, 2, 3]
        counts = [int(rng.integers(1, 4)), int(rng.integers(3, 13)), int(rng.integers(1, 7)), int(rng.integers(0, 4))]
        for r, m in zip(edge_rows, counts):
            for _ in range(m):
                secs.append(s)
                rows.append(r)
                pads.append(rng.uniform(20.0, 23.0))
                times.append(rng.uniform(100.0, 104.0))
    pads = np.array(pads, np.float32)
    times = np.array(times, np.float32)
    if ties:
        pads = (np.round(pads * 2) / 2).astype(np.float32)
        times = (np.round(times * 2) / 2).astype(np.float32)
    perm = rng.permutation(len(rows))
    return (np.array(secs, np.uint16)[perm], np.array(rows, np.uint16)[perm], pads[perm], times[perm])


def _claims_by_rule(sec, row, pad, tim, down, up, rule):
    """Edge-row claims recomputed in Python from the brute-force A1 links (caller
    indices) under a selectable rule; 'min' is the reading, the others are
    plausible mistakes the tests must be able to tell apart."""
    npads = lambda r: 66 + (144 * r + 151) // 302
    pitch = lambda r: 4000 + (4000 * r + 151) // 302
    q = lambda v: int(np.rint(np.float64(v) * 64.0))
    yq = lambda c: (q(pad[c]) - 32 * (npads(int(row[c])) - 1)) * pitch(int(row[c]))
    n = len(sec)
    key = lambda c: (float(tim[c]), float(pad[c]), c)        # row-local order
    d, u = down.copy(), up.copy()
    for e in range(n):
        re_ = int(row[e])
        if re_ not in (0, 151):
            continue
        rc = 1 if re_ == 0 else 150
        cl = [i for i in range(n) if sec[i] == sec[e] and row[i] == rc and (down[i] if re_ == 0 else up[i]) == e]
        if not cl:
            win = -1
        else:
            def cost(i):
                j, k = int(down[i]), int(up[i])
                d2y = yq(j) + yq(k) - 2 * yq(i)
                d2z = (q(tim[j]) + q(tim[k]) - 2 * q(tim[i])) * 5160
                return d2y * d2y + d2z * d2z
            cl.sort(key=key)
            if rule == "min":
                win = min(cl, key=lambda i: (cost(i), key(i)))
            elif rule == "last_of_equal":
                win = min(cl, key=lambda i: (cost(i), tuple(-x for x in key(i))))
            elif rule == "first":
                win = cl[0]
            elif rule == "last":
                win = cl[-1]
            elif rule == "max":
                win = max(cl, key=lambda i: (cost(i), tuple(-x for x in key(i))))
        if re_ == 0:
            u[e] = win
        else:
            d[e] = win
    return d, u


def _edge_corpus():
    out = []
    for seed in range(40):
        rng = np.random.default_rng(7000 + seed)
        out.append(_random_edge_tiny(rng, ties=seed % 2 == 1))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_edge_claims_match_bruteforce(seed):
    sec, row, pad, tim = _edge_corpus()[seed]
    res = orc.track(sec, row, pad, tim)
    order = res["order"]
    od = np.where(res["down"] >= 0, order[np.maximum(res["down"], 0)], -1)
    ou = np.where(res["up"] >= 0, order[np.maximum(res["up"], 0)], -1)
    bd, bu = orc.bruteforce_links(sec, row, pad, tim)
    assert np.array_equal(od, bd[order])
    assert np.array_equal(ou, bu[order])


def test_edge_claim_corpus_tells_the_rules_apart():
    """The random corpus exercises several claimants and cost ties, and every
    plausible wrong claim rule disagrees with the oracle on it somewhere, while the
    reading agrees everywhere."""
    wrong = {"first": 0, "last": 0, "max": 0, "last_of_equal": 0}
    multi = ties = 0
    for sec, row, pad, tim in _edge_corpus():
        bd, bu = orc.bruteforce_neighbours(sec, row, pad, tim)
        res = orc.track(sec, row, pad, tim)
        order = res["order"]
        od = np.where(res["down"] >= 0, order[np.maximum(res["down"], 0)], -1)[np.argsort(order)]
        ou = np.where(res["up"] >= 0, order[np.maximum(res["up"], 0)], -1)[np.argsort(order)]
        d, u = _claims_by_rule(sec, row, pad, tim, bd, bu, "min")
        assert np.array_equal(d, od) and np.array_equal(u, ou)
        for rule in wrong:
            d2, u2 = _claims_by_rule(sec, row, pad, tim, bd, bu, rule)
            wrong[rule] += int(not (np.array_equal(d2, od) and np.array_equal(u2, ou)))
        d_last, u_last = _claims_by_rule(sec, row, pad, tim, bd, bu, "last_of_equal")
        ties += int(not (np.array_equal(d_last, d) and np.array_equal(u_last, u)))
        for e in np.where((row == 0) | (row == 151))[0]:
            rc = 1 if row[e] == 0 else 150
            link = bd if row[e] == 0 else bu
            multi += int(np.sum((row == rc) & (sec == sec[e]) & (link == e)) >= 3)
    assert multi >= 10 and ties >= 2, (multi, ties)
    assert all(v > 0 for v in wrong.values()), wrong
