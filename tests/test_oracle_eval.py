"""Pins of the oracle's efficiency / clone / fake evaluation against a hand-built
case whose rates are worked out by hand (definitions: a track is matched when one
generator label holds >= 90 % of its clusters; findable = (generator track, sector)
with >= 30 clusters)."""
import numpy as np

import oracle as orc
import pytest
import tpcsynth as ts


def test_eval_hand_built_case():
    lab, sec, trk = [], [], []

    def add(label, track, count, sector=0):
        lab.extend([label] * count)
        sec.extend([sector] * count)
        trk.extend([track] * count)

    add(0, 0, 38); add(-1, 0, 2)        # T0: 38/40 of label 0 -> matched (findable 0)
    add(0, 1, 20)                       # T1: label 0 again -> clone
    add(0, -1, 2)                       # two label-0 clusters unassigned (label 0 has 60)
    add(1, 2, 10); add(2, 2, 5)         # T2: 10/15 -> fake
    add(1, -1, 29)                      # label 1 has 40 clusters in sector 0 (findable)
    add(2, 3, 12)                       # T3: label 2 (20 clusters, not findable): matched, not counted
    add(2, -1, 3)
    add(3, 4, 6); add(4, 4, 6)          # T4: majority tie -> label 3, 6/12 -> fake
    add(-1, 5, 8); add(1, 5, 1)         # T5: majority noise -> fake
    add(5, -1, 35, sector=7)            # label 5: findable in sector 7, never found
    lab, sec, trk = np.array(lab), np.array(sec), np.array(trk)
    perm = np.random.default_rng(0).permutation(len(lab))   # order must not matter
    ev = orc.evaluate(lab[perm], sec[perm], trk[perm], n_tracks=6, n_gen_tracks=6)
    assert ev["n_findable"] == 3          # (0, s0), (1, s0), (5, s7)
    assert ev["n_findable_found"] == 1
    assert ev["n_matched_findable_tracks"] == 2
    assert ev["n_fake"] == 3
    assert abs(ev["efficiency"] - 1 / 3) < 1e-15
    assert abs(ev["clone_rate"] - 1 / 3) < 1e-15
    assert abs(ev["fake_rate"] - 3 / 6) < 1e-15


def test_eval_perfect_and_empty():
    lab = np.repeat(np.arange(4), 50)
    sec = np.zeros_like(lab)
    ev = orc.evaluate(lab, sec, lab.copy(), n_tracks=4, n_gen_tracks=4)
    assert ev["efficiency"] == 1.0 and ev["clone_rate"] == 0.0 and ev["fake_rate"] == 0.0
    ev = orc.evaluate(lab, sec, np.full_like(lab, -1), n_tracks=0, n_gen_tracks=4)
    assert ev["efficiency"] == 0.0 and ev["n_tracks"] == 0


def test_package_evaluator_matches_oracle():
    """The host-side evaluator of the package reproduces the oracle's counts."""
    from paper_2102_08862_gb300.evaluate import evaluate as pkg_eval
    f = ts.generate(ts.c1())
    res = orc.track(f.sector, f.row, f.pad, f.time)
    ng = int(f.trk_qpt.shape[0])
    for mf in (10, 30):
        want = orc.evaluate(f.label, f.sector, res["cluster_track"], res["n_tracks"], ng, min_findable=mf)
        got = pkg_eval(f.label, f.sector, res["cluster_track"], res["n_tracks"], ng, min_findable=mf)
        assert got == pytest.approx(want)
    # a noisy assignment: random track ids over a subset of clusters
    rng = np.random.default_rng(3)
    ct = np.where(rng.random(f.n) < 0.7, rng.integers(0, 50, f.n), -1).astype(np.int32)
    want = orc.evaluate(f.label, f.sector, ct, 50, ng, min_findable=5, match_frac=0.3)
    got = pkg_eval(f.label, f.sector, ct, 50, ng, min_findable=5, match_frac=0.3)
    assert got == pytest.approx(want)
