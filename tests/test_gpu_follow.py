"""Track following and joining (config.follow = 1) on the GPU against the oracle.

Membership is decided in FP32 on the GPU and in FP64 in the oracle, so tracks are
compared one by one: every oracle track whose margin is >= 1 (no decision about
its path, its clusters or the clusters it proposed came within the tolerance of
a threshold or a tie) must be a GPU track with exactly the same clusters, and
its refit must agree within the fit's tolerances.  The other tracks are counted
and must be few."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import COV_RTOL, FLOORS, PARAM_RTOL, as_dev, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_EXEMPT = 0.03  # at most 3 % of the tracks may sit near a decision boundary


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


def _gpu_follow(tpcca, dev, s, r, p, t, sorted_input=True, **kw):
    kw.setdefault("follow", 1)
    tr = tpcca.TimeFrameTracker(len(s) + 16, **kw)
    try:
        return run_gpu(tr, torch, dev, s, r, p, t, sorted_input=sorted_input, debug=False)
    finally:
        tr.close()


def compare_followed(g, o, offset=0, max_exempt=MAX_EXEMPT, sector=None):
    """Clear oracle tracks (margin >= 1) against the GPU's; returns the number of
    exempt tracks.  offset: position of these clusters in the GPU arrays; sector:
    the GPU's sector id of these tracks when it differs from the oracle's (an
    instance of a batched call)."""
    ct_o = o["cluster_track"]
    ct_g = g["cluster_track"][offset:offset + ct_o.size]
    n_o = o["n_tracks"]
    if n_o == 0:
        assert (ct_g < 0).all()
        return 0
    clear = o["margin"] >= 1.0
    exempt = int((~clear).sum())
    assert exempt <= max(2, max_exempt * n_o), f"{exempt} of {n_o} tracks near a decision boundary"
    first = o["tracks"]["first_cluster"] - 0  # caller index within this slice
    gid = ct_g[first]
    assert np.all(gid[clear] >= 0), "a clear oracle track has no GPU track"
    # every cluster of a clear oracle track is in the matching GPU track ...
    m = ct_o >= 0
    sel = m & clear[np.where(m, ct_o, 0)]
    assert np.array_equal(ct_g[sel], gid[ct_o[sel]]), "membership of clear tracks"
    # ... and that GPU track holds no other cluster
    size_o = np.bincount(ct_o[m], minlength=n_o)
    size_g = np.bincount(ct_g[ct_g >= 0], minlength=int(ct_g.max()) + 1 if (ct_g >= 0).any() else 1)
    assert np.array_equal(size_g[gid[clear]], size_o[clear]), "GPU tracks with extra clusters"
    assert abs(int((np.unique(ct_g[ct_g >= 0])).size) - n_o) <= exempt
    # the refit of every clear track
    ot = o["tracks"][clear]
    k = gid[clear]
    for f in ("nhits", "row_first", "row_last", "ndf", "status"):
        assert np.array_equal(g[f][k].astype(np.int64), ot[f].astype(np.int64)), f
    want_sector = ot["sector"].astype(np.int64) if sector is None else np.full(k.size, sector)
    assert np.array_equal(g["sector"][k].astype(np.int64), want_sector), "sector"
    assert np.array_equal(g["first_cluster"][k] - offset, ot["first_cluster"])
    assert np.array_equal(g["t_ref"][k], ot["t_ref"].astype(np.float32))
    dp = np.abs(g["params"][k].astype(np.float64) - ot["p"])
    lim = PARAM_RTOL * np.maximum(np.abs(ot["p"]), FLOORS)
    assert not (dp > lim).any(), f"refit parameters: worst ratio {(dp / lim).max():.3g}"
    C = ot["C"]
    diag = C[:, [0, 2, 5, 9, 14]]
    ii, jj = np.tril_indices(5)
    dc = np.abs(g["cov"][k].astype(np.float64) - C)
    clim = COV_RTOL * np.maximum(np.abs(C), 1e-3 * np.sqrt(diag[:, ii] * diag[:, jj]))
    assert not (dc > clim).any(), f"refit covariance: worst ratio {(dc / clim).max():.3g}"
    return exempt


@pytest.mark.parametrize("drop", [(70,), (6,), (145,), (40, 41), (30, 90)])
def test_broken_helices_are_joined_as_in_the_oracle(env, drop):
    from test_oracle_follow import _helices
    tpcca, dev = env
    s, r, p, t, _ = _helices(8, drop)  # generated helix by helix: not sorted
    o = orc.track_follow(s, r, p, t)
    g = _gpu_follow(tpcca, dev, s, r, p, t, sorted_input=False)
    assert compare_followed(g, o) == 0
    assert g["n_tracks"] == o["n_tracks"]
    assert np.array_equal(g["cluster_track"], o["cluster_track"])


def test_c1_matches_the_oracle(env):
    tpcca, dev = env
    f = ts.generate(ts.c1())
    o = orc.track_follow(f.sector, f.row, f.pad, f.time)
    g = _gpu_follow(tpcca, dev, f.sector, f.row, f.pad, f.time)
    compare_followed(g, o)
    assert o["stats"][2] > 0 and o["stats"][1] > 0  # joins and pick-ups happened


@pytest.fixture(scope="module")
def slice2():
    f = ts.generate(ts.c2())
    m = f.sector < 3
    return f.sector[m], f.row[m], f.pad[m], f.time[m], f.label[m]


@pytest.mark.parametrize("sorted_input", [True, False])
def test_dense_slice_matches_the_oracle(env, slice2, sorted_input):
    tpcca, dev = env
    s, r, p, t, lab = slice2
    o = orc.track_follow(s, r, p, t)
    if sorted_input:
        g = _gpu_follow(tpcca, dev, s, r, p, t)
        compare_followed(g, o)
    else:
        perm = np.random.default_rng(5).permutation(len(s))
        g = _gpu_follow(tpcca, dev, s[perm], r[perm], p[perm], t[perm], sorted_input=False)
        # back to the oracle's order: cluster_track and first_cluster are caller indices
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        g2 = dict(g)
        ct = np.empty_like(g["cluster_track"])
        ct[perm] = g["cluster_track"]
        g2["cluster_track"] = ct
        g2["first_cluster"] = perm[g["first_cluster"]]
        compare_followed(g2, o)


def test_joins_cut_clones_on_the_gpu(env, slice2):
    tpcca, dev = env
    s, r, p, t, lab = slice2
    f2 = ts.generate(ts.c2())
    n_gen = f2.trk_qpt.shape[0]
    tr = tpcca.TimeFrameTracker(len(s) + 16)
    try:
        plain = run_gpu(tr, torch, dev, s, r, p, t, debug=False)
    finally:
        tr.close()
    fol = _gpu_follow(tpcca, dev, s, r, p, t)
    ea = orc.evaluate(lab, s, plain["cluster_track"], plain["n_tracks"], n_gen)
    eb = orc.evaluate(lab, s, fol["cluster_track"], fol["n_tracks"], n_gen)
    assert eb["efficiency"] >= ea["efficiency"] - 5e-4
    assert eb["clone_rate"] < ea["clone_rate"] / 4


def test_batched_instances_follow_independently(env):
    tpcca, dev = env
    b = ts.batched(12, seed=9, n_min=2e3, n_max=3e4, ms_min=0.2, ms_max=1.0)
    f, off = b.frame, b.offsets
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=off.size - 1, follow=1)
    try:
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
    finally:
        tr.close()
    first_id = 0
    for k in range(off.size - 1):
        a, e = off[k], off[k + 1]
        o = orc.track_follow(np.zeros(e - a, np.uint16), f.row[a:e], f.pad[a:e], f.time[a:e])
        compare_followed(g, o, offset=a, sector=k)
        ids = g["cluster_track"][a:e]
        if (ids >= 0).any():
            assert ids[ids >= 0].min() >= first_id
            first_id = ids.max() + 1
        assert np.all(g["sector"][np.unique(ids[ids >= 0])] == k)


def test_graph_and_host_paths_equal_the_direct_call(env, slice2):
    tpcca, dev = env
    s, r, p, t, _ = slice2
    tr = tpcca.TimeFrameTracker(len(s) + 16, follow=1)
    try:
        direct = run_gpu(tr, torch, dev, s, r, p, t, debug=False)
        sd, rd, pd, td = as_dev(torch, dev, s, r, p, t)
        cap = len(s) // 10 + 1
        for _ in range(2):
            tr._out["cluster_track"].fill_(-7)
            nt = tr.track_graph(sd, rd, pd, td, capacity=cap)
            torch.cuda.synchronize()
            assert tpcca.tpc_tf_status(tr.handle, 0) == 0
            assert int(nt.item()) == direct["n_tracks"]
            assert np.array_equal(tr._out["cluster_track"][:len(s)].cpu().numpy(), direct["cluster_track"])
        host = tr.track_host(s, r, p, t, capacity=cap)
        assert host["n_tracks"] == direct["n_tracks"]
        assert np.array_equal(host["cluster_track"], direct["cluster_track"])
        m = direct["n_tracks"]
        assert np.array_equal(host["params"][:m], direct["params"][:m])
    finally:
        tr.close()


def test_capacity_error_reports_the_followed_count(env, slice2):
    tpcca, dev = env
    s, r, p, t, _ = slice2
    full = _gpu_follow(tpcca, dev, s, r, p, t)
    tr = tpcca.TimeFrameTracker(len(s) + 16, follow=1)
    try:
        with pytest.raises(tpcca.TpcError) as ei:
            run_gpu(tr, torch, dev, s, r, p, t, capacity=full["n_tracks"] - 1, debug=False)
        assert ei.value.code == tpcca.TPC_ERR_CAPACITY
        g = run_gpu(tr, torch, dev, s, r, p, t, capacity=full["n_tracks"], debug=False)
        assert np.array_equal(g["cluster_track"], full["cluster_track"])
    finally:
        tr.close()


def test_pruned_mode_follow_keeps_every_chain_whole(env, slice2):
    """With the classifier the chains differ from the plain ones, so the check is
    structural: every chain track of the pruned call lies inside one followed
    track, pick-ups are clusters no chain held, rows strictly increase."""
    import json
    import os
    tpcca, dev = env
    s, r, p, t, _ = slice2
    w = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2102_08862_gb300",
                     "weights", "link_classifier")
    blob = open(w + ".bin", "rb").read()
    tau = json.load(open(w + ".json"))["tau"]
    outs = {}
    for fol in (0, 1):
        tr = tpcca.TimeFrameTracker(len(s) + 16, mode=tpcca.TPC_MODE_PRUNED, tau=tau, follow=fol)
        try:
            tr.load_mlp(blob)
            outs[fol] = run_gpu(tr, torch, dev, s, r, p, t, debug=False)
        finally:
            tr.close()
    a, b = outs[0]["cluster_track"], outs[1]["cluster_track"]
    assert np.all(b[a >= 0] >= 0)
    pairs = np.unique(np.stack([a[a >= 0], b[a >= 0]], 1), axis=0)
    assert np.unique(pairs[:, 0]).size == pairs.shape[0], "a chain split over two followed tracks"
    assert outs[1]["n_tracks"] < outs[0]["n_tracks"]
    order = np.lexsort((r, b))
    bs, rs = b[order], r[order].astype(int)
    keep = bs >= 0
    bs, rs = bs[keep], rs[keep]
    same = bs[1:] == bs[:-1]
    assert np.all(rs[1:][same] > rs[:-1][same])
    nh = np.bincount(b[b >= 0], minlength=outs[1]["n_tracks"])
    assert np.array_equal(outs[1]["nhits"][:outs[1]["n_tracks"]], nh)


# ---------------------------------------------------------------- cross-sector links
def test_crossing_helices_are_linked_as_in_the_oracle(env):
    from test_oracle_follow import _crossing_helices
    tpcca, dev = env
    s, r, p, t, _ = _crossing_helices(10)  # not sorted
    o = orc.track_follow(s, r, p, t, fp=orc.follow_params(links=1))
    g = _gpu_follow(tpcca, dev, s, r, p, t, sorted_input=False, follow=2)
    assert np.all(o["margin"] >= 1) and np.all(o["xmargin"] >= 1)
    assert np.array_equal(g["cluster_track"], o["cluster_track"])
    assert np.array_equal(g["next_track"][:g["n_tracks"]], o["next"])
    assert (o["next"] >= 0).sum() >= 5


@pytest.mark.parametrize("sorted_input", [True, False])
def test_dense_slice_links_match_the_oracle(env, slice2, sorted_input):
    tpcca, dev = env
    s, r, p, t, _ = slice2
    o = orc.track_follow(s, r, p, t, fp=orc.follow_params(links=1))
    if sorted_input:
        g = _gpu_follow(tpcca, dev, s, r, p, t, follow=2)
        ct_g = g["cluster_track"]
    else:
        perm = np.random.default_rng(6).permutation(len(s))
        g = _gpu_follow(tpcca, dev, s[perm], r[perm], p[perm], t[perm], sorted_input=False, follow=2)
        ct_g = np.empty_like(g["cluster_track"])
        ct_g[perm] = g["cluster_track"]
    n_o = o["n_tracks"]
    clear = (o["margin"] >= 1) & (o["xmargin"] >= 1)
    gid = ct_g[o["tracks"]["first_cluster"]]  # the GPU track of each oracle track
    nxt_o = o["next"]
    want = np.where(nxt_o >= 0, gid[np.maximum(nxt_o, 0)], -1)
    both = clear & ((nxt_o < 0) | clear[np.maximum(nxt_o, 0)])
    got = g["next_track"][gid[both]]
    assert np.array_equal(got, want[both]), f"{(got != want[both]).sum()} links differ"
    assert (~both).sum() <= MAX_EXEMPT * n_o  # links of tracks near a decision boundary
    assert (nxt_o >= 0).sum() > 1000


def test_full_size_10ms_frame_follow_sampled_sectors(env):
    """The 10 ms frame (~32M clusters) with follow = 2, as the benchmark's follow line
    runs it.  Whole frame: the chains of the follow-free call each lie inside one
    followed track, rows strictly increase along every track, links join tracks of
    neighbouring sectors of one side.  Two sectors (sectors follow independently;
    links, which cross sectors, are checked structurally) are recomputed by the
    oracle: every oracle track clear of the band is a GPU track with exactly its
    clusters and the same refit."""
    tpcca, dev = env
    f = ts.generate(ts.c3())
    outs = {}
    for fol in (0, 2):
        tr = tpcca.TimeFrameTracker(f.n, follow=fol)
        try:
            outs[fol] = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
        finally:
            tr.close()
    a, g = outs[0]["cluster_track"], outs[2]
    b = g["cluster_track"]
    nt = g["n_tracks"]
    assert np.all(b[a >= 0] >= 0)
    pairs = np.unique(np.stack([a[a >= 0], b[a >= 0]], 1), axis=0)
    assert np.unique(pairs[:, 0]).size == pairs.shape[0], "a chain split over two followed tracks"
    order = np.lexsort((f.row, b))
    bs, rs = b[order], f.row[order].astype(np.int64)
    keep = bs >= 0
    same = bs[keep][1:] == bs[keep][:-1]
    assert np.all(rs[keep][1:][same] > rs[keep][:-1][same])
    nxt = g["next_track"][:nt]
    linked = np.nonzero(nxt >= 0)[0]
    sec = g["sector"][:nt].astype(np.int64)
    d = (sec[nxt[linked]] % 18 - sec[linked] % 18) % 18
    assert linked.size > 50000 and np.all((d == 1) | (d == 17))
    assert np.all(sec[nxt[linked]] // 18 == sec[linked] // 18)
    assert np.unique(nxt[linked]).size == linked.size
    for s in (5, 27):
        idx = np.where(f.sector == s)[0]
        o = orc.track_follow(f.sector[idx], f.row[idx], f.pad[idx], f.time[idx])
        sub = dict(g)
        sub["cluster_track"] = b[idx]
        inv = np.full(f.n, -1, np.int64)
        inv[idx] = np.arange(len(idx))
        sub["first_cluster"] = np.where(g["first_cluster"] >= 0, inv[np.maximum(g["first_cluster"], 0)], -1)
        compare_followed(sub, o, sector=s)
