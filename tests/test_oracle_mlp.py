"""Pins of the oracle's learned link classifier: BF16 rounding, the triplet
features, the 12 -> 64 -> 64 -> 1 network, its loss gradient, the pruned
neighbour rule and the training-set extraction.  The classifier is an extension
of the paper's CA seeding (Sec. 1), which has no learned part; what is pinned
here is the reading written in oracle/mlp.c."""
import math

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from mlp_util import random_net, zero_theta, theta_views

torch = pytest.importorskip("torch")


# ---------------------------------------------------------------- BF16
def test_bf16_round_to_nearest_even_closed_forms():
    assert orc.bf16(1.0) == 1.0
    assert orc.bf16(1.0 + 2.0 ** -8) == 1.0                     # half an ulp: tie to even (down)
    assert orc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # 1.5 ulp: tie to even (up)
    assert orc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7  # above the tie
    assert orc.bf16(-3.0) == -3.0
    assert math.isinf(orc.bf16(3.4e38))                         # rounds past the largest BF16


def test_bf16_matches_torch_conversion():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(4000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 4000),
                        rng.integers(-2 ** 20, 2 ** 20, 1000).astype(np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    ours = np.array([orc.bf16(v) for v in x], np.float32)
    assert np.array_equal(ours, ref)


# ---------------------------------------------------------------- features
def test_feature_log1p_within_fp32_error_of_log1p():
    v = np.concatenate([np.linspace(0, 100, 2001), np.geomspace(1e-6, 100, 500)]).astype(np.float32)
    got = np.array([orc.feature_log1p(x) for x in v])
    # u = 1 + v is rounded first: compare with ln(fl(1 + v)) to a few FP32 ulps
    u = (np.float32(1.0) + v).astype(np.float64)
    ref = np.log(u)
    assert np.all(np.abs(got - ref) <= 4 * np.spacing(np.float32(np.maximum(ref, 1e-30))) + 1e-7)
    assert orc.feature_log1p(0.0) == 0.0


def test_features_units_and_meaning():
    # a triplet on row 10: j one cm below i, k one cm above in y; one bin apart in time
    r, yi, ti = 10, 3_200_000, 6400
    yj, yk = yi - 640_000, yi + 640_000
    tj, tk = ti - 64, ti + 64
    f = orc.mlp_features(r, yj, yi, yk, tj, ti, tk, cost=0, nj=3, nk=5)
    xr = 85.0 + r * 160.0 / 151.0
    assert abs(f[0] - 1.0) < 1e-6 and abs(f[1] - 1.0) < 1e-6           # cm
    assert abs(f[2] - 0.516) < 1e-6 and abs(f[3] - 0.516) < 1e-6       # one bin = 0.516 cm
    assert f[4] == 0.0 and f[5] == 0.0 and f[8] == 0.0                 # a straight line
    assert abs(f[6] - xr / 250.0) < 1e-6
    assert abs(f[7] - 5.0 / xr) < 1e-6                                 # y_i = 5 cm
    assert f[9] == 3 / 8 and f[10] == 5 / 8
    assert f[11] == 0.0
    # a kinked triplet: d2y = 1 cm, d2z = 2 bins; cost at the cut
    cmax = 147456000000
    f = orc.mlp_features(r, yi, yi, yi + 640_000, ti, ti, ti + 128, cost=cmax, nj=1, nk=2)
    assert abs(f[4] - 1.0) < 1e-6 and abs(f[5] - 1.032) < 1e-6
    assert abs(f[8] - 1.0 / (160.0 / 151.0) ** 2) < 1e-6
    assert abs(f[11] - math.log(101.0)) < 1e-6
    # order of the operands: f0 = y_i - y_j, f1 = y_k - y_i, f2/f3 likewise
    f = orc.mlp_features(r, yi - 64_000, yi, yi + 128_000, ti - 1, ti, ti + 2, cost=5, nj=1, nk=1)
    assert f[0] > 0 and abs(f[1] / f[0] - 2.0) < 1e-6
    assert f[2] > 0 and abs(f[3] / f[2] - 2.0) < 1e-6


# ---------------------------------------------------------------- network
def _blob(mean, inv_std, theta):
    return orc.mlp_blob(mean, inv_std, theta)


def test_logit_of_bias_only_network():
    th = zero_theta()
    theta_views(th)["b3"][:] = -1.25
    blob = _blob(np.zeros(12), np.ones(12), th)
    f = np.random.default_rng(1).standard_normal((20, 12)).astype(np.float32)
    assert np.all(orc.mlp_logits(blob, f) == -1.25)


@pytest.mark.parametrize("c", [0, 5, 11])
def test_logit_of_absolute_value_network(c):
    # h1_0 = relu(x_c), h1_1 = relu(-x_c); h2_0 = h1_0 + h1_1 = |x_c|; logit = h2_0
    th = zero_theta()
    v = theta_views(th)
    v["W1"][0, c], v["W1"][1, c] = 1.0, -1.0
    v["W2"][0, 0] = v["W2"][0, 1] = 1.0
    v["w3"][0] = 1.0
    rng = np.random.default_rng(c)
    mean = rng.standard_normal(12).astype(np.float32)
    inv_std = (0.5 + rng.random(12)).astype(np.float32)
    blob = _blob(mean, inv_std, th)
    f = rng.standard_normal((50, 12)).astype(np.float32)
    g = ((f[:, c] - mean[c]).astype(np.float32) * inv_std[c]).astype(np.float32)
    want = np.abs(np.array([orc.bf16(x) for x in g]))
    assert np.array_equal(orc.mlp_logits(blob, f), want)


def test_logit_routes_each_feature_through_its_own_weights():
    # W1[o, c] = 1 only for o = c: hidden unit c carries feature c; w3 weights them by 2^c
    th = zero_theta()
    v = theta_views(th)
    for c in range(12):
        v["W1"][c, c] = 1.0
        v["W2"][c, c] = 1.0
        v["w3"][c] = 2.0 ** c
    blob = _blob(np.zeros(12), np.ones(12), th)
    for c in range(12):
        f = np.zeros((1, 12), np.float32)
        f[0, c] = 3.0
        assert orc.mlp_logits(blob, f)[0] == 3.0 * 2.0 ** c


def test_first_hidden_layer_is_rounded_to_bf16():
    th = zero_theta()
    v = theta_views(th)
    v["W1"][0, 0] = 1.0
    v["b1"][0] = 2.0 ** -8          # z1 = 1 + 2^-8: a BF16 tie, rounds to 1
    v["W2"][0, 0] = 1.0
    v["w3"][0] = 1.0
    blob = _blob(np.zeros(12), np.ones(12), th)
    f = np.zeros((1, 12), np.float32)
    f[0, 0] = 1.0
    assert orc.mlp_logits(blob, f)[0] == 1.0
    v["b2"][0] = 2.0 ** -8          # the second layer is not rounded
    blob = _blob(np.zeros(12), np.ones(12), th)
    assert orc.mlp_logits(blob, f)[0] == 1.0 + 2.0 ** -8


# ---------------------------------------------------------------- loss, gradient
def test_loss_and_gradient_of_bias_only_network():
    th = zero_theta().astype(np.float64)
    theta_views(th)["b3"][:] = 0.3
    rng = np.random.default_rng(3)
    f = rng.standard_normal((17, 12)).astype(np.float32)
    y = (rng.random(17) < 0.4).astype(np.uint8)
    pw = 2.5
    loss, g = orc.mlp_loss_grad(th, np.zeros(12), np.ones(12), f, y, pos_weight=pw)
    w = np.where(y == 1, pw, 1.0)
    sp = math.log1p(math.exp(0.3))
    assert abs(loss - np.mean(w * (sp - y * 0.3))) < 1e-14
    sig = 1.0 / (1.0 + math.exp(-0.3))
    assert abs(g[-1] - np.mean(w * (sig - y))) < 1e-14
    assert np.all(g[:-1] == 0.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    mean, inv_std, theta = random_net(seed)
    theta = theta.astype(np.float64)
    rng = np.random.default_rng(100 + seed)
    f = (mean + rng.standard_normal((48, 12)) / inv_std).astype(np.float32)
    y = (rng.random(48) < 0.3).astype(np.uint8)
    _, g = orc.mlp_loss_grad(theta, mean, inv_std, f, y, pos_weight=1.7)
    h = 1e-6
    idx = np.arange(theta.size)
    fd = np.zeros(theta.size)
    for p in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (orc.mlp_loss_grad(tp, mean, inv_std, f, y, 1.7)[0] - orc.mlp_loss_grad(tm, mean, inv_std, f, y, 1.7)[0]) / (2 * h)
    scale = np.max(np.abs(g))
    assert scale > 1e-4
    # ReLU kinks could spoil a difference; none lies within h of a random network's pre-activations
    assert np.max(np.abs(fd - g)) <= 1e-6 * scale + 1e-9


def test_gradient_check_notices_a_wrong_sign():
    """A planted mistake (the positive-class weight applied to negatives) changes the gradient."""
    mean, inv_std, theta = random_net(4)
    rng = np.random.default_rng(5)
    f = (mean + rng.standard_normal((32, 12)) / inv_std).astype(np.float32)
    y = (rng.random(32) < 0.5).astype(np.uint8)
    _, g1 = orc.mlp_loss_grad(theta, mean, inv_std, f, y, pos_weight=3.0)
    _, g2 = orc.mlp_loss_grad(theta, mean, inv_std, f, 1 - y, pos_weight=3.0)
    assert np.max(np.abs(g1 - g2)) > 1e-3 * np.max(np.abs(g1))


# ---------------------------------------------------------------- pruned neighbours
def _tiny(seed):
    """A few rows with clusters crowded within ~1 pad and ~1 bin, so that most
    middle-row clusters have several pairs under the cost cut (odd seeds snap to a
    grid so that equal costs occur)."""
    rng = np.random.default_rng(5000 + seed)
    r0 = int(rng.integers(1, 140))
    secs, rows, pads, times = [], [], [], []
    for s in range(int(rng.integers(1, 3))):
        for r in range(r0, r0 + int(rng.integers(3, 6))):
            m = int(rng.integers(1, 9))
            secs += [s] * m
            rows += [r] * m
            pads += list(rng.uniform(22.0, 23.5, m))
            times += list(rng.uniform(100.0, 101.5, m))
    pads, times = np.array(pads, np.float32), np.array(times, np.float32)
    if seed % 2:
        pads = (np.round(pads * 4) / 4).astype(np.float32)
        times = (np.round(times * 4) / 4).astype(np.float32)
    perm = rng.permutation(len(rows))
    return (np.array(secs, np.uint16)[perm], np.array(rows, np.uint16)[perm], pads[perm], times[perm])


def _brute_pruned(sec, row, pad, tim, blob, tau, prm):
    """Per cluster: every (j, k) of the adjacent rows inside the windows, by
    enumeration over all clusters (no sort, no search); scores from the oracle's
    own logit (pinned above); the rule applied literally."""
    pq, tq, yq, zq = orc.quantize(row, pad, tim)
    order = orc.sort_order(sec, row, pad, tim)
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    n = sec.size
    down, up = np.full(n, -1), np.full(n, -1)
    for i in range(n):
        r = int(row[i])
        if r == 0 or r == 151:
            continue
        js = [j for j in range(n) if sec[j] == sec[i] and row[j] == r - 1 and abs(int(tq[j]) - int(tq[i])) <= prm.wt_q
              and abs(int(yq[j]) - int(yq[i])) <= prm.wy_q]
        ks = [k for k in range(n) if sec[k] == sec[i] and row[k] == r + 1 and abs(int(tq[k]) - int(tq[i])) <= prm.wt_q
              and abs(int(yq[k]) - int(yq[i])) <= prm.wy_q]
        cands = []
        for j in js:
            for k in ks:
                d2y = int(yq[j]) + int(yq[k]) - 2 * int(yq[i])
                d2z = int(zq[j]) + int(zq[k]) - 2 * int(zq[i])
                c = d2y * d2y + d2z * d2z
                if c <= prm.cost_max_q:
                    cands.append((c, int(rank[j]), int(rank[k]), j, k))
        if not cands:
            continue
        plain = min(cands)
        choice = plain
        if len(cands) >= 2:
            feats = np.stack([orc.mlp_features(r, yq[j], yq[i], yq[k], tq[j], tq[i], tq[k], c, len(js), len(ks))
                              for c, _, _, j, k in cands])
            sc = 1.0 / (1.0 + np.exp(-orc.mlp_logits(blob, feats)))
            kept = [cd for cd, s in zip(cands, sc) if s >= tau]
            if kept:
                choice = min(kept)
        down[i], up[i] = choice[3], choice[4]
    return down, up


@pytest.mark.parametrize("seed", range(16))
def test_pruned_neighbours_match_bruteforce(seed):
    sec, row, pad, tim = _tiny(seed)
    if sec.size == 0:
        return
    mean, inv_std, theta = random_net(seed, feature_scale=True)
    blob = orc.mlp_blob(mean, inv_std, theta)
    prm = orc.params()
    order = orc.sort_order(sec, row, pad, tim)
    for tau in (0.3, 0.5, 0.7):
        d, u, _, _, stats = orc.neighbours_pruned(sec[order], row[order], pad[order], tim[order], blob, tau)
        od = np.where(d >= 0, order[np.maximum(d, 0)], -1)
        ou = np.where(u >= 0, order[np.maximum(u, 0)], -1)
        bd, bu = _brute_pruned(sec, row, pad, tim, blob, tau, prm)
        assert np.array_equal(od, bd[order]) and np.array_equal(ou, bu[order])


def test_pruned_reduces_to_plain_at_extreme_thresholds():
    f = ts.generate(ts.c1())
    d0, u0, c0 = orc.neighbours_sorted(f.sector, f.row, f.pad, f.time)
    mean, inv_std, theta = random_net(9, feature_scale=True)
    blob = orc.mlp_blob(mean, inv_std, theta)
    for tau in (0.0, 1.5):  # every pair passes / no pair passes (fallback to the plain choice)
        d, u, c, band, stats = orc.neighbours_pruned(f.sector, f.row, f.pad, f.time, blob, tau)
        assert np.array_equal(d, d0) and np.array_equal(u, u0) and np.array_equal(c, c0)
        assert stats[0] > 0 and stats[1] >= 2 * stats[0] and stats[2] == 0
    d, u, c, band, stats = orc.neighbours_pruned(f.sector, f.row, f.pad, f.time, blob, 1.5)
    assert stats[3] == stats[0]  # all ambiguous clusters fell back


# ---------------------------------------------------------------- training set
def test_training_triplets_invariants_c1():
    f = ts.generate(ts.c1())
    feat, lab, tri = orc.training_triplets(f.sector, f.row, f.pad, f.time)
    assert feat.shape[0] == lab.shape[0] == tri.shape[0] > 50
    res = orc.track(f.sector, f.row, f.pad, f.time)
    order = res["order"]
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    pq, tq, yq, zq = orc.quantize(f.row, f.pad, f.time)
    i_s, j_s, k_s = rank[tri[:, 0]], rank[tri[:, 1]], rank[tri[:, 2]]
    # every cluster appears with >= 2 pairs; at most one positive each
    ui, cnt = np.unique(i_s, return_counts=True)
    assert np.all(cnt >= 2)
    pos = np.bincount(i_s, weights=lab, minlength=order.size)
    assert pos.max() <= 1
    # positives = plain choice with both links mutual
    want = ((res["down"][i_s] == j_s) & (res["up"][i_s] == k_s) & (res["mdown"][i_s] == j_s)
            & (res["mup"][i_s] == k_s))
    assert np.array_equal(lab.astype(bool), want)
    assert lab.sum() > 0 and lab.sum() < lab.size
    # rows reproduce from the features' definition
    for m in range(0, feat.shape[0], max(1, feat.shape[0] // 25)):
        i, j, k = tri[m]
        d2y = int(yq[j]) + int(yq[k]) - 2 * int(yq[i])
        d2z = int(zq[j]) + int(zq[k]) - 2 * int(zq[i])
        g = orc.mlp_features(f.row[i], yq[j], yq[i], yq[k], tq[j], tq[i], tq[k], d2y * d2y + d2z * d2z,
                             int(round(feat[m, 9] * 8)), int(round(feat[m, 10] * 8)))
        assert np.array_equal(g, feat[m])
        assert d2y * d2y + d2z * d2z <= 147456000000
