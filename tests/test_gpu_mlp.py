"""GPU parity of the learned link classifier (through the C ABI) with the CPU
oracle: features and labels of the training set bit for bit, logits within the
BF16/FP32 tolerance, pruned links identical outside the score band around tau,
gradients of the training kernels against the FP64 oracle gradient, and one Adam
step against its closed form.  The classifier extends the paper's CA seeding
(Sec. 1), which has no learned part."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import compare_links, compare_tracks, run_gpu, as_dev
from mlp_util import logit_flip_bound, random_net

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# GPU logit vs oracle logit: FP32 accumulation against FP64 moves a logit by
# ~1e-6 relative; a first-layer unit whose FP32 sum lands on the other side of a
# BF16 rounding boundary than the FP64 sum moves it by one BF16 step of that unit
# (2^-8 relative) times its weight path, ~1e-3 at the scales here.
LOGIT_ATOL, LOGIT_RTOL = 5e-3, 5e-3
# per row (scorer test): 2^-18 of the scale of the FP32 sums, plus 1.5 x the
# first-layer rounding flips that mlp_util.logit_flip_bound allows for that row
LOGIT_SUM_TOL = 2.0 ** -18


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def c1():
    return ts.generate(ts.c1())


@pytest.fixture(scope="module")
def two_sectors():
    """Sectors 0-1 of a 2 ms Pb-Pb-like frame (seed 2): ~3e5 clusters, thousands of ambiguous clusters."""
    f = ts.generate(ts.c2())
    m = f.sector < 2
    return ts.Frame(sector=f.sector[m], row=f.row[m], pad=f.pad[m], time=f.time[m], label=f.label[m],
                    trk_qpt=f.trk_qpt, trk_phi0=f.trk_phi0, trk_eta=f.trk_eta, trk_t0=f.trk_t0,
                    trk_collision=f.trk_collision, n_collisions=f.n_collisions, frame_bins=f.frame_bins)


def _net(seed=3):
    mean, inv_std, theta = random_net(seed, feature_scale=True)
    return orc.mlp_blob(mean, inv_std, theta)


def _dev_tensor(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _sort_rows(tri):
    return np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0]))


# ------------------------------------------------------------------ training set
@pytest.mark.parametrize("unsorted", [False, True])
def test_extract_matches_oracle_training_set(env, c1, unsorted):
    tpcca, dev = env
    f = c1
    perm = np.random.default_rng(4).permutation(f.n) if unsorted else np.arange(f.n)
    s, r, p, t = f.sector[perm], f.row[perm], f.pad[perm], f.time[perm]
    of, ol, otri = orc.training_triplets(s, r, p, t)
    tr = tpcca.TimeFrameTracker(f.n + 16)
    try:
        gf, gl, gtri = tr.extract(*as_dev(torch, dev, s, r, p, t), sorted_input=not unsorted)
        gf, gl, gtri = gf.cpu().numpy(), gl.cpu().numpy(), gtri.cpu().numpy()
    finally:
        tr.close()
    assert gf.shape == of.shape and of.shape[0] > 100
    go, oo = _sort_rows(gtri), _sort_rows(otri)
    assert np.array_equal(gtri[go], otri[oo])
    assert np.array_equal(gl[go], ol[oo])
    assert np.array_equal(gf[go].view(np.uint32), of[oo].view(np.uint32)), "features must match bit for bit"


def test_extract_capacity_counts_all_rows(env, c1):
    tpcca, dev = env
    tr = tpcca.TimeFrameTracker(c1.n + 16)
    try:
        full = tr.extract(*as_dev(torch, dev, c1.sector, c1.row, c1.pad, c1.time))[0].shape[0]
        d = torch.device("cuda", 0)
        s, r, p, t = as_dev(torch, dev, c1.sector, c1.row, c1.pad, c1.time)
        cl = tpcca.tpc_clusters(n=c1.n, flags=tpcca.TPC_INPUT_SORTED, sector=s.data_ptr(), row=r.data_ptr(),
                                pad=p.data_ptr(), time=t.data_ptr())
        feat = torch.full((10, 12), -1.0, device=d)
        lab = torch.full((11,), 7, dtype=torch.uint8, device=d)
        cnt = torch.zeros(1, dtype=torch.int32, device=d)
        assert tpcca.tpc_mlp_extract(tr.handle, cl, feat.data_ptr(), lab.data_ptr(), None, 10, cnt.data_ptr(), 0) == 0
        torch.cuda.synchronize()
        assert int(cnt.item()) == full
        assert int(lab[10].item()) == 7  # nothing written past the capacity
    finally:
        tr.close()


# ------------------------------------------------------------------ scoring
@pytest.mark.parametrize("engine", [0, 1])  # tcgen05 (tensor memory), mma.sync
def test_scores_match_oracle_logits(env, c1, engine):
    tpcca, dev = env
    blob = _net()
    feat, _, _ = orc.training_triplets(c1.sector, c1.row, c1.pad, c1.time)
    rng = np.random.default_rng(8)
    # ragged, and enough rows (~90 k) that most SMs run two or more CTAs at once
    extra = (rng.standard_normal((90_333, 12)) * [0.5, 0.5, 1, 1, .2, .2, .2, .1, .2, .1, .1, 1.5]
             + [0, 0, 0, 0, 0, 0, .66, 0, 0, .15, .15, 2]).astype(np.float32)
    feat = np.concatenate([feat, extra]).astype(np.float32)  # not a multiple of 16 or 256 rows
    want = orc.mlp_logits(blob, feat)
    tr = tpcca.TimeFrameTracker(1024)
    try:
        tr.load_mlp(blob)
        got = tr.score(_dev_tensor(feat, dev), engine=engine).cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        assert tpcca.tpc_tf_status(tr.handle, 0) == 0
    finally:
        tr.close()
    err = np.abs(got - want)
    flips, scale = logit_flip_bound(*tpcca.unpack_blob(blob), feat)
    lim = LOGIT_SUM_TOL * scale + 1.5 * flips
    assert np.all(err <= lim), f"worst {np.max(err / lim):.3g} of the tolerance (row {int(np.argmax(err / lim))})"
    assert np.median(err) < 1e-4
    assert (flips > 0).mean() < 0.4  # the bound widens only for rows near a rounding midpoint


@pytest.mark.parametrize("engine", [0, 1])  # tcgen05 (tensor memory), mma.sync
def test_scores_carry_the_second_layer_bias_exactly(env, engine):
    """With W1, b1 and W2 zero, Z2 = b2 exactly and the logit is b3 + sum_o w3_o b2_o (all
    positive here, so every unit is active and rounding errors of b2 add up): the GPU may differ
    from the FP64 oracle only by its FP32 sum of 65 positive terms, at most 64 x 2^-24 = 2^-18 of
    the sum in any summation order.  Each b2 needs all 24 bits of its significand (1 + 2^-9 +
    2^-17 times a power of two: three BF16 parts); carried as two parts it would be off by 2^-17
    of itself, twice the bound."""
    tpcca, dev = env
    from mlp_util import theta_views, zero_theta
    rng = np.random.default_rng(21)
    theta = zero_theta()
    v = theta_views(theta)
    frac = np.float32(1.0 + 2.0 ** -9 + 2.0 ** -17)
    v["b2"][:] = (frac * np.float32(2.0) ** rng.integers(-6, 3, 64)).astype(np.float32)
    v["w3"][:] = np.abs(rng.standard_normal(64)) * 0.5 + 0.05
    v["b3"][:] = 0.25
    mean, inv_std = np.zeros(12, np.float32), np.ones(12, np.float32)
    blob = orc.mlp_blob(mean, inv_std, theta)
    feat = rng.standard_normal((1000, 12)).astype(np.float32)
    want = orc.mlp_logits(blob, feat)
    assert np.all(want == want[0])  # the inputs do not reach the logit
    tr = tpcca.TimeFrameTracker(1024)
    try:
        tr.load_mlp(blob)
        got = tr.score(_dev_tensor(feat, dev), engine=engine).cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        assert tpcca.tpc_tf_status(tr.handle, 0) == 0
    finally:
        tr.close()
    total = float(want[0])  # b3 + sum of the positive products: the scale of the FP32 sum
    np.testing.assert_allclose(got, want, rtol=0, atol=2.0 ** -18 * total)


def test_score_and_pruned_mode_need_weights(env, c1):
    tpcca, dev = env
    tr = tpcca.TimeFrameTracker(c1.n + 16, mode=tpcca.TPC_MODE_PRUNED, tau=0.5)
    try:
        with pytest.raises(tpcca.TpcError):
            tr.track(*as_dev(torch, dev, c1.sector, c1.row, c1.pad, c1.time))
        with pytest.raises(tpcca.TpcError):
            tr.score(torch.zeros((4, 12), device=dev))
        with pytest.raises(tpcca.TpcError):
            tr.load_mlp(b"TPCM" + bytes(100))
    finally:
        tr.close()


# ------------------------------------------------------------------ pruned tracking
def _tau_in_gap(blob, feat, lo=0.3, hi=0.7, gap=4e-3):
    """A threshold whose band holds no oracle score of the frame."""
    sc = np.sort(1.0 / (1.0 + np.exp(-orc.mlp_logits(blob, feat))))
    sc = sc[(sc > lo - gap) & (sc < hi + gap)]
    edges = np.concatenate([[lo], sc, [hi]])
    k = int(np.argmax(np.diff(edges)))
    assert edges[k + 1] - edges[k] > gap, "no free threshold"
    return float(0.5 * (edges[k] + edges[k + 1]))


def _pruned_gpu(tpcca, dev, f, blob, tau, **kw):
    tr = tpcca.TimeFrameTracker(f.n + 16, mode=tpcca.TPC_MODE_PRUNED, tau=tau, **kw)
    try:
        tr.load_mlp(blob)
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time)
        g["n_pruned"] = tr.pruned_clusters()
    finally:
        tr.close()
    return g


@pytest.mark.parametrize("row_cap,engine", [(0, 0), (0, 1), (16, 0)])
def test_pruned_c1_full_parity(env, c1, row_cap, engine):
    """row_cap 0: windows staged, the pairs rescored from the tiles' regions, packed into
    dense rows for the dense scorer (engine 0: tcgen05 tiles of 128 rows, 1: mma.sync
    tiles of 16); row_cap 16: windows read from global memory, rescoring by the
    separate list kernel."""
    tpcca, dev = env
    blob = _net()
    feat, _, _ = orc.training_triplets(c1.sector, c1.row, c1.pad, c1.time)
    tau = _tau_in_gap(blob, feat)
    o = orc.track(c1.sector, c1.row, c1.pad, c1.time, mlp=blob, tau=tau)
    assert not o["band"].any()
    assert o["stats"][2] > 0, "the classifier changes some choices"
    g = _pruned_gpu(tpcca, dev, c1, blob, tau, row_cap=row_cap, mlp_engine=engine)
    assert g["n_pruned"] == o["stats"][0]
    compare_links(g, o)
    compare_tracks(g, o)


@pytest.mark.parametrize("tau", [0.0, 1.5])
def test_pruned_extremes_equal_plain(env, c1, tau):
    tpcca, dev = env
    blob = _net()
    plain = orc.track(c1.sector, c1.row, c1.pad, c1.time)
    g = _pruned_gpu(tpcca, dev, c1, blob, tau)
    compare_links(g, plain)
    compare_tracks(g, plain)


@pytest.mark.parametrize("engine", [0, 1])
def test_pruned_links_outside_band_two_sectors(env, two_sectors, engine):
    tpcca, dev = env
    f = two_sectors
    blob = _net(5)
    tau = 0.5
    o = orc.track(f.sector, f.row, f.pad, f.time, mlp=blob, tau=tau)
    g = _pruned_gpu(tpcca, dev, f, blob, tau, mlp_engine=engine)
    assert o["stats"][0] > 1000 and o["stats"][2] > 50
    assert g["n_pruned"] == o["stats"][0]
    assert np.array_equal(g["order"], o["order"])
    rows = f.row[o["order"]]
    mid = (rows > 0) & (rows < 151) & ~o["band"]
    assert np.array_equal(g["down"][mid], o["down"][mid])
    assert np.array_equal(g["up"][mid], o["up"][mid])
    # the band is a small share of the scored clusters
    assert o["band"].sum() <= max(5, 0.01 * o["stats"][0])
    if not o["band"].any():
        compare_links(g, o)
        compare_tracks(g, o)


# ------------------------------------------------------------------ training
def _rows(f, n=None):
    feat, lab, _ = orc.training_triplets(f.sector, f.row, f.pad, f.time)
    return (feat, lab) if n is None else (feat[:n], lab[:n])


@pytest.mark.parametrize("engine", [0, 1])  # tcgen05 (tensor memory), mma.sync
def test_gradient_matches_fp64_oracle(env, two_sectors, engine):
    tpcca, dev = env
    # 1000 rows: 15 groups of 64 (mma.sync) or 7 tiles of 128 (tcgen05) and a ragged tail
    feat, lab = _rows(two_sectors, 1000)
    mean, inv_std, theta = random_net(11, feature_scale=True)
    blob = orc.mlp_blob(mean, inv_std, theta)
    pw = 1.8
    loss_o, grad_o = orc.mlp_loss_grad(theta, mean, inv_std, feat, lab, pos_weight=pw)
    tr = tpcca.Trainer(blob, pos_weight=pw, max_batch=4096, engine=engine)
    try:
        F, L = _dev_tensor(feat, dev), _dev_tensor(lab, dev)
        grad_g, loss_g = tr.gradient(F, L)
        again, loss_again = tr.gradient(F, L)
        assert torch.equal(grad_g, again) and loss_g == loss_again  # bitwise reproducible
    finally:
        tr.close()
    grad_g = grad_g.cpu().numpy().astype(np.float64)
    assert abs(loss_g - loss_o) <= 2e-3 * abs(loss_o)
    off = 0
    for name, shape in tpcca.MLP_PARAM_SHAPES:
        k = int(np.prod(shape))
        a, b = grad_g[off:off + k], grad_o[off:off + k]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        assert rel <= 2e-2, f"{name}: relative gradient error {rel:.3g}"
        # element by element: BF16 operands (inputs, weights, the first hidden layer
        # and the back-propagated errors, each 2^-8 relative) move an entry by a few
        # BF16 steps of the terms it sums, which cancel more in small entries: the
        # bound is a floor of 2^-4 of the group's RMS plus 2^-4 of the entry itself
        # (the largest entry seen on this batch reached about half of it); a wrong
        # entry (another row's or column's sum, a dropped term) exceeds it
        floor = 2.0 ** -4 * np.sqrt(np.mean(b * b)) + 1e-12
        excess = np.abs(a - b) / (floor + 2.0 ** -4 * np.abs(b))
        assert excess.max() <= 1.0, f"{name}: entry {int(excess.argmax())} off by {excess.max():.3g} of its bound"
        if k > 1:  # a planted mistake in the oracle's copy (two entries swapped) breaks the bound
            w = b.copy()
            i0, i1 = int(np.argmax(np.abs(b))), int(np.argmin(np.abs(b)))
            w[[i0, i1]] = w[[i1, i0]]
            assert (np.abs(a - w) / (floor + 2.0 ** -4 * np.abs(w))).max() > 1.0, name
        off += k


@pytest.mark.parametrize("engine", [0, 1])
def test_gradient_with_index_gather(env, c1, engine):
    tpcca, dev = env
    feat, lab = _rows(c1)
    idx = np.random.default_rng(2).permutation(feat.shape[0])[:200].astype(np.int32)
    mean, inv_std, theta = random_net(12, feature_scale=True)
    blob = orc.mlp_blob(mean, inv_std, theta)
    tr = tpcca.Trainer(blob, engine=engine)
    try:
        g1, l1 = tr.gradient(_dev_tensor(feat, dev), _dev_tensor(lab, dev), _dev_tensor(idx, dev))
        g2, l2 = tr.gradient(_dev_tensor(feat[idx], dev), _dev_tensor(lab[idx], dev))
    finally:
        tr.close()
    assert torch.equal(g1, g2) and l1 == l2


@pytest.mark.parametrize("engine", [0, 1])
def test_first_adam_step_closed_form(env, c1, engine):
    tpcca, dev = env
    feat, lab = _rows(c1)
    mean, inv_std, theta = random_net(13, feature_scale=True)
    blob = orc.mlp_blob(mean, inv_std, theta)
    lr = 1e-3
    tr = tpcca.Trainer(blob, lr=lr, engine=engine)
    try:
        F, L = _dev_tensor(feat, dev), _dev_tensor(lab, dev)
        g, _ = tr.gradient(F, L)
        tr.step(F, L)
        _, _, theta1 = tpcca.unpack_blob(tr.blob())
    finally:
        tr.close()
    g = g.cpu().numpy().astype(np.float64)
    # step 1: bias-corrected moments are g and g^2, so the step is lr * g / (|g| + eps)
    want = theta.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(theta1, want, rtol=0, atol=1e-6 * lr + 1e-7)


def test_training_lowers_the_loss_and_normalises(env, two_sectors):
    tpcca, dev = env
    feat, lab = _rows(two_sectors)
    F, L = _dev_tensor(feat, dev), _dev_tensor(lab, dev)
    npos = int(lab.sum())
    tr = tpcca.Trainer(tpcca.init_blob(1), pos_weight=(lab.size - npos) / max(npos, 1), max_batch=1024)
    try:
        tr.normalise(F)
        mean, inv_std, _ = tpcca.unpack_blob(tr.blob())
        ref_mean = feat.astype(np.float64).mean(0)
        ref_std = feat.astype(np.float64).std(0)
        assert np.allclose(mean, ref_mean, rtol=1e-5, atol=1e-6)
        assert np.allclose(1.0 / inv_std, ref_std, rtol=1e-4)
        gen = torch.Generator(device=dev).manual_seed(0)
        losses = []
        for ep in range(20):
            perm = torch.randperm(feat.shape[0], device=dev, generator=gen).to(torch.int32)
            for b0 in range(0, feat.shape[0] - 1023, 1024):
                losses.append(float(tr.step(F, L, perm[b0:b0 + 1024]).item()))
    finally:
        tr.close()
    first, last = np.mean(losses[:5]), np.mean(losses[-5:])
    assert last < 0.8 * first, (first, last)
