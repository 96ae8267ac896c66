"""Batched calls (many sector x time-frame instances in one call, one launch per
stage), CUDA-graph replay and the autotuner, through the C ABI on the GPU.

A batched call gives every instance its own sector id; each instance must get
exactly the oracle's result for that instance alone (the instances share no
clusters, so the path treats them as independent sectors).  Graph replay and
every tile choice of the autotuner must reproduce the direct call bit for bit."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import FLOORS, PARAM_RTOL, as_dev, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def batch():
    return ts.batched(40, seed=7, n_min=2e3, n_max=6e4, ms_min=0.2, ms_max=2.0)


def _outputs(g):
    return {k: g[k] for k in ("cluster_track", "params", "cov", "chi2", "ndf", "nhits", "first_cluster", "sector",
                              "row_first", "row_last", "status", "n_tracks", "down", "up", "mup")}


def _same(g1, g2):
    for k, v in _outputs(g1).items():
        w = g2[k]
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, w), k
        else:
            assert v == w, k


def test_batched_call_equals_oracle_per_instance(env, batch):
    tpcca, dev = env
    f, off = batch.frame, batch.offsets
    n_inst = off.size - 1
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=n_inst)
    try:
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
    finally:
        tr.close()
    ct = g["cluster_track"]
    first_id = 0
    checked = 0
    for k in range(n_inst):
        a, b = off[k], off[k + 1]
        o = orc.track(np.zeros(b - a, np.uint16), f.row[a:b], f.pad[a:b], f.time[a:b])
        nt = o["n_tracks"]
        got = ct[a:b]
        want = np.where(o["cluster_track"] >= 0, o["cluster_track"] + first_id, -1)
        assert np.array_equal(got, want), f"instance {k}"
        sl = slice(first_id, first_id + nt)
        assert np.array_equal(g["sector"][sl].astype(np.int64), np.full(nt, k))
        assert np.array_equal(g["nhits"][sl], o["tracks"]["nhits"])
        assert np.array_equal(g["first_cluster"][sl], o["tracks"]["first_cluster"] + a)
        dp = np.abs(g["params"][sl].astype(np.float64) - o["tracks"]["p"])
        assert np.all(dp <= PARAM_RTOL * np.maximum(np.abs(o["tracks"]["p"]), FLOORS))
        first_id += nt
        checked += nt
    assert g["n_tracks"] == first_id and checked > 100


@pytest.mark.parametrize("mode", ["plain", "pruned"])
def test_tile_variants_give_identical_results(env, mode):
    tpcca, dev = env
    f = ts.generate(ts.c2())
    m = f.sector < 3
    s, r, p, t = f.sector[m], f.row[m], f.pad[m], f.time[m]
    kw = {}
    blob = None
    if mode == "pruned":
        import json
        import os
        w = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2102_08862_gb300",
                         "weights", "link_classifier")
        blob = open(w + ".bin", "rb").read()
        kw = dict(mode=tpcca.TPC_MODE_PRUNED, tau=json.load(open(w + ".json"))["tau"])
    res = {}
    for tile in (512, 768, 1024):
        tr = tpcca.TimeFrameTracker(int(m.sum()) + 16, nb_tile=tile, **kw)
        try:
            if blob:
                tr.load_mlp(blob)
            res[tile] = run_gpu(tr, torch, dev, s, r, p, t)
        finally:
            tr.close()
    _same(res[512], res[768])
    _same(res[1024], res[768])


def test_graph_replay_equals_direct_call_and_reads_new_inputs(env, batch):
    tpcca, dev = env
    f, off = batch.frame, batch.offsets
    n_inst = off.size - 1
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=n_inst)
    try:
        direct = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
        s, r, p, t = as_dev(torch, dev, f.sector, f.row, f.pad, f.time)
        cap = max(16, f.n // 10 + 1)
        for _ in range(3):
            tr._out["cluster_track"].fill_(-7)
            nt = tr.track_graph(s, r, p, t, capacity=cap)
            torch.cuda.synchronize()
            assert tpcca.tpc_tf_status(tr.handle, 0) == 0
            assert int(nt.item()) == direct["n_tracks"]
            assert np.array_equal(tr._out["cluster_track"][:f.n].cpu().numpy(), direct["cluster_track"])
            m = direct["n_tracks"]
            assert np.array_equal(tr._out["params"][:m].cpu().numpy(), direct["params"][:m])
        # new data in the same buffers: the graph reads it at launch time
        t2 = t.clone()
        t.add_(0.25)
        tr.track_graph(s, r, p, t, capacity=cap)
        torch.cuda.synchronize()
        ct_graph = tr._out["cluster_track"][:f.n].cpu().numpy().copy()
        shifted = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, (t2 + 0.25).cpu().numpy(), debug=False)
        assert np.array_equal(ct_graph, shifted["cluster_track"])
    finally:
        tr.close()


def test_autotuner_choice_is_valid_and_kept(env, batch):
    tpcca, dev = env
    f, off = batch.frame, batch.offsets
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=off.size - 1)
    try:
        before = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
        tile, fit = tr.autotune(*as_dev(torch, dev, f.sector, f.row, f.pad, f.time), trials=2)
        assert tile in (512, 768, 1024) and fit in (tpcca.TPC_FIT_THREAD, tpcca.TPC_FIT_WARP)
        after = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
        assert np.array_equal(before["cluster_track"], after["cluster_track"])
        with pytest.raises(tpcca.TpcError):
            tr.autotune(*as_dev(torch, dev, f.sector, f.row, f.pad, f.time), trials=0)
    finally:
        tr.close()


def test_many_sectors_need_sorted_input(env, batch):
    tpcca, dev = env
    f = batch.frame
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=40)
    try:
        with pytest.raises(tpcca.TpcError):
            tr.track(*as_dev(torch, dev, f.sector, f.row, f.pad, f.time), sorted_input=False)
    finally:
        tr.close()
