"""The serving runtime (tpc_server_*) on the GPU: frames of differing length
submitted together run concurrently on several slots, and every result is the
same as the frame tracked alone through the library's direct entry point and as
the CPU oracle's assignment (exactly in plain mode; in pruned mode outside the
tracks touched by a classifier score within 1e-3 of tau, where FP32 and FP64 may
decide differently).  Also the memory budget (it limits the slots) and a request
no budget can hold."""
import json
import os
import time

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2102_08862_gb300",
                       "weights", "link_classifier")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def frames():
    fs = [ts.generate(ts.continuous(ms, seed)) for ms, seed in ((0.3, 21), (0.8, 22), (0.5, 23), (1.2, 24))]
    fs.append(ts.generate(ts.c1()))
    return fs


def _alone(tpcca, dev, f, **kw):
    blob = kw.pop("blob", None)
    tr = tpcca.TimeFrameTracker(f.n + 16, **kw)
    try:
        if blob:
            tr.load_mlp(blob)
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
    finally:
        tr.close()
    return g["cluster_track"], g["n_tracks"]


@pytest.mark.parametrize("mode", ["plain", "pruned"])
def test_results_equal_alone_and_in_the_mix(env, frames, mode):
    tpcca, dev = env
    kw, skw = {}, {}
    if mode == "pruned":
        blob = open(WEIGHTS + ".bin", "rb").read()
        tau = json.load(open(WEIGHTS + ".json"))["tau"]
        kw = dict(mode=tpcca.TPC_MODE_PRUNED, tau=tau, blob=blob)
        skw = dict(mode=tpcca.TPC_MODE_PRUNED, tau=tau)
    alone = [_alone(tpcca, dev, f, **dict(kw)) for f in frames]
    srv = tpcca.Server(max_slots=3, mlp_blob=kw.get("blob"), **skw)
    try:
        ids = {}
        for rep in range(2):  # every frame twice, all submitted before any result is read
            for k, f in enumerate(frames):
                ids[srv.submit(f.sector, f.row, f.pad, f.time)] = k
        got, slots = {}, set()
        deadline = time.time() + 120
        while len(got) < len(ids):
            assert time.time() < deadline, "server did not finish"
            for res, ct in srv.poll(wait_ms=2000):
                assert res["status"] == 0
                got[res["id"]] = (ct.copy(), res["n_tracks"])
                slots.add(res["slot"])
                assert res["t_submit"] <= res["t_start"] <= res["t_done"]
        assert len(slots) >= 2, "frames ran on several slots"
        for rid, k in ids.items():
            ct, nt = got[rid]
            assert nt == alone[k][1]
            assert np.array_equal(ct, alone[k][0])
        # every served frame against the oracle
        for k, f in enumerate(frames):
            ct = next(got[rid][0] for rid, kk in ids.items() if kk == k)
            if mode == "plain":
                ref = orc.track(f.sector, f.row, f.pad, f.time)
                assert np.array_equal(ct, ref["cluster_track"]), k
            else:
                ref = orc.track(f.sector, f.row, f.pad, f.time, mlp=kw["blob"], tau=tau)
                rct = ref["cluster_track"]
                band = ref["order"][np.nonzero(ref["band"])[0]]  # caller indices near the threshold
                excl = np.zeros(f.n, bool)
                for ids_ in (rct, ct):  # tracks that hold a band cluster, on either side
                    hit = np.unique(ids_[band][ids_[band] >= 0])
                    excl |= np.isin(ids_, hit)
                assert excl.mean() < 0.02, (k, excl.mean())
                if band.size == 0:
                    assert np.array_equal(ct, rct), k
                    continue
                # elsewhere the same partition into tracks (ids may shift by the tracks that differ)
                g, o = ct[~excl], rct[~excl]
                assert np.array_equal(g < 0, o < 0), k
                pairs = np.unique(np.stack([g[g >= 0], o[o >= 0]]), axis=1)
                assert np.unique(pairs[0]).size == pairs.shape[1] == np.unique(pairs[1]).size, k
        st = srv.stats()
        assert 2 <= st["slots"] <= 3 and st["queued"] == 0
    finally:
        srv.close()


def test_budget_limits_the_slots(env, frames):
    tpcca, dev = env
    cfg = tpcca.tpc_default_config()
    cfg.max_clusters = 1 << 20
    one = tpcca.tpc_tf_arena_bytes(cfg)
    small = [ts.generate(ts.c1(seed=s)) for s in (1, 2, 3)]  # ~8k clusters: 1 Mi-cluster slots
    srv = tpcca.Server(budget_bytes=int(one * 1.5), max_slots=4)  # room for a single such slot
    try:
        ids = [srv.submit(f.sector, f.row, f.pad, f.time) for f in small]
        done = []
        deadline = time.time() + 60
        while len(done) < len(ids):
            assert time.time() < deadline, "server did not finish"
            done += srv.poll(wait_ms=2000)
        assert all(r["status"] == 0 for r, _ in done)
        assert srv.stats()["slots"] == 1
        for (r, ct), f in zip(sorted(done, key=lambda x: x[0]["id"]), small):
            assert np.array_equal(ct, _alone(tpcca, dev, f)[0])
    finally:
        srv.close()


def test_request_larger_than_the_budget_fails(env, frames):
    tpcca, dev = env
    srv = tpcca.Server(budget_bytes=1 << 20, max_slots=2)  # 1 MiB: no slot fits
    try:
        f = frames[0]
        rid = srv.submit(f.sector, f.row, f.pad, f.time)
        res = srv.poll(wait_ms=5000)
        assert len(res) == 1 and res[0][0]["id"] == rid and res[0][0]["status"] == tpcca.TPC_ERR_CAPACITY
    finally:
        srv.close()
