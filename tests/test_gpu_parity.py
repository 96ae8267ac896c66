"""GPU parity of the CUDA path (through the C ABI) with the CPU oracle.

Links, start hits and the cluster -> track assignment must match bit for bit;
fitted parameters within 1e-4 relative (floors 1 cm, 1 cm, 0.01, 0.01, 0.1 c/GeV),
covariances within 1e-3 (floor 1e-3 sqrt(C_ii C_jj)), FP32 against FP64."""
import ctypes

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import compare_links, compare_tracks, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build
    _build.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def tracker(dev):
    from paper_2102_08862_gb300 import tpcca
    tr = tpcca.TimeFrameTracker(8_000_000)
    yield tr
    tr.close()


@pytest.fixture(scope="module")
def c1():
    return ts.generate(ts.c1())


def _oracle(f, perm=None):
    if perm is None:
        return orc.track(f.sector, f.row, f.pad, f.time)
    return orc.track(f.sector[perm], f.row[perm], f.pad[perm], f.time[perm])


def test_c1_parity(dev, tracker, c1):
    g = run_gpu(tracker, torch, dev, c1.sector, c1.row, c1.pad, c1.time)
    o = _oracle(c1)
    assert o["n_tracks"] > 50
    compare_links(g, o)
    compare_tracks(g, o)


def test_c1_unsorted_input(dev, tracker, c1):
    perm = np.random.default_rng(9).permutation(c1.n)
    g = run_gpu(tracker, torch, dev, c1.sector[perm], c1.row[perm], c1.pad[perm], c1.time[perm], sorted_input=False)
    o = _oracle(c1, perm)
    compare_links(g, o)
    compare_tracks(g, o)


def test_pileup_sector_parity(dev, tracker):
    """One sector of a 2 ms frame with ~100 piled-up collisions: rows of ~1000
    clusters span several tiles of every kernel and end in ragged tails."""
    cfg = ts.c2(seed=12)
    cfg.sector_only = 7
    f = ts.generate(cfg)
    g = run_gpu(tracker, torch, dev, f.sector, f.row, f.pad, f.time)
    o = _oracle(f)
    compare_links(g, o)
    compare_tracks(g, o)


def test_global_memory_kernel_parity(dev, c1):
    """Rows larger than the staged-row capacity take the global-memory kernel."""
    from paper_2102_08862_gb300 import tpcca
    tr = tpcca.TimeFrameTracker(200_000, row_cap=16)
    try:
        g = run_gpu(tr, torch, dev, c1.sector, c1.row, c1.pad, c1.time)
        o = _oracle(c1)
        compare_links(g, o)
        compare_tracks(g, o)
    finally:
        tr.close()


def test_unaligned_input_parity(dev, tracker, c1):
    """Cluster arrays that start 4 bytes past a 16-byte boundary (element-aligned
    only) give the same result: staging may not assume vector alignment."""
    n = c1.n
    s, r, p, t = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
                  (c1.sector.view(np.int16), c1.row.view(np.int16), c1.pad, c1.time))
    pad_buf = torch.empty(n + 1, dtype=torch.float32, device=dev)
    time_buf = torch.empty(n + 1, dtype=torch.float32, device=dev)
    pad_buf[1:] = p
    time_buf[1:] = t
    res = tracker.track(s, r, pad_buf[1:], time_buf[1:])
    o = _oracle(c1)
    assert np.array_equal(res.cluster_track.cpu().numpy(), o["cluster_track"])
    assert res.n_tracks == o["n_tracks"]


@pytest.mark.parametrize("fit_variant", [0, 1])
def test_fit_variants(dev, c1, fit_variant):
    from paper_2102_08862_gb300 import tpcca
    tr = tpcca.TimeFrameTracker(200_000, fit_variant=fit_variant)
    try:
        g = run_gpu(tr, torch, dev, c1.sector, c1.row, c1.pad, c1.time)
        compare_tracks(g, _oracle(c1))
    finally:
        tr.close()


def test_edge_cases(dev, tracker):
    # empty frame
    e = np.zeros(0)
    g = run_gpu(tracker, torch, dev, e, e, e, e, debug=False)
    assert g["n_tracks"] == 0
    # one cluster
    g = run_gpu(tracker, torch, dev, [3], [75], [10.0], [100.0])
    assert g["n_tracks"] == 0 and g["cluster_track"][0] == -1 and g["down"][0] == -1
    # one straight chain through all rows of sector 35 and rows 0/151 only elsewhere
    rows = np.arange(152)
    sec = np.full(152, 35)
    pad = 0.5 * (66 + (144 * rows + 151) // 302 - 1) + 0.25   # 0.25 pad off the centre line
    tim = 300.0 - 0.5 * rows
    sec = np.concatenate([[0, 0], sec])
    rows = np.concatenate([[0, 151], rows])
    pad = np.concatenate([[5.0, 5.0], pad])
    tim = np.concatenate([[1.0, 1.0], tim])
    o = orc.track(sec, rows, pad, tim)
    order = o["order"]
    g = run_gpu(tracker, torch, dev, sec[order], rows[order], pad[order], tim[order])
    o = orc.track(sec[order], rows[order], pad[order], tim[order])
    compare_links(g, o)
    compare_tracks(g, o)
    assert g["n_tracks"] == 1 and g["nhits"][0] == 152


@pytest.mark.parametrize("length", [11, 12, 13])
def test_chain_length_threshold(dev, tracker, length):
    rows = np.arange(40, 40 + length)
    pad = np.full(length, 50.0) + 0.1 * np.arange(length)
    tim = 1000.0 + 0.3 * np.arange(length)
    sec = np.full(length, 4)
    g = run_gpu(tracker, torch, dev, sec, rows, pad, tim)
    o = orc.track(sec, rows, pad, tim)
    compare_links(g, o)
    compare_tracks(g, o)
    # the end clusters of a chain away from rows 0/151 are not linked (A1 needs both neighbours)
    assert g["n_tracks"] == (1 if length - 2 >= 10 else 0)


def test_invalid_input_is_reported_and_context_survives(dev, tracker, c1):
    from paper_2102_08862_gb300 import tpcca
    bad_pad = c1.pad.copy()
    bad_pad[len(bad_pad) // 2] = np.nan
    with pytest.raises(tpcca.TpcError) as ei:
        run_gpu(tracker, torch, dev, c1.sector, c1.row, bad_pad, c1.time, debug=False)
    assert ei.value.code == tpcca.TPC_ERR_INPUT
    bad_sec = c1.sector.copy()
    bad_sec[-1] = 40
    with pytest.raises(tpcca.TpcError) as ei:
        run_gpu(tracker, torch, dev, bad_sec, c1.row, c1.pad, c1.time, debug=False)
    assert ei.value.code == tpcca.TPC_ERR_INPUT
    # flagged as sorted but not sorted by time
    swapped = c1.time.copy()
    swapped[[10, 11]] = swapped[[11, 10]]
    if swapped[10] != swapped[11]:
        with pytest.raises(tpcca.TpcError) as ei:
            run_gpu(tracker, torch, dev, c1.sector, c1.row, c1.pad, swapped, debug=False)
        assert ei.value.code == tpcca.TPC_ERR_INPUT
    # the context is intact: a valid call still matches the oracle
    g = run_gpu(tracker, torch, dev, c1.sector, c1.row, c1.pad, c1.time)
    compare_tracks(g, _oracle(c1))


def test_capacity_errors(dev, c1):
    from paper_2102_08862_gb300 import tpcca
    tr = tpcca.TimeFrameTracker(c1.n)
    try:
        o = _oracle(c1)
        with pytest.raises(tpcca.TpcError) as ei:
            run_gpu(tr, torch, dev, c1.sector, c1.row, c1.pad, c1.time, capacity=5, debug=False)
        assert ei.value.code == tpcca.TPC_ERR_CAPACITY
        # the assignment is still complete and the count is the required one
        assert int(tr._out["n_tracks"][0].item()) == o["n_tracks"]
        assert np.array_equal(tr._out["cluster_track"][:c1.n].cpu().numpy(), o["cluster_track"])
    finally:
        tr.close()
    small = tpcca.TimeFrameTracker(100)
    try:
        with pytest.raises(tpcca.TpcError) as ei:
            run_gpu(small, torch, dev, c1.sector, c1.row, c1.pad, c1.time, debug=False)
        assert ei.value.code == tpcca.TPC_ERR_CAPACITY
    finally:
        small.close()


def test_host_entry_point_matches_device_path(dev, tracker, c1):
    from paper_2102_08862_gb300 import tpcca
    o = _oracle(c1)
    n = c1.n
    cap = 4096
    ct = np.zeros(n, np.int32)
    arrs = dict(params=np.zeros((cap, 5), np.float32), cov=np.zeros((cap, 15), np.float32),
                t_ref=np.zeros(cap, np.float32), x=np.zeros(cap, np.float32), chi2=np.zeros(cap, np.float32),
                ndf=np.zeros(cap, np.int32), nhits=np.zeros(cap, np.int32), first_cluster=np.zeros(cap, np.int32),
                sector=np.zeros(cap, np.uint16), row_first=np.zeros(cap, np.uint16),
                row_last=np.zeros(cap, np.uint16), status=np.zeros(cap, np.uint8))
    nt = np.zeros(1, np.uint32)
    ptr = lambda a: a.ctypes.data
    sec, row = np.ascontiguousarray(c1.sector), np.ascontiguousarray(c1.row)
    pad, tim = np.ascontiguousarray(c1.pad), np.ascontiguousarray(c1.time)
    cl = tpcca.tpc_clusters(n=n, flags=tpcca.TPC_INPUT_SORTED, sector=ptr(sec), row=ptr(row), pad=ptr(pad),
                            time=ptr(tim))
    tr = tpcca.tpc_tracks(cluster_track=ptr(ct), track_capacity=cap, n_tracks=ptr(nt),
                          **{k: ptr(v) for k, v in arrs.items()})
    rc = tpcca.tpc_track_timeframe_host(tracker.handle, cl, tr, 0)
    assert rc == tpcca.TPC_OK, tpcca.tpc_last_error()
    g = dict(arrs)
    g["cluster_track"] = ct
    g["n_tracks"] = int(nt[0])
    compare_tracks(g, o)


@pytest.mark.parametrize("mode", ["plain", "pruned"])
def test_host_entry_point_pipelined_over_sector_ranges(dev, mode):
    """A frame of more than 4M sorted clusters through the host-buffer entry point:
    in page-locked buffers it is copied in and tracked as sector ranges (a range
    copied while the previous one is tracked), in pageable ones in one piece; both
    results must be the device path's, byte for byte."""
    import json
    import os
    from paper_2102_08862_gb300 import tpcca
    f = ts.generate(ts.c2())
    assert f.n >= 1 << 22
    kw = {}
    blob = None
    if mode == "pruned":
        w = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2102_08862_gb300",
                         "weights", "link_classifier")
        blob = open(w + ".bin", "rb").read()
        kw = dict(mode=tpcca.TPC_MODE_PRUNED, tau=json.load(open(w + ".json"))["tau"])
    tr = tpcca.TimeFrameTracker(f.n + 16, **kw)
    try:
        if blob:
            tr.load_mlp(blob)
        cap = f.n // 10 + 1
        direct = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, capacity=cap, debug=False)
        for pinned in (True, True, False):
            host = tr.track_host(f.sector, f.row, f.pad, f.time, capacity=cap, pinned=pinned)
            assert host["n_tracks"] == direct["n_tracks"]
            assert np.array_equal(host["cluster_track"], direct["cluster_track"])
            m = direct["n_tracks"]
            for k in ("params", "cov", "t_ref", "x", "chi2", "ndf", "nhits", "first_cluster", "row_first",
                      "row_last", "status"):
                assert np.array_equal(host[k][:m], direct[k][:m]), k
            assert np.array_equal(host["sector"][:m].astype(np.int64), direct["sector"][:m].astype(np.int64))
        with pytest.raises(tpcca.TpcError) as ei:  # the capacity error and count survive the ranges
            tr.track_host(f.sector, f.row, f.pad, f.time, capacity=direct["n_tracks"] - 1, pinned=True)
        assert ei.value.code == tpcca.TPC_ERR_CAPACITY
        # no records wanted (capacity 0): the same assignment, the count still reported
        none = tr.track_host(f.sector, f.row, f.pad, f.time, capacity=0, pinned=True)
        assert none["n_tracks"] == direct["n_tracks"]
        assert np.array_equal(none["cluster_track"], direct["cluster_track"])
    finally:
        tr.close()


def test_repeated_calls_are_identical_and_allocate_nothing(dev, tracker, c1):
    s, r, p, t = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
                  (c1.sector.view(np.int16), c1.row.view(np.int16), c1.pad, c1.time))
    first = tracker.track(s, r, p, t).cluster_track.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        res = tracker.track(s, r, p, t)
        assert torch.equal(res.cluster_track, first)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_sector_shards_union_equals_whole_frame(dev, tracker):
    """Sectors are independent: tracking sector subsets in separate calls and
    gathering the results gives the whole-frame result (the multi-GPU shard)."""
    cfg = ts.c2(seed=31)
    cfg.frame_bins = 2000.0
    f = ts.generate(cfg)
    whole = run_gpu(tracker, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
    shards = [np.arange(0, 12), np.arange(12, 30), np.arange(30, 36)]
    ct = np.full(f.n, -1, np.int64)
    offset = 0
    firsts = []
    for secs in shards:
        idx = np.where(np.isin(f.sector, secs))[0]
        g = run_gpu(tracker, torch, dev, f.sector[idx], f.row[idx], f.pad[idx], f.time[idx], debug=False)
        c = g["cluster_track"].astype(np.int64)
        ct[idx] = np.where(c >= 0, c + offset, -1)
        firsts.append(idx[g["first_cluster"][:g["n_tracks"]]])
        offset += g["n_tracks"]
    assert offset == whole["n_tracks"]
    assert np.array_equal(ct, whole["cluster_track"])
    assert np.array_equal(np.concatenate(firsts), whole["first_cluster"][:offset])


@pytest.mark.slow
def test_c2_full_frame_parity(dev, tracker):
    f = ts.generate(ts.c2())
    g = run_gpu(tracker, torch, dev, f.sector, f.row, f.pad, f.time)
    o = _oracle(f)
    compare_links(g, o)
    compare_tracks(g, o)
    ev_g = orc.evaluate(f.label, f.sector, g["cluster_track"], g["n_tracks"], len(f.trk_qpt))
    ev_o = orc.evaluate(f.label, f.sector, o["cluster_track"], o["n_tracks"], len(f.trk_qpt))
    for k in ("efficiency", "clone_rate", "fake_rate"):
        assert abs(ev_g[k] - ev_o[k]) <= 1e-3


@pytest.mark.slow
def test_full_size_10ms_frame_sampled_sectors(dev):
    """The 10 ms frame (~32M clusters) as timed by the benchmark; the oracle
    recomputes two sectors (sectors are independent) and must agree exactly on
    their links and tracks."""
    from paper_2102_08862_gb300 import tpcca
    f = ts.generate(ts.c3())
    tr = tpcca.TimeFrameTracker(f.n)
    try:
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time)
    finally:
        tr.close()
    for secs in ([5], [27]):
        idx = np.where(np.isin(f.sector, secs))[0]
        o = orc.track(f.sector[idx], f.row[idx], f.pad[idx], f.time[idx])
        inv = np.full(f.n, -1, np.int64)
        inv[idx] = np.arange(len(idx))
        for k in ("down", "up", "mup"):
            full = g[k][idx]
            mapped = np.where(full >= 0, inv[np.maximum(full, 0)], -1)
            assert np.array_equal(mapped, o[k]), k
        assert np.array_equal(g["is_start"][idx], o["is_start"])
        # tracks of these sectors, matched by their start cluster
        sel = np.where(np.isin(g["sector"][:g["n_tracks"]], secs))[0]
        assert len(sel) == o["n_tracks"]
        sub = {k: g[k][sel] for k in ("params", "cov", "t_ref", "x", "chi2", "ndf", "nhits", "sector", "row_first",
                                       "row_last", "status")}
        sub["first_cluster"] = inv[g["first_cluster"][sel]]
        sub["n_tracks"] = len(sel)
        compare_tracks(sub, o, check_ct=False)
        ct = g["cluster_track"][idx]
        remap = np.full(g["n_tracks"], -1, np.int64)
        remap[sel] = np.arange(len(sel))
        assert np.array_equal(np.where(ct >= 0, remap[np.maximum(ct, 0)], -1), o["cluster_track"])
