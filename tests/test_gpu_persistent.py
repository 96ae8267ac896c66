"""The persistent launch (tpc_tf_config.persistent): the plain path A0-A5 as one
kernel whose stages are separated by bounded grid-wide barriers.  It runs the
same stage code as the one-launch-per-stage path, so its results must be the
oracle's (links, starts, assignment bit for bit; fits within the usual
tolerance) and identical to the stage launches' on a batched call, also when
replayed from a CUDA graph."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import as_dev, compare_links, compare_tracks, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


@pytest.mark.parametrize("tile", [512, 768, 1024])
def test_persistent_matches_oracle_one_sector(env, tile):
    tpcca, dev = env
    f = ts.generate(ts.c1())
    tr = tpcca.TimeFrameTracker(f.n + 16, persistent=1, nb_tile=tile)
    try:
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time)
        assert tr.launches_per_call() == 2  # the counters' reset and one kernel
    finally:
        tr.close()
    o = orc.track(f.sector, f.row, f.pad, f.time)
    compare_links(g, o)
    compare_tracks(g, o)


def test_persistent_unsorted_pileup_slice(env):
    """Three sectors of a 2 ms frame, shuffled: the sort runs first, then the
    persistent launch."""
    tpcca, dev = env
    f = ts.generate(ts.c2())
    m = np.nonzero(f.sector < 3)[0]
    perm = np.random.default_rng(4).permutation(m.size)
    s, r, p, t = f.sector[m][perm], f.row[m][perm], f.pad[m][perm], f.time[m][perm]
    tr = tpcca.TimeFrameTracker(m.size + 16, persistent=1)
    try:
        g = run_gpu(tr, torch, dev, s, r, p, t, sorted_input=False)
    finally:
        tr.close()
    o = orc.track(s, r, p, t)
    compare_links(g, o)
    compare_tracks(g, o)


def test_persistent_batched_graph_equals_stage_launches(env):
    tpcca, dev = env
    b = ts.batched(40, seed=7, n_min=2e3, n_max=6e4, ms_min=0.2, ms_max=2.0)
    f, off = b.frame, b.offsets
    n_inst = off.size - 1
    ref = tpcca.TimeFrameTracker(f.n + 16, n_sectors=n_inst)
    try:
        want = run_gpu(ref, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
    finally:
        ref.close()
    tr = tpcca.TimeFrameTracker(f.n + 16, n_sectors=n_inst, persistent=1)
    try:
        got = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time, debug=False)
        for k in ("cluster_track", "n_tracks", "nhits", "first_cluster", "sector", "status", "params", "cov", "chi2"):
            assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), k
        s, r, p, t = as_dev(torch, dev, f.sector, f.row, f.pad, f.time)
        cap = max(16, f.n // 10 + 1)
        for _ in range(3):  # graph replay of the two nodes
            tr._out["cluster_track"].fill_(-7)
            nt = tr.track_graph(s, r, p, t, capacity=cap)
            torch.cuda.synchronize()
            assert tpcca.tpc_tf_status(tr.handle, 0) == 0
            assert int(nt.item()) == want["n_tracks"]
            assert np.array_equal(tr._out["cluster_track"][:f.n].cpu().numpy(), want["cluster_track"])
    finally:
        tr.close()


def test_persistent_needs_plain_without_following(env):
    tpcca, dev = env
    for kw in (dict(mode=tpcca.TPC_MODE_PRUNED), dict(follow=1)):
        with pytest.raises(tpcca.TpcError) as ei:
            tpcca.TimeFrameTracker(1000, persistent=1, **kw)
        assert ei.value.code == tpcca.TPC_ERR_ARG
