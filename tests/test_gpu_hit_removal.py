"""Hit removal (compression: keep only the clusters attached to tracks) through the
C ABI: the kept clusters, in input order, and their track ids must equal the
selection written out from the oracle's cluster -> track assignment, byte for byte."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import as_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


def _frames():
    c1 = ts.generate(ts.c1())
    f = ts.generate(ts.c2())
    m = f.sector < 2
    return [(c1.sector, c1.row, c1.pad, c1.time), (f.sector[m], f.row[m], f.pad[m], f.time[m])]


@pytest.mark.parametrize("which", [0, 1])
def test_removal_keeps_tracked_clusters_in_order(env, which):
    tpcca, dev = env
    s, r, p, t = _frames()[which]
    perm = np.random.default_rng(which).permutation(s.size)  # caller order is not the sorted order
    s, r, p, t = s[perm], r[perm], p[perm], t[perm]
    o = orc.track(s, r, p, t)
    tr = tpcca.TimeFrameTracker(s.size + 16)
    try:
        ds, dr, dp, dt = as_dev(torch, dev, s, r, p, t)
        res = tr.track(ds, dr, dp, dt, sorted_input=False)
        ct = res.cluster_track
        assert np.array_equal(ct.cpu().numpy(), o["cluster_track"])
        kept = tr.remove_unassigned(ds, dr, dp, dt, ct)
    finally:
        tr.close()
    mask = o["cluster_track"] >= 0
    assert 0 < mask.sum() < s.size
    assert np.array_equal(kept["sector"].cpu().numpy().view(np.uint16), s[mask])
    assert np.array_equal(kept["row"].cpu().numpy().view(np.uint16), r[mask])
    assert np.array_equal(kept["pad"].cpu().numpy().view(np.uint32), p[mask].view(np.uint32))
    assert np.array_equal(kept["time"].cpu().numpy().view(np.uint32), t[mask].view(np.uint32))
    assert np.array_equal(kept["track"].cpu().numpy(), o["cluster_track"][mask])


def test_removal_of_an_empty_frame(env):
    tpcca, dev = env
    tr = tpcca.TimeFrameTracker(16)
    try:
        z = lambda dt: torch.zeros(0, dtype=dt, device=dev)
        kept = tr.remove_unassigned(z(torch.int16), z(torch.int16), z(torch.float32), z(torch.float32),
                                    z(torch.int32))
        assert kept["sector"].numel() == 0
    finally:
        tr.close()
