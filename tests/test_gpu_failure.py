"""Failure path of the bounded device-side waits (the look-back of the ordered
compactions).  A test lowers the handle's spin limit to a few polls and enqueues
one look-back wait whose predecessor never publishes (a flag nothing sets): the
wait must give up, the handle must report TPC_ERR_TIMEOUT through its status
word, and the next tracking call on the same handle must match the oracle.
Nothing here faults or hangs the GPU: the wait is bounded and the kernel returns."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tpcca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca


def test_wait_gives_up_and_handle_survives(tpcca):
    dev = torch.device("cuda", 0)
    f = ts.generate(ts.c1())
    tr = tpcca.TimeFrameTracker(f.n + 16)
    try:
        assert tpcca.tpc_tf_set_spin_limit(tr.handle, 4) == tpcca.TPC_OK
        assert tpcca.tpc_tf_debug_wait(tr.handle, 0) == tpcca.TPC_OK, tpcca.tpc_last_error()
        assert tpcca.tpc_tf_status(tr.handle, 0) == tpcca.TPC_ERR_TIMEOUT
        assert "gave up" in tpcca.tpc_last_error()
        # the status word of a timed-out wait is cleared by the next call; with the
        # default limit restored the handle tracks as before
        assert tpcca.tpc_tf_set_spin_limit(tr.handle, 0) == tpcca.TPC_OK
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        res = tr.track(t(f.sector.view(np.int16)), t(f.row.view(np.int16)), t(f.pad), t(f.time))
        assert tpcca.tpc_tf_status(tr.handle, 0) == tpcca.TPC_OK
        ref = orc.track(f.sector, f.row, f.pad, f.time)
        assert res.n_tracks == ref["n_tracks"]
        assert np.array_equal(res.cluster_track.cpu().numpy(), ref["cluster_track"])
    finally:
        tr.close()
