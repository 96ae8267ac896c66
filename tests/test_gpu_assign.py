"""cluster_track from the per-row assignment pass on rows longer than its
shared-memory buffer (12288 clusters, built in chunks), against the oracle: one
sector of a 20 ms frame at 80 kHz (the validated time range ends at 131072 bins),
up to ~19 k clusters per row.  The persistent launch
(which assigns straight into global memory, no buffer) is checked on the same
input."""
import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import compare_links, compare_tracks, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ASSIGN_CAP = 12288  # clusters of a row the assignment kernel builds in shared memory at once


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def dense_sector():
    c = ts.continuous(20.0, 17)
    c.rate_khz = 80.0
    c.sector_only = 0
    f = ts.generate(c)
    per_row = np.bincount(f.row.astype(np.int64), minlength=152)
    assert per_row.max() > ASSIGN_CAP, "the case must take the chunked path"
    return f, orc.track(f.sector, f.row, f.pad, f.time)


@pytest.mark.parametrize("persistent", [0, 1])
def test_long_rows_match_the_oracle(env, dense_sector, persistent):
    tpcca, dev = env
    f, o = dense_sector
    tr = tpcca.TimeFrameTracker(f.n + 16, persistent=persistent)
    try:
        g = run_gpu(tr, torch, dev, f.sector, f.row, f.pad, f.time)
    finally:
        tr.close()
    compare_links(g, o)
    compare_tracks(g, o)
