"""What the trained link classifier gains over the plain CA, on a held-out 2 ms
Pb-Pb-like frame (seed 1060: neither a training frame, 1001-1050, nor a
threshold frame, 1051-1052).  Both runs go through the C ABI on the GPU; the
rates are the oracle's evaluation against generator truth.  Requirement: the
pruned efficiency stays within 0.5 % (absolute) of the plain one; the gain is
fewer clones (a clone is a second track on the same findable particle, which
the plain rule makes where a chain breaks)."""
import json
import os

import numpy as np
import pytest

import oracle as orc
import tpcsynth as ts
from gpu_util import as_dev

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


def _quality(tpcca, dev, f, **kw):
    tr = tpcca.TimeFrameTracker(f.n + 16, **kw)
    try:
        if kw.get("mode") == tpcca.TPC_MODE_PRUNED:
            tr.load_mlp(open(WEIGHTS + ".bin", "rb").read())
        res = tr.track(*as_dev(torch, dev, f.sector, f.row, f.pad, f.time))
        ct = res.cluster_track.cpu().numpy()
        return orc.evaluate(f.label, f.sector, ct, res.n_tracks, f.trk_qpt.shape[0])
    finally:
        tr.close()


def test_trained_classifier_gain_on_held_out_frame(env):
    tpcca, dev = env
    tau = json.load(open(WEIGHTS + ".json"))["tau"]
    f = ts.generate(ts.continuous(2.0, 1060))
    plain = _quality(tpcca, dev, f)
    pruned = _quality(tpcca, dev, f, mode=tpcca.TPC_MODE_PRUNED, tau=tau)
    print("\nplain ", {k: round(plain[k], 6) for k in ("efficiency", "clone_rate", "fake_rate")},
          "\npruned", {k: round(pruned[k], 6) for k in ("efficiency", "clone_rate", "fake_rate")}, f"tau {tau}")
    assert plain["n_findable"] > 50000
    assert pruned["efficiency"] >= plain["efficiency"] - 0.005
    assert pruned["clone_rate"] < plain["clone_rate"]
    assert pruned["fake_rate"] <= plain["fake_rate"] + 0.001
