"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare its outputs with the CPU oracle's."""
import numpy as np

FLOORS = np.array([1.0, 1.0, 0.01, 0.01, 0.1])  # cm, cm, -, -, c/GeV
PARAM_RTOL = 1e-4
COV_RTOL = 1e-3


def as_dev(torch, dev, f_sector, f_row, f_pad, f_time):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return (t(np.asarray(f_sector, np.uint16).view(np.int16)), t(np.asarray(f_row, np.uint16).view(np.int16)),
            t(np.asarray(f_pad, np.float32)), t(np.asarray(f_time, np.float32)))


def run_gpu(tracker, torch, dev, sector, row, pad, time, sorted_input=True, capacity=None, debug=True):
    s, r, p, t = as_dev(torch, dev, sector, row, pad, time)
    res = tracker.track(s, r, p, t, sorted_input=sorted_input, capacity=capacity)
    torch.cuda.synchronize()
    out = {k: getattr(res, k).cpu().numpy() for k in ("cluster_track", "params", "cov", "t_ref", "x", "chi2", "ndf",
                                                    "nhits", "first_cluster", "sector", "row_first", "row_last",
                                                    "status")}
    out["n_tracks"] = res.n_tracks
    if res.next_track is not None:
        out["next_track"] = res.next_track.cpu().numpy()
    if debug:
        dbg = tracker.debug_links()
        out.update({k: v.cpu().numpy() for k, v in dbg.items()})
        out["is_start"] = out["is_start"].astype(bool)
    return out


def compare_links(g, o):
    assert np.array_equal(g["order"], o["order"]), "sort order"
    assert np.array_equal(g["down"], o["down"]), "A1/A2 down links"
    assert np.array_equal(g["up"], o["up"]), "A1/A2 up links"
    assert np.array_equal(g["mup"], o["mup"]), "mutual links"
    assert np.array_equal(g["is_start"], o["is_start"]), "start hits"


def compare_tracks(g, o, check_ct=True):
    ot = o["tracks"]
    assert g["n_tracks"] == o["n_tracks"]
    if check_ct:
        assert np.array_equal(g["cluster_track"], o["cluster_track"]), "cluster -> track assignment"
    n = len(ot)
    for k in ("nhits", "first_cluster", "row_first", "row_last", "ndf", "status"):
        assert np.array_equal(g[k][:n].astype(np.int64), ot[k].astype(np.int64)), k
    assert np.array_equal(g["sector"][:n].astype(np.int64), ot["sector"].astype(np.int64))
    assert np.array_equal(g["t_ref"][:n], ot["t_ref"].astype(np.float32)), "t_ref is the start cluster's time"
    assert np.allclose(g["x"][:n], ot["x"], rtol=0, atol=1e-4)
    dp = np.abs(g["params"][:n].astype(np.float64) - ot["p"])
    lim = PARAM_RTOL * np.maximum(np.abs(ot["p"]), FLOORS)
    bad = dp > lim
    assert not bad.any(), f"{bad.sum()} parameters outside 1e-4: worst ratio {(dp / lim).max():.3g}"
    C = ot["C"]
    diag = C[:, [0, 2, 5, 9, 14]]
    ii, jj = np.tril_indices(5)
    scale = np.sqrt(diag[:, ii] * diag[:, jj])
    dc = np.abs(g["cov"][:n].astype(np.float64) - C)
    clim = COV_RTOL * np.maximum(np.abs(C), 1e-3 * scale)
    badc = dc > clim
    assert not badc.any(), f"{badc.sum()} covariance entries outside 1e-3: worst ratio {(dc / clim).max():.3g}"
    dchi = np.abs(g["chi2"][:n] - ot["chi2"])
    assert np.all(dchi <= 1e-3 * np.maximum(ot["chi2"], 1.0)), "chi2"
