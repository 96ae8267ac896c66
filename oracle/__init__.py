"""CPU oracle of the TPC track-finding path (plain C, single-threaded; FP64 fit,
fixed-point integer linking).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  The product
library never imports, links or executes anything here, and shares no code with
it.  ``oracle.c`` documents the steps and readings it implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NROWS = 152
NSECT = 36

TRACK_DTYPE = np.dtype([
    ("t_ref", "f8"), ("x", "f8"), ("p", "f8", (5,)), ("C", "f8", (15,)), ("chi2", "f8"),
    ("ndf", "i4"), ("nhits", "i4"), ("first_cluster", "i4"), ("sector", "i4"),
    ("row_first", "i4"), ("row_last", "i4"), ("status", "i4")], align=True)


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "mlp.c", "follow.c")]
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(p) for p in srcs + [hdr])):
        return _SO
    # -ffp-contract=off: every FP32 feature operation is rounded on its own
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", _SO + ".tmp", *srcs, "-lm"], check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("wy_q", ctypes.c_int32), ("wt_q", ctypes.c_int32),
                ("cost_max_q", ctypes.c_int64), ("n_min", ctypes.c_int32)]


class FollowParams(ctypes.Structure):
    _fields_ = [("chi2_max", ctypes.c_double), ("max_miss", ctypes.c_int32), ("join_check", ctypes.c_int32),
                ("links", ctypes.c_int32), ("xs_rows", ctypes.c_int32), ("chi2_link", ctypes.c_double)]


class EvalOut(ctypes.Structure):
    _fields_ = [("n_findable", ctypes.c_int64), ("n_findable_found", ctypes.c_int64),
                ("n_matched_findable_tracks", ctypes.c_int64), ("n_fake", ctypes.c_int64),
                ("n_tracks", ctypes.c_int64), ("efficiency", ctypes.c_double),
                ("clone_rate", ctypes.c_double), ("fake_rate", ctypes.c_double)]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.or_default_params.argtypes = [ctypes.POINTER(Params)]
            lib.or_geometry.argtypes = [vp, vp, vp]
            lib.or_quantize.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
            lib.or_sort_order.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.or_neighbours_sorted.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp]
            lib.or_neighbours_sorted.restype = ctypes.c_int
            lib.or_bruteforce_neighbours.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp]
            lib.or_bruteforce_links.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp]
            lib.or_bruteforce_links.restype = ctypes.c_int
            lib.or_propagate.argtypes = [vp, ctypes.c_double, vp, vp]
            lib.or_propagate.restype = ctypes.c_int
            lib.or_seed_chain.argtypes = [i32, vp, vp, vp, vp]
            lib.or_seed_chain.restype = ctypes.c_int
            lib.or_fit_chain.argtypes = [i32, i32, vp, vp, vp, vp]
            lib.or_fit_chain.restype = ctypes.c_int
            lib.or_track.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp, vp,
                                     i64, vp, vp]
            lib.or_track.restype = ctypes.c_int
            lib.or_eval.argtypes = [i64, vp, vp, vp, i64, i64, i32, ctypes.c_double, ctypes.POINTER(EvalOut)]
            lib.or_eval.restype = ctypes.c_int
            dbl = ctypes.c_double
            lib.or_bf16.argtypes = [ctypes.c_float]
            lib.or_bf16.restype = ctypes.c_float
            lib.or_feature_log1p.argtypes = [ctypes.c_float]
            lib.or_feature_log1p.restype = ctypes.c_float
            lib.or_mlp_features.argtypes = [i32, i32, i32, i32, i32, i32, i32, i64, i32, i32, i64, vp]
            lib.or_mlp_parse.argtypes = [vp, i64, vp]
            lib.or_mlp_parse.restype = ctypes.c_int
            lib.or_mlp_logit.argtypes = [vp, vp]
            lib.or_mlp_logit.restype = dbl
            lib.or_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp, dbl, vp, vp]
            lib.or_mlp_loss_grad.restype = ctypes.c_int
            lib.or_neighbours_pruned.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, dbl, vp, vp, vp,
                                                 vp, vp]
            lib.or_neighbours_pruned.restype = ctypes.c_int
            lib.or_track_ex.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, dbl, vp, vp, vp, vp, vp,
                                        vp, vp, i64, vp, vp, vp, vp]
            lib.or_track_ex.restype = ctypes.c_int
            lib.or_default_follow.argtypes = [ctypes.POINTER(FollowParams)]
            lib.or_track_follow.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp, dbl,
                                            ctypes.POINTER(FollowParams), vp, vp, i64, vp, vp, vp, vp, vp, vp, vp,
                                            vp]
            lib.or_rotate.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
            lib.or_rotate.restype = ctypes.c_int
            lib.or_track_follow.restype = ctypes.c_int
            lib.or_training_triplets.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), i64, vp, vp, vp, vp]
            lib.or_training_triplets.restype = ctypes.c_int
            _lib = lib
    return _lib


def params(**kw) -> Params:
    p = Params()
    _load().or_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def geometry():
    x = np.zeros(NROWS, np.float64)
    npads = np.zeros(NROWS, np.int32)
    pitch = np.zeros(NROWS, np.int32)
    _load().or_geometry(_p(x), _p(npads), _p(pitch))
    return x, npads, pitch


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def quantize(row, pad, time):
    row, pad, time = _c(row, np.uint16), _c(pad, np.float32), _c(time, np.float32)
    n = row.shape[0]
    pq, tq, yq = (np.zeros(n, np.int32) for _ in range(3))
    zq = np.zeros(n, np.int64)
    _load().or_quantize(n, _p(row), _p(pad), _p(time), _p(pq), _p(tq), _p(yq), _p(zq))
    return pq, tq, yq, zq


def sort_order(sector, row, pad, time):
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    order = np.zeros(sector.shape[0], np.int32)
    _load().or_sort_order(sector.shape[0], _p(sector), _p(row), _p(pad), _p(time), _p(order))
    return order


def neighbours_sorted(sector, row, pad, time, prm: Params | None = None):
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    down, up = np.zeros(n, np.int32), np.zeros(n, np.int32)
    cost = np.zeros(n, np.int64)
    rc = _load().or_neighbours_sorted(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm),
                                      _p(down), _p(up), _p(cost))
    if rc:
        raise MemoryError("oracle: neighbours failed")
    return down, up, cost


def bruteforce_neighbours(sector, row, pad, time, prm: Params | None = None):
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    down, up = np.zeros(n, np.int32), np.zeros(n, np.int32)
    _load().or_bruteforce_neighbours(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm),
                                     _p(down), _p(up))
    return down, up


def bruteforce_links(sector, row, pad, time, prm: Params | None = None):
    """Brute-force A1 choice followed by the A2 edge-row claims (caller indices)."""
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    down, up = np.zeros(n, np.int32), np.zeros(n, np.int32)
    if _load().or_bruteforce_links(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), _p(down), _p(up)):
        raise MemoryError("oracle: brute-force links failed")
    return down, up


def propagate(p, dx):
    """Transport (y, zeta, sin phi, dzeta/ds, q/pT) by dx; returns (p2, F) or None."""
    p = _c(p, np.float64)
    out = np.zeros(5, np.float64)
    F = np.zeros(25, np.float64)
    if _load().or_propagate(_p(p), float(dx), _p(out), _p(F)):
        return None
    return out, F.reshape(5, 5)


def seed_chain(rows, pads, times):
    """Seed state (y, 0, sin phi, dzeta/ds, q/pT) at the first cluster and status."""
    rows, pads, times = _c(rows, np.int32), _c(pads, np.float32), _c(times, np.float32)
    p0 = np.zeros(5, np.float64)
    st = _load().or_seed_chain(rows.shape[0], _p(rows), _p(pads), _p(times), _p(p0))
    return p0, st


def fit_chain(sector, rows, pads, times):
    rows, pads, times = _c(rows, np.int32), _c(pads, np.float32), _c(times, np.float32)
    rec = np.zeros(1, TRACK_DTYPE)
    rc = _load().or_fit_chain(rows.shape[0], int(sector), _p(rows), _p(pads), _p(times), _p(rec))
    if rc:
        raise ValueError("oracle: chain too short to fit")
    return rec[0]


def track(sector, row, pad, time, prm: Params | None = None, track_cap: int | None = None,
          mlp: bytes | None = None, tau: float = 0.5):
    """Run the whole path (A1 pruned by the classifier `mlp`, a weight blob, when
    given).  Returns a dict with `order` (sorted position -> caller index), `down`,
    `up`, `mdown`, `mup` (sorted positions, -1 = none), `is_start`,
    `cluster_track` (caller order) and `tracks` (TRACK_DTYPE records); with `mlp`
    also `band` (sorted positions whose pruning decision lies within the score
    band around tau) and `stats` (ambiguous clusters, scored pairs, changed
    choices, fallbacks)."""
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    cap = track_cap if track_cap is not None else max(16, n // max(1, prm.n_min) + 1)
    order = np.zeros(n, np.int32)
    down, up, mdown, mup = (np.zeros(n, np.int32) for _ in range(4))
    is_start = np.zeros(n, np.uint8)
    ct = np.zeros(n, np.int32)
    tracks = np.zeros(cap, TRACK_DTYPE)
    nt = ctypes.c_int64(0)
    if mlp is None:
        rc = _load().or_track(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), _p(order), _p(down),
                              _p(up), _p(mdown), _p(mup), _p(is_start), _p(ct), cap, _p(tracks), ctypes.byref(nt))
        extra = {}
    else:
        m = _mlp_struct(mlp)
        band = np.zeros(n, np.uint8)
        stats = np.zeros(4, np.int64)
        rc = _load().or_track_ex(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), _p(m), float(tau),
                                 _p(order), _p(down), _p(up), _p(mdown), _p(mup), _p(is_start), _p(ct), cap,
                                 _p(tracks), ctypes.byref(nt), _p(band), _p(stats))
        extra = dict(band=band.astype(bool), stats=stats)
    if rc < 0:
        raise MemoryError("oracle: track failed")
    return dict(order=order, down=down, up=up, mdown=mdown, mup=mup, is_start=is_start.astype(bool),
                cluster_track=ct, tracks=tracks[:min(nt.value, cap)], n_tracks=nt.value, **extra)


def follow_params(**kw) -> FollowParams:
    fp = FollowParams()
    _load().or_default_follow(ctypes.byref(fp))
    for k, v in kw.items():
        setattr(fp, k, v)
    return fp


def track_follow(sector, row, pad, time, prm: Params | None = None, fp: FollowParams | None = None,
                 track_cap: int | None = None, mlp: bytes | None = None, tau: float = 0.5):
    """The whole path followed by track following and joining (follow.c).  Returns
    `cluster_track` (caller order), `tracks` (TRACK_DTYPE), `n_tracks`, `margin`
    (per final track; < 1 marks membership an FP32 follower may decide
    differently), `old_to_new` (chain track -> final track), `n_chains` (tracks
    before following), `stats` (proposed pick-ups, accepted pick-ups, joins,
    dropped inward pick-ups) and, with fp.links = 1, `next` (the track continuing
    each track in the neighbouring sector, -1) with its margin `xmargin`."""
    prm = prm or params()
    fp = fp or follow_params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    cap = track_cap if track_cap is not None else max(16, n // max(1, prm.n_min) + 1)
    order = np.zeros(max(n, 1), np.int32)
    ct = np.zeros(max(n, 1), np.int32)
    tracks = np.zeros(cap, TRACK_DTYPE)
    margin = np.zeros(cap, np.float64)
    o2n = np.full(max(16, n // max(1, prm.n_min) + 1), -1, np.int32)
    nt, nch = ctypes.c_int64(0), ctypes.c_int64(0)
    stats = np.zeros(4, np.int64)
    nxt = np.full(cap, -1, np.int32)
    xmargin = np.full(cap, np.inf, np.float64)
    m = _mlp_struct(mlp) if mlp is not None else None
    rc = _load().or_track_follow(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm),
                                 _p(m) if m is not None else None, float(tau), ctypes.byref(fp), _p(order), _p(ct),
                                 cap, _p(tracks), ctypes.byref(nt), _p(margin), _p(o2n), ctypes.byref(nch),
                                 _p(stats), _p(nxt), _p(xmargin))
    if rc < 0:
        raise MemoryError("oracle: track_follow failed")
    k = min(nt.value, cap)
    return dict(cluster_track=ct[:n], tracks=tracks[:k], n_tracks=nt.value, margin=margin[:k],
                old_to_new=o2n[:nch.value], n_chains=nch.value, stats=stats, order=order[:n], next=nxt[:k],
                xmargin=xmargin[:k])


def rotate(p, x, beta):
    """Local frame rotated by beta: (p', x', J) or None (see follow.c)."""
    p = _c(p, np.float64)
    out = np.zeros(5, np.float64)
    xo = np.zeros(1, np.float64)
    J = np.zeros(25, np.float64)
    if _load().or_rotate(_p(p), float(x), float(beta), _p(out), _p(xo), _p(J)):
        return None
    return out, float(xo[0]), J.reshape(5, 5)


# ------------------------------------------------------------ link classifier
MLP_IN, MLP_H = 12, 64
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1
MLP_BLOB_BYTES = 16 + 4 * (2 * MLP_IN + MLP_NPARAM)
PRUNE_BAND = 1e-3


def mlp_blob(mean, inv_std, theta) -> bytes:
    """Weight blob (the library's file format, written out here independently):
    header (magic "TPCM", version 1, 12, 64) + float32 mean, inv_std, then theta =
    W1 (64x12), b1, W2 (64x64), b2, w3, b3 flattened in that order."""
    hdr = np.array([0x4D435054, 1, MLP_IN, MLP_H], np.uint32)
    body = np.concatenate([np.asarray(mean, np.float32).ravel(), np.asarray(inv_std, np.float32).ravel(),
                           np.asarray(theta, np.float32).ravel()])
    assert body.size == 2 * MLP_IN + MLP_NPARAM
    return hdr.tobytes() + body.astype("<f4").tobytes()


def _mlp_struct(blob: bytes):
    buf = np.frombuffer(blob, np.uint8).copy()
    m = np.zeros(4 * (2 * MLP_IN + MLP_NPARAM) + 64, np.uint8)  # or_mlp is all floats
    if _load().or_mlp_parse(_p(buf), buf.size, _p(m)) != 0:
        raise ValueError("oracle: bad classifier weight blob")
    return m


def bf16(x: float) -> float:
    return float(_load().or_bf16(float(x)))


def feature_log1p(v: float) -> float:
    return float(_load().or_feature_log1p(float(v)))


def mlp_features(r, yj, yi, yk, tj, ti, tk, cost, nj, nk, cost_max=147456000000):
    f = np.zeros(MLP_IN, np.float32)
    _load().or_mlp_features(int(r), int(yj), int(yi), int(yk), int(tj), int(ti), int(tk), int(cost), int(nj),
                            int(nk), int(cost_max), _p(f))
    return f


def mlp_logits(blob: bytes, feat) -> np.ndarray:
    """Inference logits of raw feature rows (float32[M, 12])."""
    feat = _c(feat, np.float32).reshape(-1, MLP_IN)
    m = _mlp_struct(blob)
    lib = _load()
    return np.array([lib.or_mlp_logit(_p(m), _p(feat[i])) for i in range(feat.shape[0])], np.float64)


def mlp_loss_grad(theta, mean, inv_std, feat, label, pos_weight=1.0):
    """FP64 loss and gradient (blob order) over the batch."""
    theta = _c(theta, np.float64)
    mean, inv_std = _c(mean, np.float32), _c(inv_std, np.float32)
    feat = _c(feat, np.float32).reshape(-1, MLP_IN)
    label = _c(label, np.uint8)
    grad = np.zeros(MLP_NPARAM, np.float64)
    loss = ctypes.c_double(0.0)
    rc = _load().or_mlp_loss_grad(_p(theta), _p(mean), _p(inv_std), feat.shape[0], _p(feat), _p(label),
                                  float(pos_weight), ctypes.byref(loss), _p(grad))
    if rc:
        raise ValueError("oracle: empty batch")
    return loss.value, grad


def neighbours_pruned(sector, row, pad, time, blob: bytes, tau: float, prm: Params | None = None):
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    down, up = np.zeros(n, np.int32), np.zeros(n, np.int32)
    cost = np.zeros(n, np.int64)
    band = np.zeros(n, np.uint8)
    stats = np.zeros(4, np.int64)
    m = _mlp_struct(blob)
    rc = _load().or_neighbours_pruned(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), _p(m),
                                      float(tau), _p(down), _p(up), _p(cost), _p(band), _p(stats))
    if rc:
        raise MemoryError("oracle: neighbours failed")
    return down, up, cost, band.astype(bool), stats


def training_triplets(sector, row, pad, time, prm: Params | None = None, cap: int | None = None):
    """(features float32[M,12], labels uint8[M], tri int32[M,3] caller indices)."""
    prm = prm or params()
    sector, row = _c(sector, np.uint16), _c(row, np.uint16)
    pad, time = _c(pad, np.float32), _c(time, np.float32)
    n = sector.shape[0]
    lib = _load()
    cnt = ctypes.c_int64(0)
    if cap is None:
        lib.or_training_triplets(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), 0, None, None, None,
                                 ctypes.byref(cnt))
        cap = cnt.value
    feat = np.zeros((max(cap, 1), MLP_IN), np.float32)
    label = np.zeros(max(cap, 1), np.uint8)
    tri = np.zeros((max(cap, 1), 3), np.int32)
    if lib.or_training_triplets(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), cap, _p(feat),
                                _p(label), _p(tri), ctypes.byref(cnt)):
        raise MemoryError("oracle: training triplets failed")
    m = min(cnt.value, cap)
    return feat[:m], label[:m], tri[:m]


def evaluate(label, sector, cluster_track, n_tracks, n_gen_tracks, min_findable=30, match_frac=0.9):
    label, sector = _c(label, np.int32), _c(sector, np.uint16)
    ct = _c(cluster_track, np.int32)
    out = EvalOut()
    _load().or_eval(label.shape[0], _p(label), _p(sector), _p(ct), int(n_tracks), int(n_gen_tracks),
                    int(min_findable), float(match_frac), ctypes.byref(out))
    return {f: getattr(out, f) for f, _ in EvalOut._fields_}
