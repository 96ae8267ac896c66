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
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", _SO + ".tmp", src, "-lm"], check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("wy_q", ctypes.c_int32), ("wt_q", ctypes.c_int32),
                ("cost_max_q", ctypes.c_int64), ("n_min", ctypes.c_int32)]


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


def track(sector, row, pad, time, prm: Params | None = None, track_cap: int | None = None):
    """Run the whole path.  Returns a dict with `order` (sorted position -> caller
    index), `down`, `up`, `mdown`, `mup` (sorted positions, -1 = none), `is_start`,
    `cluster_track` (caller order) and `tracks` (TRACK_DTYPE records)."""
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
    rc = _load().or_track(n, _p(sector), _p(row), _p(pad), _p(time), ctypes.byref(prm), _p(order), _p(down),
                          _p(up), _p(mdown), _p(mup), _p(is_start), _p(ct), cap, _p(tracks), ctypes.byref(nt))
    if rc < 0:
        raise MemoryError("oracle: track failed")
    return dict(order=order, down=down, up=up, mdown=mdown, mup=mup, is_start=is_start.astype(bool),
                cluster_track=ct, tracks=tracks[:min(nt.value, cap)], n_tracks=nt.value)


def evaluate(label, sector, cluster_track, n_tracks, n_gen_tracks, min_findable=30, match_frac=0.9):
    label, sector = _c(label, np.int32), _c(sector, np.uint16)
    ct = _c(cluster_track, np.int32)
    out = EvalOut()
    _load().or_eval(label.shape[0], _p(label), _p(sector), _p(ct), int(n_tracks), int(n_gen_tracks),
                    int(min_findable), float(match_frac), ctypes.byref(out))
    return {f: getattr(out, f) for f, _ in EvalOut._fields_}
