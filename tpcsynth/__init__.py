"""Seeded synthetic TPC time frames: clusters in native (sector, row, pad, time)
coordinates plus generator truth.

This is the one module that both the CUDA path's tests and the CPU oracle's
tests draw inputs from.  It contains detector geometry and helix physics only,
none of the track-finding arithmetic.  The C source (``gen.c``) is compiled in
tree with gcc on first use (OpenMP when available; results do not depend on the
thread count because every random draw is a pure function of its key).

Named workloads (all synthetic; the paper's Monte-Carlo frames are not
available, these stand in for them):

* ``c1()``  one sector, one collision at t0 = 0, 200 tracks, side A, seed 1.
* ``c2()``  36 sectors, 2 ms continuous frame, 50 kHz Poisson collisions, seed 2.
* ``c3()``  36 sectors, 10 ms continuous frame, seed 3 (the paper's ~10 ms
  time frame processed whole, Sec. 1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtpcsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libtpcsynth.so (in tree).  Returns the path."""
    src = os.path.join(_HERE, "gen.c")
    hdr = os.path.join(_HERE, "gen.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO + ".tmp", src, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class TGConfig(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("single_collision", ctypes.c_int32),
        ("n_tracks", ctypes.c_int32),
        ("sector_only", ctypes.c_int32),
        ("frame_bins", ctypes.c_double),
        ("rate_khz", ctypes.c_double),
        ("mult_mean", ctypes.c_double),
        ("mult_cap", ctypes.c_int32),
        ("eta_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("phi_min", ctypes.c_double),
        ("phi_max", ctypes.c_double),
        ("pt_min", ctypes.c_double),
        ("pt_excess_mean", ctypes.c_double),
        ("sigma_y_cm", ctypes.c_double),
        ("sigma_t_bins", ctypes.c_double),
        ("noise_frac", ctypes.c_double),
        ("n_threads", ctypes.c_int32),
    ]


class _TGFrame(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("sector", ctypes.POINTER(ctypes.c_uint16)),
        ("row", ctypes.POINTER(ctypes.c_uint16)),
        ("pad", ctypes.POINTER(ctypes.c_float)),
        ("time", ctypes.POINTER(ctypes.c_float)),
        ("label", ctypes.POINTER(ctypes.c_int32)),
        ("n_tracks", ctypes.c_int64),
        ("trk_qpt", ctypes.POINTER(ctypes.c_double)),
        ("trk_phi0", ctypes.POINTER(ctypes.c_double)),
        ("trk_eta", ctypes.POINTER(ctypes.c_double)),
        ("trk_t0", ctypes.POINTER(ctypes.c_double)),
        ("trk_collision", ctypes.POINTER(ctypes.c_int32)),
        ("n_collisions", ctypes.c_int64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.tg_default_config.argtypes = [ctypes.POINTER(TGConfig)]
            lib.tg_generate.argtypes = [ctypes.POINTER(TGConfig), ctypes.POINTER(_TGFrame)]
            lib.tg_generate.restype = ctypes.c_int
            lib.tg_free.argtypes = [ctypes.POINTER(_TGFrame)]
            d = ctypes.c_double
            pd = ctypes.POINTER(ctypes.c_double)
            lib.tg_crossing.argtypes = [d, d, d, pd, pd, pd]
            lib.tg_crossing.restype = ctypes.c_int
            lib.tg_truth_at.argtypes = [d, d, d, d, ctypes.c_int, ctypes.c_int, pd, pd, pd, pd]
            lib.tg_truth_at.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Frame:
    """A generated time frame, sorted by (sector, row, time, pad, generation order)."""
    sector: np.ndarray  # uint16[n]
    row: np.ndarray     # uint16[n]
    pad: np.ndarray     # float32[n]
    time: np.ndarray    # float32[n], 0.2 us bins
    label: np.ndarray   # int32[n], generator track id or -1 (noise)
    trk_qpt: np.ndarray
    trk_phi0: np.ndarray
    trk_eta: np.ndarray
    trk_t0: np.ndarray
    trk_collision: np.ndarray
    n_collisions: int
    frame_bins: float

    @property
    def n(self) -> int:
        return int(self.sector.shape[0])


def default_config() -> TGConfig:
    c = TGConfig()
    _load().tg_default_config(ctypes.byref(c))
    return c


def generate(cfg: TGConfig) -> Frame:
    lib = _load()
    fr = _TGFrame()
    rc = lib.tg_generate(ctypes.byref(cfg), ctypes.byref(fr))
    if rc != 0:
        raise MemoryError("tpcsynth: generation failed (out of host memory)")
    n, nt = int(fr.n), int(fr.n_tracks)

    def arr(ptr, cnt, dt):
        if cnt == 0:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(ptr, shape=(cnt,)).astype(dt, copy=True)

    out = Frame(
        sector=arr(fr.sector, n, np.uint16), row=arr(fr.row, n, np.uint16),
        pad=arr(fr.pad, n, np.float32), time=arr(fr.time, n, np.float32),
        label=arr(fr.label, n, np.int32),
        trk_qpt=arr(fr.trk_qpt, nt, np.float64), trk_phi0=arr(fr.trk_phi0, nt, np.float64),
        trk_eta=arr(fr.trk_eta, nt, np.float64), trk_t0=arr(fr.trk_t0, nt, np.float64),
        trk_collision=arr(fr.trk_collision, nt, np.int32),
        n_collisions=int(fr.n_collisions), frame_bins=float(cfg.frame_bins))
    lib.tg_free(ctypes.byref(fr))
    return out


def crossing(c: float, pl: float, xr: float):
    """Closed-form first crossing of the local row plane x = xr (see gen.c)."""
    lib = _load()
    sig, y, sp = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = lib.tg_crossing(c, pl, xr, ctypes.byref(sig), ctypes.byref(y), ctypes.byref(sp))
    return (sig.value, y.value, sp.value) if ok else None


def truth_at(qpt, phi0, eta, t0_bins, sector, row):
    """Noise-free (y, time, sin(phi), dzeta/ds) of a generator track at a row crossing."""
    lib = _load()
    y, t, sp, tz = (ctypes.c_double() for _ in range(4))
    ok = lib.tg_truth_at(qpt, phi0, eta, t0_bins, sector, row,
                         ctypes.byref(y), ctypes.byref(t), ctypes.byref(sp), ctypes.byref(tz))
    return (y.value, t.value, sp.value, tz.value) if ok else None


# ---------------------------------------------------------------- named workloads
BIN_US = 0.2


def c1(seed: int = 1) -> TGConfig:
    """One sector (sector 0), one collision at t0 = 0, 200 tracks, eta in (0, 0.9),
    phi in (0, 20 deg); the frame is 500 bins (100 us, longer than the 484.5-bin drift)."""
    c = default_config()
    c.seed = seed
    c.single_collision = 1
    c.n_tracks = 200
    c.sector_only = 0
    c.frame_bins = 500.0
    c.eta_min, c.eta_max = 0.0, 0.9
    c.phi_min, c.phi_max = 0.0, math.radians(20.0)
    return c


def continuous(frame_ms: float, seed: int) -> TGConfig:
    c = default_config()
    c.seed = seed
    c.frame_bins = frame_ms * 1000.0 / BIN_US
    return c


def c2(seed: int = 2) -> TGConfig:
    """36 sectors, 2 ms continuous frame, collisions Poisson at 50 kHz."""
    return continuous(2.0, seed)


def c3(seed: int = 3) -> TGConfig:
    """36 sectors, 10 ms continuous frame (~500 collisions)."""
    return continuous(10.0, seed)


# clusters per sector per ms at 50 kHz in this generator (10 ms frame, seed 3: 31.96M / 36 / 10)
CLUSTERS_PER_SECTOR_MS_50KHZ = 8.88e4


@dataclass
class Batch:
    """Many independent (sector x time frame) instances packed for one batched call:
    `frame.sector` holds the instance id; instance k occupies clusters
    [offsets[k], offsets[k+1]) and came from sector `src_sector[k]` of a frame of
    `length_ms[k]` at `rate_khz[k]` (seed `seeds[k]`)."""
    frame: Frame
    offsets: np.ndarray
    length_ms: np.ndarray
    rate_khz: np.ndarray
    seeds: np.ndarray
    src_sector: np.ndarray


def batched(n_inst: int = 256, seed: int = 4, n_min: float = 1e4, n_max: float = 2e6, ms_min: float = 0.2,
            ms_max: float = 10.0) -> Batch:
    """Instances with cluster counts log-uniform in [n_min, n_max] and frame lengths
    uniform in [ms_min, ms_max]: each is one sector of its own continuous frame whose
    collision rate is rescaled from 50 kHz so that the expected count is the drawn one."""
    rng = np.random.default_rng(seed)
    target = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_inst))
    length = rng.uniform(ms_min, ms_max, n_inst)
    rate = 50.0 * target / (CLUSTERS_PER_SECTOR_MS_50KHZ * length)
    seeds = seed * 1_000_003 + np.arange(n_inst, dtype=np.int64)
    parts, offsets, labels_off = [], [0], 0
    src = np.arange(n_inst) % 36
    for k in range(n_inst):
        c = continuous(float(length[k]), int(seeds[k]))
        c.rate_khz = float(rate[k])
        c.sector_only = int(src[k])
        f = generate(c)
        f.sector = np.full(f.n, k, np.uint16)
        f.label = np.where(f.label >= 0, f.label + labels_off, -1).astype(np.int32)
        labels_off += f.trk_qpt.shape[0]
        parts.append(f)
        offsets.append(offsets[-1] + f.n)
    cat = lambda name, dt: np.concatenate([getattr(p, name) for p in parts]).astype(dt)
    frame = Frame(sector=cat("sector", np.uint16), row=cat("row", np.uint16), pad=cat("pad", np.float32),
                  time=cat("time", np.float32), label=cat("label", np.int32), trk_qpt=cat("trk_qpt", np.float64),
                  trk_phi0=cat("trk_phi0", np.float64), trk_eta=cat("trk_eta", np.float64),
                  trk_t0=cat("trk_t0", np.float64), trk_collision=cat("trk_collision", np.int32),
                  n_collisions=int(sum(p.n_collisions for p in parts)), frame_bins=float(max(p.frame_bins for p in parts)))
    return Batch(frame=frame, offsets=np.array(offsets, np.int64), length_ms=length, rate_khz=rate, seeds=seeds,
                 src_sector=src)
