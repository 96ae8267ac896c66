"""ctypes binding of the C ABI in include/tpcca.h (same names, argument
marshalling only: every step of the tracking path runs in libtpcca.so's CUDA
kernels).  PyTorch provides device memory and streams.

The library is built in tree by ``paper_2102_08862_gb300._build.build()``; if it is
missing, loading fails loudly -- there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

from . import _build

c_u32, c_i32, c_i64, c_f32, c_vp = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p

TPC_OK = 0
TPC_ERR_ARG = -1
TPC_ERR_CAPACITY = -2
TPC_ERR_CUDA = -3
TPC_ERR_INPUT = -4
TPC_ERR_TIMEOUT = -5
TPC_MODE_PLAIN = 0
TPC_MODE_PRUNED = 1
TPC_INPUT_SORTED = 1
TPC_FIT_THREAD = 0
TPC_FIT_WARP = 1
TPC_MMA_TCGEN05 = 0
TPC_MMA_SYNC = 1
ERROR_NAMES = {0: "TPC_OK", -1: "TPC_ERR_ARG", -2: "TPC_ERR_CAPACITY", -3: "TPC_ERR_CUDA", -4: "TPC_ERR_INPUT",
               -5: "TPC_ERR_TIMEOUT"}


class tpc_tf_config(ctypes.Structure):
    _fields_ = [("max_clusters", c_u32), ("max_tracks", c_u32), ("wy_q", c_i32), ("wt_q", c_i32),
                ("cost_max_q", c_i64), ("n_min", c_i32), ("mode", c_i32), ("tau", c_f32), ("device", c_i32),
                ("fit_variant", c_i32), ("profile_stages", c_i32), ("row_cap", c_i32), ("n_sectors", c_i32),
                ("nb_tile", c_i32), ("follow", c_i32), ("follow_chi2", c_f32), ("follow_miss", c_i32),
                ("follow_check", c_i32), ("follow_link_chi2", c_f32), ("follow_link_rows", c_i32),
                ("mlp_engine", c_i32), ("persistent", c_i32)]


class tpc_clusters(ctypes.Structure):
    _fields_ = [("n", c_u32), ("flags", c_u32), ("sector", c_vp), ("row", c_vp), ("pad", c_vp), ("time", c_vp)]


class tpc_tracks(ctypes.Structure):
    _fields_ = [("cluster_track", c_vp), ("track_capacity", c_u32), ("params", c_vp), ("cov", c_vp),
                ("t_ref", c_vp), ("x", c_vp), ("chi2", c_vp), ("ndf", c_vp), ("nhits", c_vp),
                ("first_cluster", c_vp), ("sector", c_vp), ("row_first", c_vp), ("row_last", c_vp),
                ("status", c_vp), ("n_tracks", c_vp), ("n_tracks_host", c_vp), ("next_track", c_vp)]


class tpc_mlp_train_config(ctypes.Structure):
    _fields_ = [("lr", c_f32), ("beta1", c_f32), ("beta2", c_f32), ("eps", c_f32), ("pos_weight", c_f32),
                ("max_batch", c_u32), ("device", c_i32), ("engine", c_i32)]


class tpc_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", c_i32), ("device", c_i32),
                ("tf", tpc_tf_config), ("mlp_blob", c_vp), ("mlp_bytes", ctypes.c_size_t)]


class tpc_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", c_i32), ("n_clusters", c_u32), ("n_tracks", c_u32),
                ("slot", c_i32), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


TPC_ADMIT_RUN, TPC_ADMIT_CREATE, TPC_ADMIT_REPLACE, TPC_ADMIT_WAIT = 0, 1, 2, 3

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/tpcca.h."""
    txt = open(os.path.join(_build.INCLUDE, "tpcca.h")).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(tpc_\w+)\s*\(", txt, re.M)))


def load():
    """Load libtpcca.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: build it with paper_2102_08862_gb300._build.build() "
                          "(the tracker has no CPU fallback)")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    lib.tpc_default_config.argtypes = [P(tpc_tf_config)]
    lib.tpc_default_config.restype = None
    lib.tpc_tf_create.argtypes = [P(tpc_tf_config), P(c_vp)]
    lib.tpc_tf_create.restype = ctypes.c_int
    lib.tpc_track_timeframe.argtypes = [c_vp, P(tpc_clusters), P(tpc_tracks), c_vp]
    lib.tpc_track_timeframe.restype = ctypes.c_int
    lib.tpc_track_timeframe_host.argtypes = [c_vp, P(tpc_clusters), P(tpc_tracks), c_vp]
    lib.tpc_track_timeframe_host.restype = ctypes.c_int
    lib.tpc_track_timeframe_noalloc.argtypes = [P(tpc_tf_config), P(tpc_clusters), P(tpc_tracks), c_vp]
    lib.tpc_track_timeframe_noalloc.restype = ctypes.c_int
    lib.tpc_tf_status.argtypes = [c_vp, c_vp]
    lib.tpc_tf_status.restype = ctypes.c_int
    lib.tpc_tf_destroy.argtypes = [c_vp]
    lib.tpc_tf_destroy.restype = None
    lib.tpc_last_error.argtypes = []
    lib.tpc_last_error.restype = ctypes.c_char_p
    lib.tpc_tf_debug_links.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]
    lib.tpc_tf_debug_links.restype = ctypes.c_int
    lib.tpc_tf_stage_times.argtypes = [c_vp, P(c_f32), P(ctypes.c_char_p), ctypes.c_int]
    lib.tpc_tf_stage_times.restype = ctypes.c_int
    lib.tpc_tf_launches_per_call.argtypes = [c_vp]
    lib.tpc_tf_launches_per_call.restype = ctypes.c_int
    lib.tpc_debug_quantize.argtypes = [c_vp, c_u32, c_vp, c_vp]
    lib.tpc_debug_quantize.restype = ctypes.c_int
    lib.tpc_tf_set_spin_limit.argtypes = [c_vp, c_u32]
    lib.tpc_tf_set_spin_limit.restype = ctypes.c_int
    lib.tpc_tf_debug_wait.argtypes = [c_vp, c_vp]
    lib.tpc_tf_debug_wait.restype = ctypes.c_int
    lib.tpc_tf_remove_unassigned.argtypes = [c_vp, P(tpc_clusters), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]
    lib.tpc_tf_remove_unassigned.restype = ctypes.c_int
    lib.tpc_tf_arena_bytes.argtypes = [P(tpc_tf_config), P(ctypes.c_size_t)]
    lib.tpc_tf_arena_bytes.restype = ctypes.c_int
    lib.tpc_server_default_config.argtypes = [P(tpc_server_config)]
    lib.tpc_server_default_config.restype = None
    lib.tpc_server_create.argtypes = [P(tpc_server_config), P(c_vp)]
    lib.tpc_server_create.restype = ctypes.c_int
    lib.tpc_server_submit.argtypes = [c_vp, P(tpc_clusters), P(tpc_tracks), P(ctypes.c_uint64)]
    lib.tpc_server_submit.restype = ctypes.c_int
    lib.tpc_server_poll.argtypes = [c_vp, P(tpc_server_result), ctypes.c_int, ctypes.c_int]
    lib.tpc_server_poll.restype = ctypes.c_int
    lib.tpc_server_stats.argtypes = [c_vp, P(c_i32), P(ctypes.c_uint64), P(c_i32)]
    lib.tpc_server_stats.restype = ctypes.c_int
    lib.tpc_server_destroy.argtypes = [c_vp]
    lib.tpc_server_destroy.restype = None
    lib.tpc_server_admit.argtypes = [c_u32, c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint64, P(ctypes.c_int)]
    lib.tpc_server_admit.restype = ctypes.c_int
    lib.tpc_track_timeframe_graph.argtypes = [c_vp, P(tpc_clusters), P(tpc_tracks), c_vp]
    lib.tpc_track_timeframe_graph.restype = ctypes.c_int
    lib.tpc_tf_autotune.argtypes = [c_vp, P(tpc_clusters), P(tpc_tracks), ctypes.c_int, c_vp, P(c_i32), P(c_i32),
                                    P(c_i32)]
    lib.tpc_tf_autotune.restype = ctypes.c_int
    sz = ctypes.c_size_t
    lib.tpc_mlp_blob_bytes.argtypes = []
    lib.tpc_mlp_blob_bytes.restype = sz
    lib.tpc_mlp_load.argtypes = [c_vp, c_vp, sz]
    lib.tpc_mlp_load.restype = ctypes.c_int
    lib.tpc_mlp_score.argtypes = [c_vp, c_vp, c_u32, c_vp, c_vp]
    lib.tpc_mlp_score.restype = ctypes.c_int
    lib.tpc_mlp_score_ex.argtypes = [c_vp, c_vp, c_u32, c_vp, ctypes.c_int, c_vp]
    lib.tpc_mlp_score_ex.restype = ctypes.c_int
    lib.tpc_mlp_extract.argtypes = [c_vp, P(tpc_clusters), c_vp, c_vp, c_vp, c_u32, c_vp, c_vp]
    lib.tpc_mlp_extract.restype = ctypes.c_int
    lib.tpc_tf_pruned_clusters.argtypes = [c_vp, P(c_u32), P(c_u32), c_vp]
    lib.tpc_tf_pruned_clusters.restype = ctypes.c_int
    lib.tpc_mlp_default_train_config.argtypes = [P(tpc_mlp_train_config)]
    lib.tpc_mlp_default_train_config.restype = None
    lib.tpc_mlp_trainer_create.argtypes = [P(tpc_mlp_train_config), c_vp, sz, P(c_vp)]
    lib.tpc_mlp_trainer_create.restype = ctypes.c_int
    lib.tpc_mlp_trainer_destroy.argtypes = [c_vp]
    lib.tpc_mlp_trainer_destroy.restype = None
    lib.tpc_mlp_trainer_normalise.argtypes = [c_vp, c_vp, c_u32, c_vp]
    lib.tpc_mlp_trainer_normalise.restype = ctypes.c_int
    lib.tpc_mlp_train_step.argtypes = [c_vp, c_vp, c_vp, c_vp, c_u32, c_vp, c_vp]
    lib.tpc_mlp_train_step.restype = ctypes.c_int
    lib.tpc_mlp_trainer_gradient.argtypes = [c_vp, c_vp, c_vp, c_vp, c_u32, c_vp, c_vp, c_vp]
    lib.tpc_mlp_trainer_gradient.restype = ctypes.c_int
    lib.tpc_mlp_trainer_blob.argtypes = [c_vp, c_vp, sz]
    lib.tpc_mlp_trainer_blob.restype = ctypes.c_int
    _lib = lib
    return lib


class TpcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc):
    if rc != TPC_OK:
        raise TpcError(rc, load().tpc_last_error().decode())
    return rc


# ------------------------------------------------------------ thin wrappers
def tpc_default_config() -> tpc_tf_config:
    c = tpc_tf_config()
    load().tpc_default_config(ctypes.byref(c))
    return c


def tpc_tf_create(cfg: tpc_tf_config) -> int:
    h = c_vp()
    _check(load().tpc_tf_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def tpc_track_timeframe(handle, clusters: tpc_clusters, tracks: tpc_tracks, stream: int = 0) -> int:
    return load().tpc_track_timeframe(handle, ctypes.byref(clusters), ctypes.byref(tracks), stream)


def tpc_track_timeframe_host(handle, clusters: tpc_clusters, tracks: tpc_tracks, stream: int = 0) -> int:
    return load().tpc_track_timeframe_host(handle, ctypes.byref(clusters), ctypes.byref(tracks), stream)


def tpc_track_timeframe_noalloc(cfg, clusters: tpc_clusters, tracks: tpc_tracks, stream: int = 0) -> int:
    """The tracking call without any device allocation, for callers that may not
    allocate (graph capture, fixed-budget hosts): small sorted frames only, all
    scratch in a static device array inside the library; calls must not overlap."""
    return load().tpc_track_timeframe_noalloc(ctypes.byref(cfg) if cfg is not None else None,
                                              ctypes.byref(clusters), ctypes.byref(tracks), stream)


def tpc_tf_status(handle, stream: int = 0) -> int:
    return load().tpc_tf_status(handle, stream)


def tpc_tf_destroy(handle) -> None:
    load().tpc_tf_destroy(handle)


def tpc_last_error() -> str:
    return load().tpc_last_error().decode()


def tpc_tf_debug_links(handle, order, down, up, mup, is_start, stream: int = 0) -> int:
    return load().tpc_tf_debug_links(handle, order, down, up, mup, is_start, stream)


def tpc_tf_stage_times(handle, cap: int = 16):
    ms = (c_f32 * cap)()
    names = (ctypes.c_char_p * cap)()
    n = load().tpc_tf_stage_times(handle, ms, names, cap)
    _check(min(n, 0))
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def tpc_tf_launches_per_call(handle) -> int:
    return load().tpc_tf_launches_per_call(handle)


def tpc_debug_quantize(v_ptr, n: int, q_ptr, stream: int = 0) -> int:
    return load().tpc_debug_quantize(v_ptr, n, q_ptr, stream)


def tpc_tf_set_spin_limit(handle, polls: int) -> int:
    return load().tpc_tf_set_spin_limit(handle, polls)


def tpc_tf_debug_wait(handle, stream: int = 0) -> int:
    return load().tpc_tf_debug_wait(handle, stream)


def tpc_track_timeframe_graph(handle, clusters: tpc_clusters, tracks: tpc_tracks, stream: int = 0) -> int:
    return load().tpc_track_timeframe_graph(handle, ctypes.byref(clusters), ctypes.byref(tracks), stream)


def tpc_tf_autotune(handle, clusters: tpc_clusters, tracks: tpc_tracks, trials: int = 3, stream: int = 0):
    """(nb_tile, fit_variant, mlp_engine) chosen by the autotuner (kept in the handle)."""
    t, f, e = c_i32(0), c_i32(0), c_i32(0)
    _check(load().tpc_tf_autotune(handle, ctypes.byref(clusters), ctypes.byref(tracks), trials, stream,
                                  ctypes.byref(t), ctypes.byref(f), ctypes.byref(e)))
    return int(t.value), int(f.value), int(e.value)


def tpc_tf_arena_bytes(cfg: tpc_tf_config) -> int:
    b = ctypes.c_size_t(0)
    _check(load().tpc_tf_arena_bytes(ctypes.byref(cfg), ctypes.byref(b)))
    return int(b.value)


def tpc_server_admit(n, cap, nbytes, busy, max_slots, budget, new_bytes):
    """(slot, action) of the serving runtime's admission policy."""
    import numpy as np
    cap = np.ascontiguousarray(cap, np.uint32)
    nbytes = np.ascontiguousarray(nbytes, np.uint64)
    busy = np.ascontiguousarray(busy, np.uint8)
    act = ctypes.c_int(-1)
    k = load().tpc_server_admit(int(n), cap.ctypes.data, nbytes.ctypes.data, busy.ctypes.data, int(cap.size),
                                int(max_slots), int(budget), int(new_bytes), ctypes.byref(act))
    return k, act.value


class Server:
    """The serving runtime (tpc_server_*): submit host frames, poll results.  The
    host arrays of a request are kept alive here until its result is polled."""

    def __init__(self, budget_bytes=180 << 30, max_slots=4, device=0, mlp_blob: bytes | None = None, **tf):
        cfg = tpc_server_config()
        load().tpc_server_default_config(ctypes.byref(cfg))
        cfg.hbm_budget_bytes = int(budget_bytes)
        cfg.max_slots = int(max_slots)
        cfg.device = int(device)
        for k, v in tf.items():
            setattr(cfg.tf, k, v)
        self._blob = None
        if mlp_blob is not None:
            self._blob = ctypes.create_string_buffer(bytes(mlp_blob), len(mlp_blob))
            cfg.mlp_blob = ctypes.cast(self._blob, c_vp)
            cfg.mlp_bytes = len(mlp_blob)
        h = c_vp()
        _check(load().tpc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._live = {}

    def submit(self, sector, row, pad, time, track_capacity=0):
        """Queue one frame (numpy arrays, or pinned torch CPU tensors); returns the
        request id.  Its cluster_track array is returned by poll()."""
        import numpy as np
        arrs = []
        for a, dt in ((sector, np.uint16), (row, np.uint16), (pad, np.float32), (time, np.float32)):
            if hasattr(a, "data_ptr"):
                arrs.append((a, a.data_ptr()))
            else:
                a = np.ascontiguousarray(a, dtype=dt)
                arrs.append((a, a.ctypes.data))
        n = int(len(arrs[0][0]))
        ct = np.empty(max(n, 1), np.int32)
        cl = tpc_clusters(n=n, flags=TPC_INPUT_SORTED, sector=arrs[0][1], row=arrs[1][1], pad=arrs[2][1],
                          time=arrs[3][1])
        tr = tpc_tracks(cluster_track=ct.ctypes.data, track_capacity=0)
        rid = ctypes.c_uint64(0)
        _check(load().tpc_server_submit(self.handle, ctypes.byref(cl), ctypes.byref(tr), ctypes.byref(rid)))
        self._live[rid.value] = (arrs, ct, n)
        return rid.value

    def poll(self, max_results=64, wait_ms=100):
        """Finished requests: list of (result dict, cluster_track numpy array)."""
        buf = (tpc_server_result * max_results)()
        k = load().tpc_server_poll(self.handle, buf, max_results, int(wait_ms))
        if k < 0:
            _check(k)
        out = []
        for r in buf[:k]:
            arrs, ct, n = self._live.pop(r.id)
            out.append(({f: getattr(r, f) for f, _ in tpc_server_result._fields_}, ct[:n]))
        return out

    def stats(self):
        ns, q = c_i32(0), c_i32(0)
        b = ctypes.c_uint64(0)
        _check(load().tpc_server_stats(self.handle, ctypes.byref(ns), ctypes.byref(b), ctypes.byref(q)))
        return dict(slots=ns.value, bytes=b.value, queued=q.value)

    def close(self):
        if self.handle:
            load().tpc_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tpc_mlp_blob_bytes() -> int:
    return int(load().tpc_mlp_blob_bytes())


def tpc_mlp_load(handle, blob: bytes) -> int:
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    return load().tpc_mlp_load(handle, ctypes.cast(buf, c_vp), len(blob))


def tpc_mlp_score(handle, feat_ptr, m, logit_ptr, stream=0) -> int:
    return load().tpc_mlp_score(handle, feat_ptr, m, logit_ptr, stream)


def tpc_mlp_extract(handle, clusters, feat_ptr, label_ptr, tri_ptr, cap, count_ptr, stream=0) -> int:
    return load().tpc_mlp_extract(handle, ctypes.byref(clusters), feat_ptr, label_ptr, tri_ptr, cap, count_ptr,
                                  stream)


def tpc_tf_pruned_clusters(handle, stream=0):
    """(clusters rescored from the tile regions, clusters rescored from the overflow list)."""
    a, b = c_u32(0), c_u32(0)
    _check(load().tpc_tf_pruned_clusters(handle, ctypes.byref(a), ctypes.byref(b), stream))
    return int(a.value), int(b.value)


def tpc_mlp_default_train_config() -> tpc_mlp_train_config:
    c = tpc_mlp_train_config()
    load().tpc_mlp_default_train_config(ctypes.byref(c))
    return c


# ------------------------------------------------------------ classifier weights
MLP_IN, MLP_H = 12, 64
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1
MLP_PARAM_SHAPES = [("W1", (MLP_H, MLP_IN)), ("b1", (MLP_H,)), ("W2", (MLP_H, MLP_H)), ("b2", (MLP_H,)),
                    ("w3", (MLP_H,)), ("b3", (1,))]
_BLOB_MAGIC = 0x4D435054  # "TPCM"


def pack_blob(mean, inv_std, theta) -> bytes:
    """Weight blob of the C ABI: header (magic, version 1, 12, 64) + float32 mean,
    inv_std, then theta = W1, b1, W2, b2, w3, b3 flattened in that order."""
    import numpy as np
    hdr = np.array([_BLOB_MAGIC, 1, MLP_IN, MLP_H], "<u4")
    body = np.concatenate([np.asarray(mean, "<f4").ravel(), np.asarray(inv_std, "<f4").ravel(),
                           np.asarray(theta, "<f4").ravel()])
    if body.size != 2 * MLP_IN + MLP_NPARAM:
        raise ValueError("classifier blob: wrong number of parameters")
    return hdr.tobytes() + body.tobytes()


def unpack_blob(blob: bytes):
    """(mean, inv_std, theta) of a weight blob."""
    import numpy as np
    hdr = np.frombuffer(blob[:16], "<u4")
    if hdr[0] != _BLOB_MAGIC or hdr[1] != 1 or hdr[2] != MLP_IN or hdr[3] != MLP_H:
        raise ValueError("classifier blob: bad header")
    body = np.frombuffer(blob[16:16 + 4 * (2 * MLP_IN + MLP_NPARAM)], "<f4")
    return body[:MLP_IN].copy(), body[MLP_IN:2 * MLP_IN].copy(), body[2 * MLP_IN:].copy()


def init_blob(seed: int = 0) -> bytes:
    """He-initialised weights (zero biases, identity standardisation)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in MLP_PARAM_SHAPES:
        if name.startswith("W"):
            parts.append(rng.standard_normal(shape) * np.sqrt(2.0 / shape[1]))
        elif name == "w3":
            parts.append(rng.standard_normal(shape) * np.sqrt(1.0 / MLP_H))
        else:
            parts.append(np.zeros(shape))
    theta = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    return pack_blob(np.zeros(MLP_IN), np.ones(MLP_IN), theta)


class Trainer:
    """Owns one tpc_mlp_trainer (FP32 master weights, Adam moments, BF16 copy);
    batches are torch CUDA tensors."""

    def __init__(self, blob: bytes, device: int = 0, **overrides):
        import torch
        self.torch = torch
        cfg = tpc_mlp_default_train_config()
        cfg.device = int(device)
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.device = torch.device("cuda", device)
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        h = c_vp()
        _check(load().tpc_mlp_trainer_create(ctypes.byref(cfg), ctypes.cast(buf, c_vp), len(blob), ctypes.byref(h)))
        self.handle = h.value
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self._grad = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=self.device)

    def close(self):
        if self.handle:
            load().tpc_mlp_trainer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def normalise(self, feat):
        _check(load().tpc_mlp_trainer_normalise(self.handle, feat.data_ptr(), int(feat.shape[0]), self._stream()))

    def step(self, feat, label, index=None, batch=None):
        """One Adam step; returns the device loss tensor (mean weighted BCE before the step)."""
        b = int(batch if batch is not None else (index.numel() if index is not None else feat.shape[0]))
        _check(load().tpc_mlp_train_step(self.handle, feat.data_ptr(), label.data_ptr(),
                                         index.data_ptr() if index is not None else None, b,
                                         self._loss.data_ptr(), self._stream()))
        return self._loss

    def gradient(self, feat, label, index=None):
        b = int(index.numel() if index is not None else feat.shape[0])
        _check(load().tpc_mlp_trainer_gradient(self.handle, feat.data_ptr(), label.data_ptr(),
                                               index.data_ptr() if index is not None else None, b,
                                               self._grad.data_ptr(), self._loss.data_ptr(), self._stream()))
        self.torch.cuda.synchronize(self.device)
        return self._grad.clone(), float(self._loss.item())

    def blob(self) -> bytes:
        n = tpc_mlp_blob_bytes()
        buf = ctypes.create_string_buffer(n)
        _check(load().tpc_mlp_trainer_blob(self.handle, ctypes.cast(buf, c_vp), n))
        return buf.raw


# ------------------------------------------------------------ torch convenience
@dataclass
class Tracks:
    cluster_track: "object"  # int32[n]
    n_tracks: int
    params: "object"         # float32[n_tracks, 5]
    cov: "object"            # float32[n_tracks, 15]
    t_ref: "object"
    x: "object"
    chi2: "object"
    ndf: "object"
    nhits: "object"
    first_cluster: "object"
    sector: "object"
    row_first: "object"
    row_last: "object"
    status: "object"
    next_track: "object" = None  # int32[n_tracks] with follow = 2


class TimeFrameTracker:
    """Owns one tpc_tf handle; inputs and outputs are torch CUDA tensors."""

    def __init__(self, max_clusters: int, device: int = 0, **overrides):
        import torch
        self.torch = torch
        cfg = tpc_default_config()
        cfg.max_clusters = int(max_clusters)
        cfg.device = int(device)
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.device = torch.device("cuda", device)
        self.handle = tpc_tf_create(cfg)
        self._out = None
        self._cap = 0
        self._n = 0

    def close(self):
        if self.handle:
            tpc_tf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outputs(self, n, capacity):
        t = self.torch
        if self._out is None or self._cap < capacity or self._out["cluster_track"].numel() < max(n, 1):
            cap = max(capacity, 1)
            d = self.device
            self._out = dict(
                cluster_track=t.empty(max(n, 1), dtype=t.int32, device=d),
                params=t.empty((cap, 5), dtype=t.float32, device=d),
                cov=t.empty((cap, 15), dtype=t.float32, device=d),
                t_ref=t.empty(cap, dtype=t.float32, device=d), x=t.empty(cap, dtype=t.float32, device=d),
                chi2=t.empty(cap, dtype=t.float32, device=d), ndf=t.empty(cap, dtype=t.int32, device=d),
                nhits=t.empty(cap, dtype=t.int32, device=d), first_cluster=t.empty(cap, dtype=t.int32, device=d),
                sector=t.empty(cap, dtype=t.int16, device=d), row_first=t.empty(cap, dtype=t.int16, device=d),
                row_last=t.empty(cap, dtype=t.int16, device=d), status=t.empty(cap, dtype=t.uint8, device=d),
                next_track=t.empty(cap, dtype=t.int32, device=d),
                n_tracks=t.zeros(1, dtype=t.int32, device=d))
            self._cap = cap
        return self._out

    def structs(self, sector, row, pad, time, sorted_input=True, capacity=None, host_count=None):
        """Build the tpc_clusters / tpc_tracks structs for device tensors."""
        n = int(sector.numel())
        cap = int(capacity if capacity is not None else max(16, n // max(1, self.cfg.n_min) + 1))
        o = self._outputs(n, cap)
        cl = tpc_clusters(n=n, flags=TPC_INPUT_SORTED if sorted_input else 0, sector=sector.data_ptr(),
                          row=row.data_ptr(), pad=pad.data_ptr(), time=time.data_ptr())
        tr = tpc_tracks(cluster_track=o["cluster_track"].data_ptr(), track_capacity=cap,
                        params=o["params"].data_ptr(), cov=o["cov"].data_ptr(), t_ref=o["t_ref"].data_ptr(),
                        x=o["x"].data_ptr(), chi2=o["chi2"].data_ptr(), ndf=o["ndf"].data_ptr(),
                        nhits=o["nhits"].data_ptr(), first_cluster=o["first_cluster"].data_ptr(),
                        sector=o["sector"].data_ptr(), row_first=o["row_first"].data_ptr(),
                        row_last=o["row_last"].data_ptr(), status=o["status"].data_ptr(),
                        n_tracks=o["n_tracks"].data_ptr(),
                        n_tracks_host=ctypes.addressof(host_count) if host_count is not None else None,
                        next_track=o["next_track"].data_ptr() if self.cfg.follow == 2 else None)
        return cl, tr, n, cap

    def track(self, sector, row, pad, time, sorted_input=True, capacity=None, stream=None) -> Tracks:
        t = self.torch
        st = stream if stream is not None else t.cuda.current_stream(self.device)
        cnt = c_u32(0)
        cl, tr, n, cap = self.structs(sector, row, pad, time, sorted_input, capacity, host_count=cnt)
        _check(tpc_track_timeframe(self.handle, cl, tr, st.cuda_stream))
        self._n = n
        nt = int(cnt.value)
        m = min(nt, cap)
        o = self._out
        return Tracks(cluster_track=o["cluster_track"][:n], n_tracks=nt, params=o["params"][:m], cov=o["cov"][:m],
                      t_ref=o["t_ref"][:m], x=o["x"][:m], chi2=o["chi2"][:m], ndf=o["ndf"][:m],
                      nhits=o["nhits"][:m], first_cluster=o["first_cluster"][:m], sector=o["sector"][:m],
                      row_first=o["row_first"][:m], row_last=o["row_last"][:m], status=o["status"][:m],
                      next_track=o["next_track"][:m] if self.cfg.follow == 2 else None)

    def track_graph(self, sector, row, pad, time, sorted_input=True, capacity=None, stream=None):
        """tpc_track_timeframe_graph on device tensors; returns the device track count
        tensor (nothing is synchronised)."""
        t = self.torch
        st = stream if stream is not None else t.cuda.current_stream(self.device)
        cl, tr, n, cap = self.structs(sector, row, pad, time, sorted_input, capacity, host_count=None)
        _check(tpc_track_timeframe_graph(self.handle, cl, tr, st.cuda_stream))
        self._n = n
        return self._out["n_tracks"]

    def track_host(self, sector, row, pad, time, sorted_input=True, capacity=None, pinned=False):
        """tpc_track_timeframe_host on numpy arrays (host buffers): the call copies
        them in, tracks, copies the results back and synchronises.  pinned: the
        inputs and outputs are staged in page-locked memory (the returned arrays
        are views of it), which lets a large sorted frame go through as
        overlapping sector ranges."""
        import numpy as np
        n = int(len(sector))
        cap = int(capacity) if capacity is not None else n // 10 + 1
        t = self.torch

        def empty(shape, dt):
            if not pinned:
                return np.empty(shape, dt)
            tdt = {np.uint16: t.int16, np.uint8: t.uint8, np.int32: t.int32, np.float32: t.float32}[dt]
            return t.empty(shape, dtype=tdt, pin_memory=True).numpy().view(dt)

        def host(a, dt):
            a = np.ascontiguousarray(a, dt)
            if not pinned:
                return a
            b = empty(a.shape, dt)
            b[...] = a
            return b

        hs = host(sector, np.uint16)
        hr = host(row, np.uint16)
        hp = host(pad, np.float32)
        ht = host(time, np.float32)
        out = {"cluster_track": empty(max(n, 1), np.int32), "params": empty((cap, 5), np.float32),
               "cov": empty((cap, 15), np.float32), "t_ref": empty(cap, np.float32),
               "x": empty(cap, np.float32), "chi2": empty(cap, np.float32), "ndf": empty(cap, np.int32),
               "nhits": empty(cap, np.int32), "first_cluster": empty(cap, np.int32),
               "sector": empty(cap, np.uint16), "row_first": empty(cap, np.uint16),
               "row_last": empty(cap, np.uint16), "status": empty(cap, np.uint8)}
        if self.cfg.follow == 2:
            out["next_track"] = empty(cap, np.int32)
        cnt = np.zeros(1, np.uint32)
        cl = tpc_clusters(n=n, flags=TPC_INPUT_SORTED if sorted_input else 0, sector=hs.ctypes.data,
                          row=hr.ctypes.data, pad=hp.ctypes.data, time=ht.ctypes.data)
        tr = tpc_tracks(cluster_track=out["cluster_track"].ctypes.data, track_capacity=cap,
                        n_tracks=cnt.ctypes.data, **{k: v.ctypes.data for k, v in out.items() if k != "cluster_track"})
        st = self.torch.cuda.current_stream(self.device).cuda_stream
        _check(tpc_track_timeframe_host(self.handle, cl, tr, st))
        self._n = n
        res = {k: v for k, v in out.items()}
        res["cluster_track"] = out["cluster_track"][:n]
        res["n_tracks"] = int(cnt[0])
        return res

    def autotune(self, sector, row, pad, time, sorted_input=True, capacity=None, trials=3):
        """(nb_tile, fit_variant) chosen by the library's autotuner; the tensor-core engine
        of the rescoring (pruned mode) is kept in self.mlp_engine."""
        cl, tr, n, cap = self.structs(sector, row, pad, time, sorted_input, capacity, host_count=None)
        tile, fit, self.mlp_engine = tpc_tf_autotune(self.handle, cl, tr, trials,
                                                     self.torch.cuda.current_stream(self.device).cuda_stream)
        return tile, fit

    def debug_links(self, stream=None):
        t = self.torch
        n = self._n
        d = self.device
        res = {k: t.empty(max(n, 1), dtype=t.int32, device=d) for k in ("order", "down", "up", "mup")}
        res["is_start"] = t.empty(max(n, 1), dtype=t.uint8, device=d)
        st = stream if stream is not None else t.cuda.current_stream(d)
        _check(tpc_tf_debug_links(self.handle, res["order"].data_ptr(), res["down"].data_ptr(),
                                  res["up"].data_ptr(), res["mup"].data_ptr(), res["is_start"].data_ptr(),
                                  st.cuda_stream))
        st.synchronize()
        return {k: v[:n] for k, v in res.items()}

    def stage_times(self):
        return tpc_tf_stage_times(self.handle)

    def load_mlp(self, blob: bytes):
        _check(tpc_mlp_load(self.handle, blob))

    def score(self, feat, engine=0):
        """Logits of raw feature rows (float32[m, 12] CUDA tensor); engine 0 = tcgen05, 1 = mma.sync."""
        t = self.torch
        m = int(feat.shape[0])
        out = t.empty(max(m, 1), dtype=t.float32, device=self.device)
        _check(load().tpc_mlp_score_ex(self.handle, feat.data_ptr(), m, out.data_ptr(), int(engine),
                                       t.cuda.current_stream(self.device).cuda_stream))
        return out[:m]

    def extract(self, sector, row, pad, time, sorted_input=True, cap=None):
        """Training rows of one frame: (features float32[M,12], labels uint8[M], tri int32[M,3])."""
        t = self.torch
        d = self.device
        n = int(sector.numel())
        cl = tpc_clusters(n=n, flags=TPC_INPUT_SORTED if sorted_input else 0, sector=sector.data_ptr(),
                          row=row.data_ptr(), pad=pad.data_ptr(), time=time.data_ptr())
        count = t.zeros(1, dtype=t.int32, device=d)
        st = t.cuda.current_stream(d).cuda_stream
        if cap is None:
            _check(tpc_mlp_extract(self.handle, cl, None, None, None, 0, count.data_ptr(), st))
            cap = int(count.item())
        feat = t.empty((max(cap, 1), MLP_IN), dtype=t.float32, device=d)
        label = t.empty(max(cap, 1), dtype=t.uint8, device=d)
        tri = t.empty((max(cap, 1), 3), dtype=t.int32, device=d)
        _check(tpc_mlp_extract(self.handle, cl, feat.data_ptr(), label.data_ptr(), tri.data_ptr(), cap,
                               count.data_ptr(), st))
        self._n = n
        m = min(int(count.item()), cap)
        _check(tpc_tf_status(self.handle, st))
        return feat[:m], label[:m], tri[:m]

    def remove_unassigned(self, sector, row, pad, time, cluster_track):
        """Hit removal: (sector, row, pad, time, track) of the clusters attached to a track, in input order."""
        t = self.torch
        d = self.device
        n = int(sector.numel())
        cl = tpc_clusters(n=n, flags=0, sector=sector.data_ptr(), row=row.data_ptr(), pad=pad.data_ptr(),
                          time=time.data_ptr())
        o = dict(sector=t.empty(max(n, 1), dtype=t.int16, device=d), row=t.empty(max(n, 1), dtype=t.int16, device=d),
                 pad=t.empty(max(n, 1), dtype=t.float32, device=d), time=t.empty(max(n, 1), dtype=t.float32, device=d),
                 track=t.empty(max(n, 1), dtype=t.int32, device=d))
        cnt = t.zeros(1, dtype=t.int32, device=d)
        st = t.cuda.current_stream(d).cuda_stream
        _check(load().tpc_tf_remove_unassigned(self.handle, ctypes.byref(cl), cluster_track.data_ptr(),
                                               o["sector"].data_ptr(), o["row"].data_ptr(), o["pad"].data_ptr(),
                                               o["time"].data_ptr(), o["track"].data_ptr(), cnt.data_ptr(), st))
        m = int(cnt.item())
        _check(tpc_tf_status(self.handle, st))
        return {k: v[:m] for k, v in o.items()}

    def pruned_clusters(self) -> int:
        """Clusters the classifier rescored in the last pruned call."""
        return sum(self.pruned_split())

    def pruned_split(self):
        """(from the tile regions, from the overflow list) of the last pruned call."""
        return tpc_tf_pruned_clusters(self.handle, self.torch.cuda.current_stream(self.device).cuda_stream)

    def launches_per_call(self) -> int:
        return tpc_tf_launches_per_call(self.handle)
