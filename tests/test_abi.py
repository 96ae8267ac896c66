"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
function include/tpcca.h declares, and the ctypes structs match the C layout."""
import ctypes
import os
import subprocess

import numpy as np

import pytest

from paper_2102_08862_gb300 import _build, tpcca

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return tpcca.load()


def test_exports_every_declared_function(lib):
    names = tpcca.header_functions()
    assert {"tpc_tf_create", "tpc_track_timeframe", "tpc_tf_destroy", "tpc_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "tpcca.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("tpc_tf_config %zu\ntpc_clusters %zu\ntpc_tracks %zu\n", sizeof(tpc_tf_config), sizeof(tpc_clusters),
         sizeof(tpc_tracks));
  F(tpc_tf_config, cost_max_q); F(tpc_tf_config, tau); F(tpc_tf_config, row_cap); F(tpc_tf_config, follow_chi2);
  F(tpc_tf_config, follow_check); F(tpc_tf_config, follow_link_rows); F(tpc_tf_config, mlp_engine); F(tpc_tf_config, persistent);
  F(tpc_tracks, next_track);
  F(tpc_clusters, time); F(tpc_tracks, params); F(tpc_tracks, status); F(tpc_tracks, n_tracks_host);
  printf("tpc_mlp_train_config %zu\n", sizeof(tpc_mlp_train_config));
  F(tpc_mlp_train_config, pos_weight); F(tpc_mlp_train_config, max_batch); F(tpc_mlp_train_config, device); F(tpc_mlp_train_config, engine);
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True,
                                                                 text=True).stdout.splitlines())
    assert int(vals["tpc_tf_config"]) == ctypes.sizeof(tpcca.tpc_tf_config)
    assert int(vals["tpc_clusters"]) == ctypes.sizeof(tpcca.tpc_clusters)
    assert int(vals["tpc_tracks"]) == ctypes.sizeof(tpcca.tpc_tracks)
    assert int(vals["tpc_mlp_train_config"]) == ctypes.sizeof(tpcca.tpc_mlp_train_config)
    for key, v in vals.items():
        if "." in key:
            struct, member = key.split(".")
            assert getattr(getattr(tpcca, struct), member).offset == int(v), key


def test_defaults_and_argument_errors(lib):
    c = tpcca.tpc_default_config()
    assert (c.wy_q, c.wt_q, c.cost_max_q, c.n_min) == (1280000, 384, 384000 ** 2, 10)
    # invalid configurations are rejected before any device call
    c.max_clusters = 0
    h = ctypes.c_void_p()
    assert lib.tpc_tf_create(ctypes.byref(c), ctypes.byref(h)) == tpcca.TPC_ERR_ARG
    assert "max_clusters" in tpcca.tpc_last_error()
    c.max_clusters = 100
    c.n_min = 2
    assert lib.tpc_tf_create(ctypes.byref(c), ctypes.byref(h)) == tpcca.TPC_ERR_ARG
    assert lib.tpc_tf_create(None, ctypes.byref(h)) == tpcca.TPC_ERR_ARG
    c.n_min = 10
    for k, v in (("follow", 3), ("follow_chi2", 0.0), ("follow_miss", 0), ("follow_check", 153),
                 ("follow_link_chi2", -1.0), ("follow_link_rows", 0)):
        d = tpcca.tpc_default_config()
        d.max_clusters, d.follow = 100, 2
        assert (d.follow_chi2, d.follow_miss, d.follow_check) == (16.0, 3, 4)
        assert (d.follow_link_chi2, d.follow_link_rows) == (80.0, 152)
        setattr(d, k, v)
        assert lib.tpc_tf_create(ctypes.byref(d), ctypes.byref(h)) == tpcca.TPC_ERR_ARG, k
        assert "follow" in tpcca.tpc_last_error()
    for k, v in (("persistent", 2), ("mode", tpcca.TPC_MODE_PRUNED), ("follow", 1)):
        d = tpcca.tpc_default_config()
        d.max_clusters, d.persistent = 100, 1
        setattr(d, k, v)
        assert lib.tpc_tf_create(ctypes.byref(d), ctypes.byref(h)) == tpcca.TPC_ERR_ARG, k
        assert "persistent" in tpcca.tpc_last_error()
    assert lib.tpc_track_timeframe(None, None, None, None) == tpcca.TPC_ERR_ARG
    assert lib.tpc_tf_status(None, None) == tpcca.TPC_ERR_ARG
    lib.tpc_tf_destroy(None)


def test_no_oracle_in_product_path():
    """The CUDA path must not import, link or call the oracle."""
    pkg = os.path.join(ROOT, "paper_2102_08862_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "oracle.h" not in txt, f


def test_classifier_blob_roundtrip_and_size(lib):
    rng = np.random.default_rng(0)
    mean, inv_std = rng.standard_normal(12), rng.random(12)
    theta = rng.standard_normal(tpcca.MLP_NPARAM)
    blob = tpcca.pack_blob(mean, inv_std, theta)
    assert len(blob) == tpcca.tpc_mlp_blob_bytes() == 20340
    m, s, t = tpcca.unpack_blob(blob)
    assert np.array_equal(m, mean.astype(np.float32)) and np.array_equal(t, theta.astype(np.float32))
    assert len(tpcca.init_blob(3)) == 20340
    with pytest.raises(ValueError):
        tpcca.unpack_blob(b"XXXX" + blob[4:])


def test_server_admission_policy(lib):
    """The serving runtime's admission rule on hand-built slot states (host logic, no GPU)."""
    G = 1 << 30
    adm = tpcca.tpc_server_admit
    # no slots: create one if it fits the budget, else wait
    assert adm(1000, [], [], [], 4, 10 * G, 2 * G) == (0, tpcca.TPC_ADMIT_CREATE)
    assert adm(1000, [], [], [], 4, 1 * G, 2 * G) == (-1, tpcca.TPC_ADMIT_WAIT)
    # the free slot of smallest sufficient capacity wins
    assert adm(500, [1000, 600, 400], [3 * G, 2 * G, G], [0, 0, 0], 4, 100 * G, G) == (1, tpcca.TPC_ADMIT_RUN)
    # a busy fitting slot is skipped; a new slot is made while the budget allows
    assert adm(500, [1000, 400], [3 * G, G], [1, 0], 4, 100 * G, 2 * G) == (2, tpcca.TPC_ADMIT_CREATE)
    # at max_slots: replace the largest free slot (too small) if the budget allows
    assert adm(500, [1000, 400, 300], [3 * G, G, G // 2], [1, 0, 0], 3, 100 * G, 2 * G) == \
        (1, tpcca.TPC_ADMIT_REPLACE)
    # budget exhausted and the only fitting slot busy: wait
    assert adm(500, [1000, 400], [3 * G, G], [1, 0], 4, 4 * G, 2 * G) == (-1, tpcca.TPC_ADMIT_WAIT)
    # everything busy: wait
    assert adm(10, [1000, 1000], [G, G], [1, 1], 2, 100 * G, G) == (-1, tpcca.TPC_ADMIT_WAIT)


def test_arena_estimate_grows_with_clusters(lib):
    c = tpcca.tpc_default_config()
    c.max_clusters = 1 << 20
    small = tpcca.tpc_tf_arena_bytes(c)
    c.max_clusters = 1 << 24
    big = tpcca.tpc_tf_arena_bytes(c)
    assert big > 10 * small
    c.mode = tpcca.TPC_MODE_PRUNED
    assert tpcca.tpc_tf_arena_bytes(c) > big  # the pair regions and the overflow list


def test_noalloc_rejects_misaligned_arrays_before_any_launch(lib):
    """The allocation-free entry point checks the alignment of every array on the
    host and returns TPC_ERR_ARG without touching the device (this runs without a
    GPU: any device call here would fail with TPC_ERR_CUDA instead)."""
    base = 0x10000
    good = dict(sector=base, row=base + 0x1000, pad=base + 0x2000, time=base + 0x3000)
    cases = [("sector", 1), ("row", 1), ("pad", 2), ("time", 1)]
    for field, off in cases:
        kw = dict(good)
        kw[field] += off
        cl = tpcca.tpc_clusters(n=100, flags=tpcca.TPC_INPUT_SORTED, **kw)
        tr = tpcca.tpc_tracks(cluster_track=base + 0x4000, track_capacity=0, n_tracks=base + 0x5000)
        assert lib.tpc_track_timeframe_noalloc(None, ctypes.byref(cl), ctypes.byref(tr), None) == tpcca.TPC_ERR_ARG
        assert "misaligned" in tpcca.tpc_last_error(), field
    cl = tpcca.tpc_clusters(n=100, flags=tpcca.TPC_INPUT_SORTED, **good)
    for field in ("cluster_track", "params", "sector", "n_tracks"):
        kw = dict(cluster_track=base + 0x4000, track_capacity=16, n_tracks=base + 0x5000,
                  **{k: base + 0x6000 + 0x100 * i for i, k in enumerate(
                      ("params", "cov", "t_ref", "x", "chi2", "ndf", "nhits", "first_cluster", "sector",
                       "row_first", "row_last", "status"))})
        kw[field] += 1 if field == "sector" else 2
        tr = tpcca.tpc_tracks(**kw)
        assert lib.tpc_track_timeframe_noalloc(None, ctypes.byref(cl), ctypes.byref(tr), None) == tpcca.TPC_ERR_ARG
        assert "misaligned" in tpcca.tpc_last_error(), field


def test_debug_entry_points_check_arguments(lib):
    assert lib.tpc_tf_set_spin_limit(None, 4) == tpcca.TPC_ERR_ARG
    assert lib.tpc_tf_debug_wait(None, None) == tpcca.TPC_ERR_ARG
    assert lib.tpc_debug_quantize(0x10002, 8, 0x20000, None) == tpcca.TPC_ERR_ARG
    assert lib.tpc_debug_quantize(None, 8, 0x20000, None) == tpcca.TPC_ERR_ARG
    assert lib.tpc_debug_quantize(None, 0, None, None) == tpcca.TPC_OK
