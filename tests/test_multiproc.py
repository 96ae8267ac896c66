"""The host side of runs on several GPUs, with two or five gloo ranks on the CPU.

Each rank tracks its own contiguous block of sectors of one frame (the oracle
stands in for the rank's GPU: the library's result for a sector subset equals
the oracle's, which the GPU parity tests check); the ranks exchange only their
track counts, offset their track ids by the exclusive scan and gather the
assignment: the union must equal one call over the whole frame, cluster for
cluster.  The job totals take the slowest rank's time and the sum of units."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2102_08862_gb300 import multigpu as mg


def test_sector_shards_cover_the_sectors_once():
    for world in (1, 2, 3, 4, 5, 8, 36):
        blocks = [mg.sector_shard(r, world) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == 36
        assert all(blocks[k][1] == blocks[k + 1][0] for k in range(world - 1))
        sizes = [hi - lo for lo, hi in blocks]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        mg.sector_shard(2, 2)
    with pytest.raises(ValueError):
        mg.sector_shard(0, 2, follow=2)
    assert mg.sector_shard(0, 1, follow=2) == (0, 36)


def test_track_id_offsets_are_the_exclusive_scan():
    assert mg.track_id_offsets([5, 0, 7, 2]).tolist() == [0, 5, 5, 12]
    assert mg.global_track_ids(np.array([-1, 0, 3]), 10).tolist() == [-1, 10, 13]
    assert mg.job_totals(None, 2.5, 7) == (2.5, 7.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import tpcsynth as ts
        f = ts.generate(ts.continuous(0.3, 77))
        lo, hi = mg.sector_shard(rank, world)
        mine = np.nonzero((f.sector >= lo) & (f.sector < hi))[0]
        res = oracle.track(f.sector[mine], f.row[mine], f.pad[mine], f.time[mine])
        counts = mg.gather_track_counts(dist, res["n_tracks"])
        ct = mg.global_track_ids(res["cluster_track"], int(mg.track_id_offsets(counts)[rank]))
        pieces = [None] * world
        dist.all_gather_object(pieces, (mine, ct))
        slowest, units = mg.job_totals(dist, 1.5 + rank, 10.0 * (rank + 1))
        assert slowest == 1.5 + (world - 1) and units == 10.0 * world * (world + 1) / 2
        if rank == 0:
            merged = np.full(f.n, -7, np.int32)
            for idx, c in pieces:
                merged[idx] = c
            whole = oracle.track(f.sector, f.row, f.pad, f.time)
            assert int(counts.sum()) == whole["n_tracks"] > 100
            assert np.array_equal(merged, whole["cluster_track"])
            open(os.path.join(out_dir, "ok"), "w").write(f"{whole['n_tracks']} tracks from {world} shards\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 5])  # 18/18 and 8/7/7/7/7 sectors
def test_ranks_merge_to_the_whole_frame(tmp_path, world):
    import torch.multiprocessing as mp
    import oracle
    import tpcsynth as ts
    oracle.build()  # built once here, not raced by the spawned ranks
    ts.build()
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    assert (tmp_path / "ok").read_text().endswith(f"from {world} shards\n")
