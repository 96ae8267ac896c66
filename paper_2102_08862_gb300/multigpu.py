"""Host-side logic of runs on several GPUs of one node (one process per GPU).

The tracking path shards with no collective on the data path: time frames are
independent, and so are the 36 sectors of one frame as long as cross-sector
links are off (no cluster of one sector is linked to another's by the seeding,
the chains or the fit).  With follow = 2 the follower links tracks across sector
boundaries, so a sector-sharded frame would lose the links that cross a shard
boundary: `sector_shard` refuses that mode, and such frames are sharded whole.  Every rank tracks
its own frames, or its own contiguous block of sectors of a shared frame; the
only exchange is on the host:
  * step times reduced by maximum and unit counts by sum (whole-job throughput
    = units of all ranks / the slowest rank's time);
  * with sectors split over ranks, the exclusive scan of the per-rank track
    counts, which offsets each rank's track ids so that the union numbers the
    tracks exactly as one call over the whole frame would (track ids follow the
    start cluster's order, which is sector-major).
`dist` is torch.distributed after init_process_group (NCCL on GPUs, gloo on CPU
for the tests), or None for a single process."""
from __future__ import annotations

import numpy as np

NSECT = 36


def sector_shard(rank: int, world: int, nsect: int = NSECT, follow: int = 0) -> tuple[int, int]:
    """Contiguous block [lo, hi) of sectors for this rank (sizes differ by one at
    most).  `follow` is the tracker's follow mode: with cross-sector links
    (follow = 2) sectors are not independent and a frame cannot be split."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    if follow == 2 and world > 1:
        raise ValueError("cross-sector links (follow = 2) join neighbouring sectors: shard whole frames instead")
    base, extra = divmod(nsect, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def track_id_offsets(counts) -> np.ndarray:
    """Exclusive scan of per-rank track counts: the first id of each rank's tracks."""
    c = np.asarray(counts, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(c)[:-1]]).astype(np.int64)


def job_totals(dist, ms: float, units: float, device=None) -> tuple[float, float]:
    """(maximum step time over ranks, sum of units over ranks)."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather_track_counts(dist, n_tracks: int, device=None) -> np.ndarray:
    """Every rank's track count, in rank order."""
    if dist is None:
        return np.array([n_tracks], dtype=np.int64)
    import torch
    world = dist.get_world_size()
    mine = torch.tensor([int(n_tracks)], dtype=torch.int64, device=device)
    allc = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(allc, mine)
    return np.array([int(x.item()) for x in allc], dtype=np.int64)


def global_track_ids(local_cluster_track: np.ndarray, offset: int) -> np.ndarray:
    """Local track ids of one rank's clusters turned into the whole frame's (-1 stays)."""
    ct = np.asarray(local_cluster_track)
    return np.where(ct >= 0, ct + offset, -1).astype(np.int32)
