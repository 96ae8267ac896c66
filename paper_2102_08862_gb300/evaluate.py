"""Tracking quality against generator truth (host-side measurement, not part of
the tracking path).

A track's label is the most frequent generator label of its clusters (ties go to
the smaller label; noise clusters carry -1).  A track is matched when that label
is a real generator track and holds at least `match_frac` of its clusters.
Findable = a (generator track, sector) pair with at least `min_findable`
clusters.  Efficiency = findable pairs matched by at least one track / findable;
clone rate = (matched tracks on findable pairs - findable pairs matched) /
findable; fake rate = unmatched tracks / tracks."""
from __future__ import annotations

import numpy as np

NSECT = 36


def evaluate(label, sector, cluster_track, n_tracks: int, n_gen_tracks: int, min_findable: int = 30,
             match_frac: float = 0.9) -> dict:
    label = np.asarray(label, np.int64)
    sector = np.asarray(sector, np.int64)
    ct = np.asarray(cluster_track, np.int64)
    n_tracks = int(n_tracks)
    real = label >= 0
    pair_cnt = np.bincount(label[real] * NSECT + sector[real], minlength=n_gen_tracks * NSECT)
    findable = pair_cnt >= min_findable
    n_findable = int(findable.sum())
    on = ct >= 0
    t_of, l_of, s_of = ct[on], label[on], sector[on]
    nhits = np.bincount(t_of, minlength=n_tracks)
    # count of each (track, label) combination; labels shifted by 1 so noise is 0
    key = t_of * (n_gen_tracks + 1) + (l_of + 1)
    uk, uc = np.unique(key, return_counts=True)
    ut, ul = uk // (n_gen_tracks + 1), uk % (n_gen_tracks + 1) - 1
    # per track: largest count, smallest label among the largest (uk is sorted by track, then label)
    order = np.lexsort((ul, -uc, ut))
    first = np.ones(order.size, bool)
    first[1:] = ut[order][1:] != ut[order][:-1]
    best = order[first]
    tr_label = np.full(n_tracks, -1, np.int64)
    tr_count = np.zeros(n_tracks, np.int64)
    tr_label[ut[best]] = ul[best]
    tr_count[ut[best]] = uc[best]
    tr_sector = np.zeros(n_tracks, np.int64)
    tr_sector[t_of] = s_of
    matched = (tr_label >= 0) & (nhits > 0) & (tr_count >= match_frac * nhits)
    pidx = np.where(matched, tr_label * NSECT + tr_sector, 0)
    on_findable = matched & findable[pidx]
    found = np.zeros(findable.size, bool)
    found[pidx[on_findable]] = True
    n_found = int(found.sum())
    n_fake = int((~matched).sum())
    return dict(n_findable=n_findable, n_findable_found=n_found, n_matched_findable_tracks=int(on_findable.sum()),
                n_fake=n_fake, n_tracks=n_tracks,
                efficiency=n_found / n_findable if n_findable else 0.0,
                clone_rate=(int(on_findable.sum()) - n_found) / n_findable if n_findable else 0.0,
                fake_rate=n_fake / n_tracks if n_tracks else 0.0)
