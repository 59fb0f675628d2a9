"""Host-side work split across ranks (one process per GPU).

The estimator shards naturally.  Independent series go to different ranks
with no data-path collective (weak scaling): ``series_shard`` gives each
rank a contiguous run of series whose total length is as even as the series
boundaries allow.  One long series is cut in time (``time_slices``): c3, m4
and c2 are sums over time, so each rank sums its slice (with an L-sample
halo before it and L, or 2L for the fourth order, after) and FP64
all-reduces (the series' sum for the mean, then c3, or m4 and c2) join
them.  ``max_over_ranks`` is the timing reduction the benchmark reports.
"""
from __future__ import annotations

import numpy as np


def series_shard(offsets, rank: int, world: int):
    """Contiguous series range [s0, s1) of ``rank``: the cut points are the
    series boundaries closest to equal shares of the total sample count."""
    offs = np.asarray(offsets, dtype=np.int64)
    S = offs.size - 1
    if world <= 1 or S == 0:
        return 0, S
    total = int(offs[-1] - offs[0])
    cuts = [0]
    for r in range(1, world):
        target = offs[0] + (total * r) // world
        s = int(np.searchsorted(offs, target, side="left"))
        if s > 0 and abs(int(offs[s - 1]) - target) <= abs(int(offs[min(s, S)]) - target):
            s -= 1
        cuts.append(max(cuts[-1], min(s, S)))
    cuts.append(S)
    return cuts[rank], cuts[rank + 1]


def time_slices(n: int, world: int, L: int, halo_after: int | None = None):
    """Cut one series of n samples into ``world`` contiguous time slices for
    the cumulant's sum over time: [(a, b, halo_before, halo_after)] per
    rank, slices [a, b) covering [0, n) in order, halos of up to L samples
    (fewer at the series' ends) that the lags w in [-L, L-1] reach.  The
    fourth order's c2 lags reach 2L - 1 after a sample: pass
    ``halo_after=2 * L``."""
    after = L if halo_after is None else halo_after
    out = []
    for r in range(world):
        a, b = (n * r) // world, (n * (r + 1)) // world
        out.append((a, b, min(L, a), min(after, n - b)))
    return out


def slice_with_halo(x, rank: int, world: int, L: int, halo_after: int | None = None):
    """(x[a - halo_before : b + halo_after], halo_before, halo_after) of ``rank``."""
    a, b, hb, ha = time_slices(len(x), world, L, halo_after)[rank]
    return x[a - hb:b + ha], hb, ha


def shard_arrays(values, offsets, rank: int, world: int):
    """(values, offsets) of this rank's series, offsets rebased to 0."""
    offs = np.asarray(offsets, dtype=np.int64)
    s0, s1 = series_shard(offs, rank, world)
    v = values[offs[s0]:offs[s1]]
    return v, offs[s0:s1 + 1] - offs[s0], (s0, s1)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over the ranks of the default process group (the
    benchmark's step time); the value itself when not distributed."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
