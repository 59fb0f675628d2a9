"""The multi-process path on CPU (gloo, world size 2 and 3): series sharding
covers every series exactly once, each rank's shard computed separately
equals the single-process result, the timing reduction takes the maximum,
and one long series cut into time slices with halos, joined by two FP64 sum
all-reduces (series total, then c3), gives the whole series' c3."""
import os
import socket

import numpy as np
import pytest

import hos_synth
from paper_1805_11775_gb300.shard import max_over_ranks, series_shard, shard_arrays, slice_with_halo, time_slices


def test_series_shard_partitions_and_balances():
    lens = hos_synth.intraday_lengths(97, 3)
    offs = np.zeros(98, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    for world in (1, 2, 3, 4, 8):
        ranges = [series_shard(offs, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 97
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0 and a0 <= a1
        loads = [offs[b] - offs[a] for a, b in ranges]
        assert max(loads) - min(loads) <= 2 * lens.max()
    assert series_shard(np.array([0]), 0, 4) == (0, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lens = np.array([300, 1200, 40, 800, 650, 999, 120], dtype=np.int64)
    vals, offs = hos_synth.student_t_returns(lens, 8)
    v, o, (s0, s1) = shard_arrays(vals, offs, rank, world)
    B = np.stack([oracle.bispectrum(v[o[s]:o[s + 1]], 6, 12) for s in range(o.size - 1)]) \
        if o.size > 1 else np.zeros((0, 12, 12), complex)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), B)
    np.save(os.path.join(out_dir, f"range{rank}.npy"), np.array([s0, s1]))
    t = max_over_ranks(1.0 + rank, dist)
    np.save(os.path.join(out_dir, f"tmax{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process(tmp_path, oracle):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    lens = np.array([300, 1200, 40, 800, 650, 999, 120], dtype=np.int64)
    vals, offs = hos_synth.student_t_returns(lens, 8)
    whole = np.stack([oracle.bispectrum(vals[offs[s]:offs[s + 1]], 6, 12) for s in range(lens.size)])
    parts = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    ranges = [tuple(np.load(tmp_path / f"range{r}.npy")) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == lens.size
    np.testing.assert_array_equal(np.concatenate(parts), whole)
    assert all(float(np.load(tmp_path / f"tmax{r}.npy")[0]) == 2.0 for r in range(world))


def test_time_slices_cover_the_series_with_halos():
    for n, world, L in [(1000, 1, 8), (1000, 3, 8), (97, 4, 30), (10, 8, 4), (5, 3, 9)]:
        sl = time_slices(n, world, L)
        assert sl[0][0] == 0 and sl[-1][1] == n
        for (a0, b0, _, _), (a1, _, _, _) in zip(sl, sl[1:]):
            assert b0 == a1
        for a, b, hb, ha in sl:
            assert a <= b and hb == min(L, a) and ha == min(L, n - b)
    x = np.arange(50.0)
    piece, hb, ha = slice_with_halo(x, 1, 3, 4)
    a, b, _, _ = time_slices(50, 3, 4)[1]
    np.testing.assert_array_equal(piece, x[a - 4:b + 4])
    assert (hb, ha) == (4, 4)


def _slice_share(xh, hb, ha, mean, L, n_total):
    """(1/n) sum over the slice's i of y(i)y(i+w1)y(i+w2), y = x - mean on the
    window xh, zero outside it, as [w2 + L, w1 + L] (lags in [-L, L-1])."""
    y = xh - mean
    m = y.size
    idx = np.arange(hb, m - ha)
    out = np.zeros((2 * L, 2 * L))
    for w1 in range(-L, L):
        j1 = idx + w1
        y1 = np.where((j1 >= 0) & (j1 < m), y[np.clip(j1, 0, m - 1)], 0.0)
        for w2 in range(-L, L):
            j2 = idx + w2
            y2 = np.where((j2 >= 0) & (j2 < m), y[np.clip(j2, 0, m - 1)], 0.0)
            out[w2 + L, w1 + L] = np.sum(y[idx] * y1 * y2) / n_total
    return out


def _slice_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = hos_synth.ar2(701, 31)
    L = 6
    xh, hb, ha = slice_with_halo(x, rank, world, L)
    tot = torch.tensor([np.sum(xh[hb:xh.size - ha])], dtype=torch.float64)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    c3 = torch.from_numpy(_slice_share(xh, hb, ha, float(tot[0]) / x.size, L, x.size))
    dist.all_reduce(c3, op=dist.ReduceOp.SUM)
    np.save(os.path.join(out_dir, f"c3_{rank}.npy"), c3.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_time_sliced_ranks_sum_to_the_whole_series_c3(tmp_path, oracle, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_slice_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    x = hos_synth.ar2(701, 31)
    L = 6
    ref = oracle.c3(oracle.demean(x), L)[:2 * L, :2 * L].T  # [w2 + L, w1 + L]
    for r in range(world):
        got = np.load(tmp_path / f"c3_{r}.npy")
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _slice_moments(xh, hb, ha, mean, L, n_total):
    """(1/n) sums over the slice's own i of y(i)y(i+w1)y(i+w2)y(i+w3) over
    [-L, L-1]^3 and of y(i)y(i+t), t in [0, 2L-1], y = x - mean on the window
    xh (zero outside it)."""
    y = xh - mean
    m = y.size
    idx = np.arange(hb, m - ha)

    def lagged(w):
        j = idx + w
        return np.where((j >= 0) & (j < m), y[np.clip(j, 0, m - 1)], 0.0)

    ys = {w: lagged(w) for w in range(-L, 2 * L)}
    m4 = np.zeros((2 * L,) * 3)
    for w1 in range(-L, L):
        for w2 in range(-L, L):
            p = y[idx] * ys[w1] * ys[w2]
            for w3 in range(-L, L):
                m4[w1 + L, w2 + L, w3 + L] = np.sum(p * ys[w3]) / n_total
    c2 = np.array([np.sum(y[idx] * ys[t]) / n_total for t in range(2 * L)])
    return m4, c2


def _slice4_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = hos_synth.ma(333, 32)
    L = 3
    xh, hb, ha = slice_with_halo(x, rank, world, L, halo_after=2 * L)
    tot = torch.tensor([np.sum(xh[hb:xh.size - ha])], dtype=torch.float64)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    m4, c2 = _slice_moments(xh, hb, ha, float(tot[0]) / x.size, L, x.size)
    m4t, c2t = torch.from_numpy(m4), torch.from_numpy(c2)
    dist.all_reduce(m4t, op=dist.ReduceOp.SUM)
    dist.all_reduce(c2t, op=dist.ReduceOp.SUM)
    np.save(os.path.join(out_dir, f"m4_{rank}.npy"), m4t.numpy())
    np.save(os.path.join(out_dir, f"c2_{rank}.npy"), c2t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_time_sliced_ranks_give_the_whole_series_c4(tmp_path, oracle, world):
    """Slices with an L-sample halo before and 2L after, joined by FP64 sum
    all-reduces of the total, of m4 and of c2 (lags >= 0; c2 is even), give
    the whole series' c4 = m4 - three c2 c2 products."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_slice4_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    x = hos_synth.ma(333, 32)
    L = 3
    ref = oracle.c4(oracle.demean(x), L)[:2 * L, :2 * L, :2 * L]
    for r in range(world):
        m4 = np.load(tmp_path / f"m4_{r}.npy")
        c2p = np.load(tmp_path / f"c2_{r}.npy")
        c2 = lambda t: c2p[abs(t)]  # noqa: E731
        c4 = np.empty_like(m4)
        for w1 in range(-L, L):
            for w2 in range(-L, L):
                for w3 in range(-L, L):
                    c4[w1 + L, w2 + L, w3 + L] = (m4[w1 + L, w2 + L, w3 + L] - c2(w1) * c2(w3 - w2)
                                                  - c2(w2) * c2(w3 - w1) - c2(w3) * c2(w2 - w1))
        assert np.abs(c4 - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fourth_order_time_slices_reach_2L_after():
    for n, world, L in [(1000, 3, 8), (97, 4, 30), (10, 8, 4)]:
        for a, b, hb, ha in time_slices(n, world, L, halo_after=2 * L):
            assert hb == min(L, a) and ha == min(2 * L, n - b)
