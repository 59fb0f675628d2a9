"""The multi-process path on CPU (gloo, world size 2): series sharding covers
every series exactly once, each rank's shard computed separately equals the
single-process result, and the timing reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest

import hos_synth
from paper_1805_11775_gb300.shard import max_over_ranks, series_shard, shard_arrays


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
