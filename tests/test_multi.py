"""Work sharing across ranks (host logic; the data path has no exchange):
contiguous shards, the ragged partition by cost, and the max-over-ranks
timing, the last over a real two-process gloo group on the CPU."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1404_1810_gb300.multi import max_over_ranks, partition_ragged, shard


@pytest.mark.parametrize("total,world", [(0, 1), (1, 2), (7, 3), (4096, 8), (4097, 8), (5, 8)])
def test_shards_cover_the_batch(total, world):
    got = [shard(total, world, r) for r in range(world)]
    assert sum(c for _, c in got) == total
    nxt = 0
    for first, count in got:
        assert first == nxt
        nxt = first + count
    counts = [c for _, c in got]
    assert max(counts) - min(counts) <= 1


def test_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard(10, 0, 0)
    with pytest.raises(ValueError):
        shard(10, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_ragged_partition_is_exact_and_balanced(world):
    lg = synth.ragged_log2n(20000, 4, 18)
    parts = partition_ragged(lg, world)
    allidx = np.concatenate(parts)
    assert np.array_equal(np.sort(allidx), np.arange(len(lg)))
    cost = (np.int64(1) << lg.astype(np.int64)) * lg.astype(np.int64)
    loads = np.array([cost[p].sum() for p in parts])
    # LPT is within one largest item of the ideal share
    assert loads.max() - loads.sum() / world <= cost.max()
    assert partition_ragged(lg, world)[0].tolist() == parts[0].tolist()   # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shard(4097, world, rank)
        lg = synth.ragged_log2n(1000, 4, 18)
        mine = partition_ragged(lg, world)[rank]
        t = max_over_ranks(1.5 + rank)             # each rank's "time"
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{first} {count} {len(mine)} {t}\n")
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_group(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    assert [int(r[0]) for r in rows] == [0, 2049]
    assert sum(int(r[1]) for r in rows) == 4097
    assert sum(int(r[2]) for r in rows) == 1000
    assert all(float(r[3]) == 2.5 for r in rows)   # the maximum, seen by every rank


def test_max_over_ranks_without_a_group():
    assert max_over_ranks(3.25) == 3.25
