"""The multi-rank plan on CPU (host logic only, not a test of the library
across ranks): two gloo ranks each take their shard of instances by global
index (bench.py's plan), compute it with the oracle, and all-gather; the
union equals one rank computing everything, and the timing reduction takes
the slowest rank.  The library's own sharded handles (rng_create_shard) are
checked against one handle on a single GPU in the -m gpu tests."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SEED = 0x0123456789ABCDEF
CASES = [(0, 0, 256), (3, 0, 256), (5, 2, 256), (0, 1, 256), (2, 0, 64), (6, 0, 4)]  # (kind, flags, n per rank)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    results = []
    for kind, flags, per in CASES:
        first, count, total = bench.shard_range(rank, world, per)
        mine = O.generate(kind, SEED, total, 9, flags=flags, i_lo=first, i_hi=first + count)
        t = torch.from_numpy(mine.astype(np.int64))
        parts = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(parts, t)
        results.append(torch.cat(parts).numpy())
    slowest = bench.max_over_ranks(float(rank + 1) * 10.0, dist)
    if rank == 0:
        np.save(os.path.join(outdir, "gathered.npy"), np.array(results, dtype=object), allow_pickle=True)
        np.save(os.path.join(outdir, "slowest.npy"), np.array([slowest]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_reassemble_the_whole(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    import oracle as O
    for (kind, flags, per), got in zip(CASES, gathered):
        whole = O.generate(kind, SEED, world * per, 9, flags=flags)
        assert np.array_equal(got.astype(np.uint32), whole), (kind, flags)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 20.0
