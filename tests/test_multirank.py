"""The multi-rank host logic of the benchmark on CPU (gloo, two ranks): each
rank runs its own shard of independent jobs with no data exchange, and the
job's time is the slowest rank's, its work the sum of all ranks'. One GPU per
rank on a GPU machine; here the ranks are CPU processes."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = bench.shard(64, rank, world)
        ms, units = bench.reduce_over_ranks(10.0 + rank, 1000.0 * (rank + 1), world)
        q.put((rank, mine, ms, units))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_jobs_and_reduce_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    shards = [o[1] for o in out]
    # every job on exactly one rank, balanced
    assert sorted(shards[0] + shards[1]) == list(range(64))
    assert len(shards[0]) == len(shards[1]) == 32
    for _, _, ms, units in out:
        assert ms == 11.0            # the slowest rank's time
        assert units == 3000.0       # all ranks' work


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(5.0, 7.0, 1) == (5.0, 7.0)
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
