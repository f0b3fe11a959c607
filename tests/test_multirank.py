"""The benchmark's multi-GPU logic on CPU with two gloo ranks: each rank
solves its own independent problem (distinct seeds, weak scaling); the job
time is the maximum over ranks and the work is summed.  The only
communication is this host-side control; the walks exchange nothing."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 0.5 * (rank + 1)]
    counts = [10 * (rank + 1), 7]
    t, c = bench.combine_ranks(times, counts, dist, "cpu")
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([bench.rank_seed(rank)], dtype=torch.int64))
    out[rank] = (t, c, [int(x) for x in seeds])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_combine_max_time_and_sum_work():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, c, seeds = out[r]
        assert t == [2.0, 1.0]           # max over ranks
        assert c == [30.0, 14.0]         # sum over ranks
        assert len(set(seeds)) == world  # independent problems
    # whole-job throughput = summed work / slowest rank
    t, c, _ = out[0]
    assert c[0] / t[0] == 15.0


def test_single_process_needs_no_collective():
    import bench
    t, c = bench.combine_ranks([3.0], [9], None, "cpu")
    assert t == [3.0] and c == [9.0]
