"""The multi-GPU path is replicas only: nodes are independent, every rank solves
its own share, and the only cross-rank operations are the timing barrier and the
max over ranks of the elapsed time.  This checks that host logic with two gloo
ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank's own elapsed time; the job takes the slowest
    ms = 100.0 + 25.0 * rank
    dist.barrier()
    ms_max = bench.max_over_ranks(ms, dist, device="cpu")
    nodes = list(range(37))
    mine = bench.shard(nodes, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    rate = bench.whole_job_rate(4, world, ms_max)
    out[rank] = (ms_max, gathered, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        ms_max, gathered, rate = out[r]
        assert ms_max == 125.0                      # max over ranks
        flat = sorted(x for part in gathered for x in part)
        assert flat == list(range(37))              # shards disjoint and complete
        assert abs(rate - 4 * 2 / 0.125) < 1e-9     # all units / slowest rank's time


def test_single_rank_helpers_without_a_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.shard(list(range(5)), 0, 1) == [0, 1, 2, 3, 4]
    assert bench.whole_job_rate(8, 1, 2000.0) == 4.0
