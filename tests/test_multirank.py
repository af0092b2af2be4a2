"""Host-side logic of the multi-GPU bench (one replica per rank, no data-path collective):
world_size-2 gloo ranks on the CPU (no GPU needed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1010_1233_gb300 import workloads as W
        p = bench.rank_replica(W.d2q9_16384(64)["replicas"][0], rank)
        # rank 1 is slower: the job time must be the slowest rank's
        value, tmax = bench.job_throughput(64 * 64, 10, 1.0 + rank, world)
        q.put((rank, p["seed"], p["stream"], value, tmax))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    seeds = {r[1] for r in res}
    streams = {r[2] for r in res}
    assert len(seeds) == world and len(streams) == world         # independent noise per rank
    for _, _, _, value, tmax in res:
        assert tmax == 2.0                                        # max over ranks
        assert abs(value - world * 64 * 64 * 10 / 2.0 / 1e6) < 1e-12


def test_single_rank_no_collective():
    value, tmax = bench.job_throughput(100, 5, 0.5, 1)
    assert tmax == 0.5 and abs(value - 100 * 5 / 0.5 / 1e6) < 1e-15
