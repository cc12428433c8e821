"""The benchmark's multi-rank host logic at world size 2 on CPU (gloo).

Planes are independent problems: under torchrun every rank solves its own
synthetic plane (its own seed) with no data-path collective, the job's time
is the slowest rank's (a MAX reduction over ranks) and the whole-job rate
counts every rank's planes over that time."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.plane_seed(bench.WORKLOADS["shtmg_plane_nside2048"], rank))
        q.put((rank, ms, seeds, bench.whole_job_rate(world, 5, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_the_slowest_rank_on_distinct_planes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, seeds, rate in res:
        assert ms == 150.0
        assert seeds == [1210002, 1210003]
        assert abs(rate - 2 * 5 / 0.150) < 1e-9


def test_single_process_keeps_its_own_time():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(123.5, "cpu") == 123.5
    assert bench.whole_job_rate(1, 5, 250.0) == 20.0
