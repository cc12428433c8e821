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


def _split_worker(rank, world, port, q):
    """One plane's MG patches split by NEST bundle range: each rank solves
    its own bundles (the oracle's partial-sky solve of Sec. 3.4 on its range;
    no data-path collective, patches are independent) and the ranks' patch
    solutions, gathered, equal the whole plane's."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import binning, healpix as hp, mg as omg
        from workloads import synthetic
        nf, ns, lmax, nb, ncell = 32, 8, 16, 2, 16
        z, phi = synthetic.lognormal_particles(100_000, 41)
        kappa = binning.kappa_from_counts(binning.bin_counts(nf, z, phi), z.numel() / hp.npix(nf), 1.0)
        lo, hi = bench.bundle_range(nb, rank, world)
        mine = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, fixed_cycles=3, bundles=torch.arange(lo, hi))
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, mine["u"]))
        if rank == 0:
            full = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, fixed_cycles=3)
            u = torch.cat([p[2] for p in parts])
            cover = sum(p[1] - p[0] for p in parts)
            q.put((cover, float((u - full["u"]).abs().max()), [p[:2] for p in parts]))
        else:
            q.put(None)
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_one_plane_by_bundle_range():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cover, diff, ranges = [r for r in res if r is not None][0]
    assert cover == 48 and ranges == [(0, 24), (24, 48)]
    assert diff == 0.0


def test_bundle_ranges_cover_every_bundle_once():
    for nb in (1, 2, 32):
        for world in (1, 2, 3, 8):
            rs = [bench.bundle_range(nb, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == 12 * nb * nb
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1

