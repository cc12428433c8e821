#!/usr/bin/env python3
"""Throughput of the lens-plane hot path on GB300: lens planes per second.

One step = one lens plane through the whole path of the paper's Sec. 3:
bin the plane's particles to HEALPix pixels (Sec. 3.2), build its source
kappa^(m) (Eq. lenspoisson), solve for the potential with the SHT+MG solver
(SHT at nside_sht / lmax, FAS multigrid V-cycles on all bundle patches to
the residual tolerance, Sec. 3.2), then put every ray of the Nside-2048 grid
on the plane and advance it to the next one (lens-field lookup, Eq. Atraj,
Eq. betaprop, Eq. posprop, Appendix B transport).

Default workload (single plane, SHT+MG, Nside 2048): a seeded lognormal
light-cone shell Poisson-sampled to 5e7 particles, nside_sht 512, lmax 1024,
bundle Nside 32 (12288 patches of 256^2 cells), tolerance 1e-10, FP64, and
50,331,648 rays.  All inputs are larger than L2, so no flush is needed.

  python bench.py [--gpus N --steps K --warmup W] [--precision fp64|fp32]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

Under torchrun every rank solves its own plane (independent seeds; weak
scaling) and rank 0 prints one JSON line with the whole-job planes/s.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import cosmology, synthetic  # noqa: E402

METRIC = "lens planes/s (SHT+MG, Nside=2048)"
UNIT = "planes/s"

WORKLOADS = {
    # the single-plane SHT+MG configuration the metric is quoted on
    "shtmg_plane_nside2048": dict(nside=2048, particles=50_000_000, nside_sht=512, lmax=1024, nside_bundle=32,
                                  ncell=256, tol=1e-10, nu1=2, nu2=2, max_cycles=60, seed=1210002),
    # a small case of the same kernels (profiling)
    "shtmg_plane_nside512": dict(nside=512, particles=3_000_000, nside_sht=128, lmax=256, nside_bundle=8,
                                 ncell=256, tol=1e-10, nu1=2, nu2=2, max_cycles=60, seed=1210002),
}

# batches of pure-SHT plane solves of mixed size (mixed precision, one plan:
# persistent launches over every plane, CUDA graph, autotuned launch shapes)
BATCH_WORKLOADS = {
    "sht_batch_mixed_sizes": dict(sizes=[(512, 1024)] * 32 + [(1024, 2048)] * 24 + [(2048, 4096)] * 8,
                                  seed=1210004, fp64_sample=2),
    "sht_batch_small": dict(sizes=[(128, 256)] * 8 + [(256, 512)] * 4, seed=1210004, fp64_sample=2),
    # one full class (21 planes with derivatives) at Nside 512: the profiling case of the batch kernels
    "sht_batch_nside512": dict(sizes=[(512, 1024)] * 21, seed=1210004, fp64_sample=1),
}
# adaptive Epanechnikov smoothing of the plane's particles (Sec. 3.2) at the
# benchmark plane's size, sigma = 2.5 pixel scales
SMOOTH_WORKLOADS = {
    "smooth_particles_nside2048": dict(nside=2048, particles=50_000_000, sigma_pix=2.5, seed=1210002,
                                       oracle_sample=16),
    "smooth_particles_small": dict(nside=256, particles=1_000_000, sigma_pix=2.5, seed=1210002, oracle_sample=64),
}
SMOOTH_METRIC = "particles/s (Epanechnikov smoothing with exact mass conservation onto HEALPix)"

# grid search for the images of galaxies (Sec. 2.3) on the rays of the
# benchmark plane: the plane is solved and its rays stepped once (set-up),
# then the images of uniformly placed galaxies on the next sphere are found
IMAGE_WORKLOADS = {
    "image_search_nside2048": dict(plane="shtmg_plane_nside2048", galaxies=10_000_000, max_images=4,
                                   seed=1210006, oracle_sample=32),
    "image_search_small": dict(plane="shtmg_plane_nside512", galaxies=500_000, max_images=4, seed=1210006,
                               oracle_sample=32),
}
IMAGE_METRIC = "galaxies/s (grid search for lensed images with transported Jacobians, rays on Nside 2048)"

BATCH_METRIC = "lens planes/s (batched mixed-precision SHT Poisson, Nside 512/1024/2048, lmax = 2 Nside)"

# gradient of a galaxy-shear loss with respect to every plane's convergence
# map (pure-SHT planes, FP64), checkpointed per plane
ADJOINT_WORKLOADS = {
    "gal_adjoint_nside1024": dict(nplanes=16, nside=1024, lmax=2048, ngal=1_000_000, z_lo=0.3, z_hi=1.5,
                                  seed=1210005, fd_pixels=4),
    "gal_adjoint_small": dict(nplanes=4, nside=128, lmax=256, ngal=100_000, z_lo=0.3, z_hi=1.5, seed=1210005,
                              fd_pixels=4),
}
ADJOINT_METRIC = "loss+gradient evaluations/s (galaxy shear through SHT planes, adjoint w.r.t. all kappa maps)"

# multiple-plane ray tracing through a light cone of SHT+MG planes: every ray
# of the Nside grid traced through all planes (one step = one traversal), then
# the kappa, E, B and omega spectra of the final Jacobians in the image basis
LIGHTCONE_WORKLOADS = {
    "lightcone_nside2048": dict(nplanes=40, dchi=50.0, particles=20_000_000, nside=2048, nside_sht=512, lmax=1024,
                                nside_bundle=32, ncell=256, tol=1e-10, seed=1210003, spectra_lmax=1024),
    "lightcone_small": dict(nplanes=8, dchi=50.0, particles=2_000_000, nside=256, nside_sht=64, lmax=128,
                            nside_bundle=8, ncell=128, tol=1e-10, seed=1210003, spectra_lmax=256),
}
LIGHTCONE_METRIC = "rays/s (full traversal of the light cone's SHT+MG planes, rays on every pixel centre)"

FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
# FP64 operations of one ray step on an SHT+MG plane (k_ray_step, patch
# lookup included), counted operation by operation on the formulas of the
# kernel (an FMA is 2, a square root, reciprocal square root or division 1,
# the small-angle series of asin and of the rotation coefficients term by
# term): unit vector x / chi_n 3 and tangent basis 11; patch lookup 301
# (rotation to the patch frame 15, angles 39, bilinear blend of the 6 x 6
# stencil block 189 = cell fractions 4 + row/column blends 36 + the two
# sets of six blended first-derivative weights 12 + first-derivative sums of
# the six rows 66 + five blended partials 63 + scales 8, Appendix A 10,
# rotation to the global basis 48); Eq. Atraj 29; Eq. betaprop 81; Eq.
# posprop 15; new unit vector and basis 14; Appendix B transport 32 and two
# Q A Q^T as rotations of the traceless parts 41.
RAY_STEP_FLOPS_MG = 527
KERNELS = ("k_smooth_restrict", "k_prolong_smooth", "k_sub_vcycle", "k_coarse_solve", "k_resnorm", "k_resid_mixed",
           "k_combine", "k_mg_setup_base", "k_mg_setup_defect", "k_ray_step", "k_bin",
           "k_legendre_analysis", "k_legendre_synthesis", "k_ring_analysis", "k_ring_synthesis", "k_poisson_rhs",
           "k_degrade", "k_rays_init", "k_counts_to_kappa", "k_max_ratio", "k_split_ff")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 8:
                for k, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def plane_geometry():
    """Plane 20 of 40 shells of 50 Mpc/h (flat LCDM, Om = 0.25)."""
    pl = cosmology.lens_planes(40, 50.0)
    m = 20
    return pl["chi"][m - 1], pl["chi"][m], pl["chi"][m + 1], pl["scale"][m] * pl["growth"][m]


def kernel_models(cfg, precision, cycles, nsteps):
    """Algorithmic work of the modelled kernels over the timed steps:
    {name: (bound, amount, unit)}, summed over the levels that run the fused
    kernels (all but the coarsest).  FP32 (HBM-bound), per cell of the level
    and V-cycle: pre-smoothing + restriction reads f and, unless the
    correction starts at zero (coarse levels; the first V-cycle of each
    mixed refinement on the finest level), u; it writes u and the coarse
    source (9 or 13 B); prolongation + post-smoothing reads u, f and the
    coarse correction and writes u (13 B).  FP64 (FP64-ALU-bound, an FMA
    counts 2 flops): 8 flops per cell and sweep (3 FMA + 1 add + 1
    multiply), 10 per cell for the restricted residual and 7 for the
    prolongation.  The FP64
    residual of the mixed path (float-float on the FP32 pipe): 32 bytes per
    fine cell per refinement (one refinement per two V-cycles), and 12 for
    the first residual of a solve (e = 0: the defect in, the FP32 source out)."""
    npatch = 12 * cfg["nside_bundle"] ** 2
    cells_cycle = 0
    n = cfg["ncell"]
    while n > band_floor(cfg):
        cells_cycle += npatch * n * n
        n //= 2
    cells0 = npatch * cfg["ncell"] ** 2
    ncyc = sum(cycles)
    nzero = sum((c + 1) // 2 for c in cycles) if precision == "mixed" else 0
    out = {}
    if precision == "fp64":
        out["k_smooth_restrict"] = ("alu", (8.0 * cfg["nu1"] + 10.0) * cells_cycle * ncyc, "flop")
        out["k_prolong_smooth"] = ("alu", (8.0 * cfg["nu2"] + 7.0) * cells_cycle * ncyc, "flop")
    else:
        out["k_smooth_restrict"] = ("hbm", 9.0 * cells_cycle * ncyc + 4.0 * cells0 * (ncyc - nzero), "byte")
        out["k_prolong_smooth"] = ("hbm", 13.0 * cells_cycle * ncyc, "byte")
    if precision == "mixed":
        # float-float residual: e (8 B) and d (4 B) in, source (8 B) in, e (8 B) and r (4 B) out per fine
        # cell; the first of a solve reads the source (8 B) and writes r (4 B)
        n0 = cfg["ncell"]
        nref = sum((c + 1) // 2 for c in cycles)
        out["k_resid_mixed"] = ("hbm", (32.0 * nref + 12.0 * len(cycles)) * npatch * n0 * n0, "byte")
    # the ray step: FP64-ALU bound (228 B of state per ray against ~540 FP64
    # operations), one step of every ray per plane
    out["k_ray_step"] = ("alu", float(RAY_STEP_FLOPS_MG) * 12 * cfg["nside"] ** 2 * nsteps, "flop")
    return out


def band_floor(cfg):
    """Largest level size NOT run by the band kernels: the levels of 32 cells
    and below (down to the 8 x 8 coarsest) run in one k_sub_vcycle launch."""
    return 32 if cfg["ncell"] >= 16 and cfg["nu1"] >= 1 else 8


# DRAM bytes (read + write) of one V-cycle of the FP32 band kernels per
# patch of 256^2 cells, over its three band levels (256 .. 64), from the ncu
# capture of the Nside-512 plane (768 patches; every level's launch of the
# first V-cycle).  Traffic grows with the number of patches, so a launch at
# another patch count moves (this x patches / 3) bytes on average.
BAND_DRAM_PER_PATCH_CYCLE = {
    "k_prolong_smooth": (0.0329 + 0.1283 + 0.0182 + 0.4107 + 0.1685) * 1e9 / 768,
}


def band_traffic(name, cfg, precision):
    """Measured DRAM bytes per launch of a band kernel at this workload's
    patch count (FP32 band kernels of 256-cell patches only), else None."""
    per = BAND_DRAM_PER_PATCH_CYCLE.get(name)
    if per is None or cfg["ncell"] != 256 or precision == "fp64":
        return None
    return per * 12 * cfg["nside_bundle"] ** 2 / 3


def roofline(prof, models, peaks, peak_kind, traffic=None):
    """Roofline entries of the modelled kernels, largest total time first;
    traffic: {kernel: measured DRAM bytes per launch}."""
    traffic = traffic or {}
    ents = []
    for name, (bound, amount, unit) in models.items():
        n, ms = prof.get(name, (0, 0.0))
        if ms <= 0:
            continue
        if bound == "alu":
            ach = amount / (ms / 1e3) / 1e12
            ents.append({"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "launches": n,
                         "avg_launch_ms": ms / n,
                         "peak_source": "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz (derived; an FMA "
                                        "microbenchmark measured 1.20 TFLOP/s)"})
        else:
            ach = amount / (ms / 1e3) / 1e9
            pk = peaks.get("hbm_gbs", 6800.0)
            ents.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                         "frac": ach / pk, "traffic": traffic.get(name), "launches": n, "avg_launch_ms": ms / n,
                         "peak_source": f"HBM copy, {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"})
    ents.sort(key=lambda e: -e["avg_launch_ms"] * e["launches"])
    return ents


def plane_seed(cfg, rank):
    """Seed of the synthetic plane of one rank: every rank solves its own
    shell (independent problems, no data-path collective)."""
    return cfg["seed"] + rank


def bundle_range(nside_bundle, rank, world):
    """Contiguous NEST bundle range [lo, hi) of one rank when one plane's MG
    patches and rays are split over ranks (Sec. 3.1: bundles are the unit of
    work, NEST order keeps each range compact on the sphere): the 12 N_b^2
    bundles in near-equal consecutive shares."""
    nb = 12 * nside_bundle * nside_bundle
    return nb * rank // world, nb * (rank + 1) // world


def max_over_ranks(value, device):
    """The largest value over all ranks (a job's time is that of its slowest
    rank); the value itself without a process group."""
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_rate(world, units_per_rank, ms_max):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (weak scaling)."""
    return world * units_per_rank / (ms_max / 1000.0)


def run_gpu(args, cfg, rank, world):
    import paper_1210_3069_gb300 as clc
    clc.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ctx = clc.Context(dev.index)
    nf = cfg["nside"]
    npix = 12 * nf * nf
    chi_prev, chi_n, chi_next, scale = plane_geometry()
    prec = {"fp32": clc.FP32, "fp64": clc.FP64, "mixed": clc.MIXED}[args.precision]
    P = clc.mg_params(cfg["nside_sht"], cfg["lmax"], cfg["nside_bundle"], ncell=cfg["ncell"], nu1=cfg["nu1"],
                      nu2=cfg["nu2"], max_cycles=cfg["max_cycles"], tol=cfg["tol"], precision=prec,
                      refine_cycles=args.refine_cycles)
    # seeded synthetic plane (a different shell per rank)
    z, phi = synthetic.lognormal_particles(cfg["particles"], plane_seed(cfg, rank), device=dev)
    nbar = z.numel() / npix
    counts = torch.zeros(npix, dtype=torch.int32, device=dev)
    kappa = torch.empty(npix, dtype=torch.float64, device=dev)
    sol = ctx.solution(nf, P)
    rays = ctx.rays(npix)
    host_z = z.cpu().pin_memory()
    host_phi = phi.cpu().pin_memory()
    host_A = torch.empty(4, npix, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    cycles = []

    def step(zz=z, pp=phi, used=None, solution=None):
        solution = sol if solution is None else solution
        counts.zero_()
        ctx.bin_particles(zz, pp, nf, counts=counts)
        if used is not None:
            used.record(stream)   # the particle buffer may be refilled from here on
        ctx.counts_to_kappa(counts, nf, nbar, scale, kappa=kappa)
        ctx.poisson_shtmg(kappa, nf, solution, check=False)
        cycles.append(solution.info()[0])
        ctx.rays_init_pixels(rays, nf, chi_n, cfg["nside_bundle"])
        ctx.ray_step(rays, chi_prev, chi_n, chi_next, sol=solution)

    # End to end, pipelined as a production driver would run it: each step's
    # particles are copied in from pinned host memory on a copy stream while
    # the previous step computes (two device buffers), and each step's ray
    # Jacobians leave through a device staging buffer, copied to pinned host
    # memory while the next step computes.  Every step's copies are inside the
    # timed region.
    copy_stream = torch.cuda.Stream(dev)
    zb, pb = [z, torch.empty_like(z)], [phi, torch.empty_like(phi)]
    A_stage = torch.empty_like(rays.A)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]
    ev_staged, ev_out = torch.cuda.Event(), torch.cuda.Event()

    def e2e_run(nsteps, start_event):
        copy_stream.wait_event(start_event)
        with torch.cuda.stream(copy_stream):
            zb[0].copy_(host_z, non_blocking=True)
            pb[0].copy_(host_phi, non_blocking=True)
            ev_in[0].record(copy_stream)
        for k in range(nsteps):
            cur, nxt = k % 2, (k + 1) % 2
            if k + 1 < nsteps:
                with torch.cuda.stream(copy_stream):
                    if k >= 1:
                        copy_stream.wait_event(ev_used[nxt])   # step k - 1 has binned from buffer nxt
                    zb[nxt].copy_(host_z, non_blocking=True)
                    pb[nxt].copy_(host_phi, non_blocking=True)
                    ev_in[nxt].record(copy_stream)
            stream.wait_event(ev_in[cur])
            step(zb[cur], pb[cur], ev_used[cur])
            if k >= 1:
                stream.wait_event(ev_out)   # the staging buffer has reached the host
            A_stage.copy_(rays.A)
            ev_staged.record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_staged)
                host_A.copy_(A_stage, non_blocking=True)
                ev_out.record(copy_stream)
        stream.wait_stream(copy_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = ctx.launch_count()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    prof = {k: ctx.profile_query(k) for k in KERNELS}
    ctx.profile(False)
    timed_cycles = cycles[-args.steps:]
    ms = max_over_ranks(ms, dev)
    # end to end through the public API with host buffers
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps = max(1, args.steps)
    e2e_run(e2e_steps, e0)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dev)
    fp64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        fp64 = fp64_comparison(args, ctx, cfg, sol, step, kappa, clc, dev)
    sol.close()
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, prof=prof, cycles=timed_cycles, clocks=clocks.summary(),
                npix=npix, h2d=2 * 8 * z.numel(), d2h=4 * 8 * npix, fp64=fp64)


def fp64_comparison(args, ctx, cfg, sol, step, kappa, clc, dev):
    """The same step with the plain FP64 solver on the same plane (the
    metric's comparison): FP64 ms per step, and the relative L2 difference of
    the five lens fields between the two solutions at a seeded sample of
    pixels (both stop at the same relative residual)."""
    nf = cfg["nside"]
    npix = 12 * nf * nf
    g = torch.Generator(device=dev)
    g.manual_seed(cfg["seed"] + 17)
    pix = torch.randint(0, npix, (1_000_000,), generator=g, device=dev)
    mine = {k: v[pix] for k, v in ctx.poisson_shtmg(kappa, nf, sol, derivatives=True, check=False).items()}
    torch.cuda.synchronize()
    sol.close()
    P = clc.mg_params(cfg["nside_sht"], cfg["lmax"], cfg["nside_bundle"], ncell=cfg["ncell"], nu1=cfg["nu1"],
                      nu2=cfg["nu2"], max_cycles=cfg["max_cycles"], tol=cfg["tol"], precision=clc.FP64)
    s64 = ctx.solution(nf, P)
    step(solution=s64)                     # warm-up
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.fp64_steps):
        step(solution=s64)
    ev1.record()
    torch.cuda.synchronize()
    ms64 = ev0.elapsed_time(ev1) / args.fp64_steps
    cyc64 = s64.info()[0]
    ref = ctx.poisson_shtmg(kappa, nf, s64, derivatives=True, check=False)
    err = {}
    for k, v in ref.items():
        w = v[pix]
        err[k] = float(torch.linalg.vector_norm(mine[k] - w) / torch.linalg.vector_norm(w))
    s64.close()
    return {"value": 1000.0 / ms64, "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
            "mg_cycles": cyc64, "rel_l2_vs_fp64": err, "max_rel_l2_vs_fp64": max(err.values()),
            "sample": "1e6 seeded pixels, alpha and U of both solutions (both stopped at the same relative "
                      "residual tolerance)"}


def batch_maps(ctx, sizes, seed, dev):
    """Seeded lognormal density-contrast maps (unit-variance lognormal of a
    C_l ~ l^-2 Gaussian field) at the RING pixel centres of every plane."""
    import paper_1210_3069_gb300 as clc
    centres, maps = {}, []
    for i, (ns, _) in enumerate(sizes):
        if ns not in centres:
            rays = ctx.rays(12 * ns * ns)
            ctx.rays_init_pixels(rays, ns, 1.0, 0)
            torch.cuda.synchronize()
            n = rays.x
            centres[ns] = (n[2].clone(), torch.remainder(torch.atan2(n[1], n[0]), 2 * math.pi))
            del rays, n
        z, phi = centres[ns]
        modes = synthetic.random_field_modes(256, 2.0, 2.0 * ns, seed + i, device=dev)
        maps.append(synthetic.lognormal_density(z, phi, modes).double() - 1.0)
    del clc
    return maps


def run_batch(args, wl):
    """Throughput of one mixed-size batch plan (all planes per step) and of
    the FP64 per-plane path on a sample of the same planes."""
    import paper_1210_3069_gb300 as clc
    clc.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = clc.Context(0)
    sizes = wl["sizes"]
    P = len(sizes)
    maps = batch_maps(ctx, sizes, wl["seed"], dev)
    names = ("psi", "a_th", "a_ph", "u_tt", "u_pp", "u_tp")
    outs = [{k: torch.empty(12 * ns * ns, dtype=torch.float64, device=dev) for k in names} for ns, _ in sizes]
    t0 = time.perf_counter()
    plan = ctx.sht_plan([a for a, _ in sizes], [b for _, b in sizes], derivatives=True, graph=True, tune=True)
    plan.execute(maps, outs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = plan.info()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.execute(maps, outs)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            plan.execute(maps, outs)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    ctx.profile(False)
    # end to end: pinned host maps in, potentials out, through the plan
    host_in = [m.cpu().pin_memory() for m in maps]
    host_psi = [torch.empty(m.numel(), dtype=torch.float64).pin_memory() for m in maps]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, min(args.steps, 2))):
        for d, h in zip(maps, host_in):
            d.copy_(h, non_blocking=True)
        plan.execute(maps, outs)
        for h, o in zip(host_psi, outs):
            h.copy_(o["psi"], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / max(1, min(args.steps, 2))
    h2d = sum(m.numel() * 8 for m in maps)
    # FP64 per-plane path on a sample of each size (its lambda table must fit)
    plan.close()
    ctx.release_caches()
    fp64 = {}
    errs = []
    for ns, L in sorted(set(sizes)):
        idx = [i for i, s in enumerate(sizes) if s == (ns, L)][:wl["fp64_sample"]]
        try:
            for i in idx:
                ref = ctx.poisson_sht(maps[i], ns, L, precision=clc.FP64)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ref = ctx.poisson_sht(maps[i], ns, L, precision=clc.FP64)
                torch.cuda.synchronize()
                fp64.setdefault(f"{ns}/{L}", []).append((time.perf_counter() - t0) * 1e3)
                e = {k: float(torch.linalg.vector_norm(outs[i][k] - ref[k]) / torch.linalg.vector_norm(ref[k]))
                     for k in names}
                errs.append({"plane": i, "nside": ns, "lmax": L, "rel_l2_vs_fp64": e})
                del ref
        except clc.CalclensError as exc:
            fp64[f"{ns}/{L}"] = f"not run: {str(exc)[:120]}"
        ctx.release_caches()
    fp64_ms = {k: (sum(v) / len(v) if isinstance(v, list) else v) for k, v in fp64.items()}
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, clocks=clocks.summary(), P=P, info=info,
                setup_s=setup_s, fp64_ms_per_plane=fp64_ms, errors=errs, h2d=h2d, d2h=h2d)


def run_adjoint(args, wl):
    """Forward shears and the adjoint gradient of L = sum (gamma - gamma_target)^2
    over all planes (one step = forward + backward); FD check of the gradient
    at a few pixels (central, step 1e-6)."""
    import paper_1210_3069_gb300 as clc
    clc.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = clc.Context(0)
    N, ns, L = wl["nplanes"], wl["nside"], wl["lmax"]
    om = 0.25
    chi_max = cosmology.chi_of_z(wl["z_hi"], om)
    pl = cosmology.lens_planes(N, chi_max / N, om)
    chi = pl["chi"]
    rays = ctx.rays(12 * ns * ns)
    ctx.rays_init_pixels(rays, ns, 1.0, 0)
    torch.cuda.synchronize()
    zc, pc = rays.x[2].clone(), torch.remainder(torch.atan2(rays.x[1], rays.x[0]), 2 * math.pi)
    del rays

    def planes(seed):
        out = []
        for m in range(N):
            modes = synthetic.random_field_modes(256, 2.0, 2.0 * ns, seed + m, device=dev)
            delta = synthetic.lognormal_density(zc, pc, modes).double() - 1.0
            out.append(pl["scale"][m] * pl["growth"][m] * delta)
        return torch.stack(out)

    kappas = planes(wl["seed"])
    gz, gphi = synthetic.uniform_sphere(wl["ngal"], wl["seed"] + 100, device=dev)
    gen = torch.Generator(device=dev).manual_seed(wl["seed"] + 200)
    zg = wl["z_lo"] + (wl["z_hi"] - wl["z_lo"]) * torch.rand(wl["ngal"], generator=gen, dtype=torch.float64,
                                                              device=dev)
    zgrid = torch.linspace(0.0, wl["z_hi"] + 0.01, 2048, dtype=torch.float64)
    cgrid = torch.tensor([cosmology.chi_of_z(float(z), om) for z in zgrid], dtype=torch.float64)
    gchi = torch.from_numpy(__import__("numpy").interp(zg.cpu().numpy(), zgrid.numpy(), cgrid.numpy())).to(dev)
    with torch.no_grad():
        target, _ = ctx.gal_trace(planes(wl["seed"] + 5000), ns, L, chi, gz, gphi, gchi, tape=False)

    def step():
        k = kappas.clone().requires_grad_(True)
        g = clc.galaxy_shear(ctx, k, ns, L, chi, gz, gphi, gchi)
        loss = ((g - target) ** 2).sum()
        loss.backward()
        return loss.detach(), k.grad

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            loss, grad = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    # forward alone
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx.gal_trace(kappas, ns, L, chi, gz, gphi, gchi, tape=False)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    # finite differences of the loss at a few pixels (largest gradient entries)
    def lossv(k):
        g, _ = ctx.gal_trace(k, ns, L, chi, gz, gphi, gchi, tape=False)
        return float(((g - target) ** 2).sum())
    def central(m, p, h):
        kp, km = kappas.clone(), kappas.clone()
        kp[m, p] += h
        km[m, p] -= h
        return (lossv(kp) - lossv(km)) / (2 * h)

    fd = []
    for j in range(wl["fd_pixels"]):
        m = j % N
        p = int(grad[m].abs().argmax())
        a = float(grad[m, p])
        f6 = central(m, p, 1e-6)
        # a 10x larger step has 10x less rounding and still negligible truncation
        f5 = central(m, p, 1e-5)
        fd.append({"plane": m, "pixel": p, "adjoint": a, "fd_h1e-6": f6, "rel_diff_h1e-6": abs(f6 - a) / abs(a),
                   "fd_h1e-5": f5, "rel_diff_h1e-5": abs(f5 - a) / abs(a)})
    return dict(ms=ms, fwd_ms=fwd_ms, launches=launches, clocks=clocks.summary(), loss=float(loss), fd=fd)


def adjoint_line(args, wl, r):
    return {
        "metric": ADJOINT_METRIC, "value": args.steps / (r["ms"] / 1000.0), "unit": "gradients/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, **{k: v for k, v in wl.items() if k != "seed"},
                   "loss": "sum of squared shear differences from a catalogue traced through other seeded planes",
                   "checkpoints": "ray state entering every plane; lens maps recomputed",
                   "l2": "inputs larger than L2 (no flush)"},
        "forward_ms": r["fwd_ms"], "loss": r["loss"], "fd_check": r["fd"],
        "e2e": None, "gpu_launches": r["launches"], "clocks": r["clocks"],
    }


def run_smooth(args, wl):
    """Particles per second of the smoothing step (zero the map, smooth every
    particle, form kappa), and the oracle on a sample of the same particles."""
    import paper_1210_3069_gb300 as clc
    from oracle import smoothing as osm
    clc.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = clc.Context(0)
    nside, n = wl["nside"], wl["particles"]
    npix = 12 * nside * nside
    sigma = wl["sigma_pix"] * math.sqrt(4 * math.pi / npix)
    z, phi = synthetic.lognormal_particles(n, wl["seed"], device=dev)
    n = z.numel()   # Poisson-sampled: about the requested number
    rho = torch.zeros(npix, dtype=torch.float64, device=dev)
    kappa = torch.empty(npix, dtype=torch.float64, device=dev)
    nbar = n / npix

    def step(zz=z, pp=phi):
        rho.zero_()
        ctx.smooth_particles(zz, pp, nside, sigma, rho=rho)
        ctx.density_to_kappa(rho, nside, nbar, 1.0, kappa=kappa)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    launches0 = ctx.launch_count()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_query("k_smooth_particles")
    ctx.profile(False)
    mass_err = abs(float(rho.sum()) - n) / n
    # end to end: particles in from pinned host memory, kappa out
    hz, hp_ = z.cpu().pin_memory(), phi.cpu().pin_memory()
    hk = torch.empty(npix, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        z.copy_(hz, non_blocking=True)
        phi.copy_(hp_, non_blocking=True)
        step()
        hk.copy_(kappa, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    # the oracle on a sample of the particles (all-pixel brute force)
    cpu = None
    if not args.no_cpu_baseline:
        k = wl["oracle_sample"]
        zs, ps = z[:k].cpu(), phi[:k].cpu()
        t0 = time.perf_counter()
        osm.smooth_particles(nside, zs, ps, sigma)
        secs = time.perf_counter() - t0
        cpu = {"value": k / secs, "unit": "particles/s", "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"{k} particles of the same set, all-pixel oracle at Nside {nside}"}
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, prof=prof, clocks=clocks.summary(), n=n, npix=npix,
                sigma=sigma, mass_err=mass_err, cpu=cpu)


def run_images(args, wl):
    """Galaxies per second of the image search on the rays of one solved
    plane, and the oracle on a sample of the same galaxies."""
    import paper_1210_3069_gb300 as clc
    from oracle import healpix as ohp, images as oim
    clc.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = clc.Context(0)
    cfg = WORKLOADS[wl["plane"]]
    nf = cfg["nside"]
    npix = 12 * nf * nf
    chi_prev, chi_n, chi_next, scale = plane_geometry()
    P = clc.mg_params(cfg["nside_sht"], cfg["lmax"], cfg["nside_bundle"], ncell=cfg["ncell"], nu1=cfg["nu1"],
                      nu2=cfg["nu2"], max_cycles=cfg["max_cycles"], tol=cfg["tol"], precision=clc.MIXED)
    z, phi = synthetic.lognormal_particles(cfg["particles"], cfg["seed"], device=dev)
    counts = torch.zeros(npix, dtype=torch.int32, device=dev)
    ctx.bin_particles(z, phi, nf, counts=counts)
    kappa = ctx.counts_to_kappa(counts, nf, z.numel() / npix, scale)
    del z, phi, counts
    sol = ctx.solution(nf, P)
    ctx.poisson_shtmg(kappa, nf, sol, check=False)
    rays = ctx.rays(npix)
    ctx.rays_init_pixels(rays, nf, chi_n, cfg["nside_bundle"])
    ctx.ray_step(rays, chi_prev, chi_n, chi_next, sol=sol)
    del sol
    M, K = wl["galaxies"], wl["max_images"]
    gz, gp = synthetic.uniform_sphere(M, wl["seed"], device=dev)
    sg = torch.sqrt((1 - gz) * (1 + gz))
    g = torch.stack([sg * torch.cos(gp), sg * torch.sin(gp), gz]).contiguous()
    del gz, gp, sg
    torch.cuda.synchronize()

    def step(gg=g):
        return ctx.find_images(nf, rays.x, rays.A, gg, K)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    launches0 = ctx.launch_count()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            out = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    prof = {k: ctx.profile_query(k) for k in ("k_find_images", "k_image_bounds")}
    ctx.profile(False)
    nimg = out[0]
    hist = torch.bincount(nimg.clamp(max=3).long(), minlength=4).cpu().tolist()
    # end to end: galaxies in from pinned host memory, every output back
    hg = g.cpu().pin_memory()
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in out]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        g.copy_(hg, non_blocking=True)
        o = step()
        for h, t in zip(host_out, o):
            h.copy_(t, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    d2h = sum(t.numel() * t.element_size() for t in out)
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on a sample of the galaxies, each tested against the
        # triangles of the pixels within (largest ray displacement + four
        # pixel sizes) of it, the pixels found from a dense grid of points
        k = wl["oracle_sample"]
        x = rays.x.T.cpu()
        A = rays.A.T.reshape(npix, 2, 2).cpu()
        cen = ohp.pix2vec_ring(nf, torch.arange(npix))
        xn = x / torch.linalg.vector_norm(x, dim=-1, keepdim=True)
        dmax = float(torch.atan2(torch.linalg.vector_norm(torch.linalg.cross(xn, cen, dim=-1), dim=-1),
                                 (xn * cen).sum(-1)).max())
        del cen, xn
        h = math.sqrt(4 * math.pi / npix)
        gs = g[:, :k].T.cpu()
        secs = 0.0
        for m in range(k):
            own = _pixels_near(nf, gs[m], dmax + 4 * h)
            t0 = time.perf_counter()
            oim.find_images(nf, x, A, gs[m:m + 1], K, owners=own)
            secs += time.perf_counter() - t0
        cpu = {"value": k / secs, "unit": "galaxies/s", "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"{k} galaxies of the same set, oracle on the triangles of the pixels within the largest "
                         f"ray displacement ({dmax:.2e} rad) + 4 pixel sizes of each"}
    return dict(ms=ms, e2e_ms=e2e_ms, launches=launches, prof=prof, clocks=clocks.summary(), M=M, npix=npix,
                hist=hist, h2d=g.numel() * 8, d2h=d2h, cpu=cpu, nside=nf)


def _pixels_near(nside, g, radius):
    """RING pixels hit by a grid of points (a quarter pixel apart) within
    `radius` of the unit vector g."""
    from oracle import healpix as ohp
    g = g / torch.linalg.vector_norm(g)
    h = math.sqrt(4 * math.pi / (12 * nside * nside))
    n = int(math.ceil(radius / (0.25 * h)))
    u = torch.linspace(-radius, radius, 2 * n + 1, dtype=torch.float64)
    a = torch.linalg.cross(g, torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64))
    a = a / torch.linalg.vector_norm(a)
    b = torch.linalg.cross(g, a)
    U, V = torch.meshgrid(u, u, indexing="ij")
    r = torch.sqrt(U * U + V * V)
    keep = r <= radius
    U, V, r = U[keep], V[keep], r[keep]
    d = (U[:, None] * a + V[:, None] * b) / torch.where(r > 0, r, 1.0)[:, None]
    pts = torch.cos(r)[:, None] * g + torch.sin(r)[:, None] * d
    phi = torch.remainder(torch.atan2(pts[:, 1], pts[:, 0]), 2 * math.pi)
    return torch.unique(ohp.ang2pix_ring(nside, pts[:, 2].clamp(-1, 1), phi))


def images_line(args, wl, r):
    value = r["M"] * args.steps / (r["ms"] / 1e3)
    n, kms = r["prof"]["k_find_images"]
    roof = None
    if kms > 0:
        # FP64-ALU-bound (ncu: FP64 pipe 83% busy, DRAM 3%).  Algorithmic FP64
        # work per galaxy, what any search must do once the containing
        # triangle is known: its three triple products and three hemisphere
        # dots (57 flops), barycentric weights and the normalised image (35),
        # the interpolation weights (20) and, for each of the four
        # interpolation rays, normalisation, tangent basis, transport
        # rotation, Q A Q^T and the weighted sum (106): about 540 flops
        per_gal = 57 + 35 + 20 + 4 * 106
        ach = per_gal * r["M"] * n / (kms / 1e3) / 1e12
        roof = {"kernel": "k_find_images", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "launches": n,
                "avg_launch_ms": kms / max(n, 1),
                "peak_source": "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz (derived)"}
    return {
        "metric": IMAGE_METRIC, "value": value, "unit": "galaxies/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nside_rays": r["nside"], "rays": r["npix"], "galaxies": r["M"],
                   "max_images": wl["max_images"], "rays_from": wl["plane"] + " (one solved plane, one ray step)",
                   "l2": "inputs larger than L2 (no flush)"},
        "images_per_galaxy_hist": {"0": r["hist"][0], "1": r["hist"][1], "2": r["hist"][2], "3+": r["hist"][3]},
        "stage_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in r["prof"].items()},
        "roofline": roof,
        "e2e": {"value": r["M"] / (r["e2e_ms"] / 1e3), "unit": "galaxies/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"], "clocks": r["clocks"], "cpu_baseline": r["cpu"],
    }


def smooth_line(args, wl, r):
    peaks, peak_kind = load_peaks()
    n = r["n"]
    value = n * args.steps / (r["ms"] / 1e3)
    # FP64 ALU work: about pi sigma^2 / Omega_pix pixels within each kernel,
    # about 20 FP64 flops to test and weigh each (chord, rotation, asin^2
    # series, weight), once; the deposit is FP64 atomics
    per_particle = math.pi * wl["sigma_pix"] ** 2 * 20.0
    launches, kms = r["prof"]
    roof = None
    if kms > 0:
        ach = per_particle * n * launches / (kms / 1e3) / 1e12
        roof = {"kernel": "k_smooth_particles", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz (derived)"}
    return {
        "metric": SMOOTH_METRIC, "value": value, "unit": "particles/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nside": wl["nside"], "particles": n, "sigma_rad": r["sigma"],
                   "sigma_pixel_scales": wl["sigma_pix"], "l2": "inputs larger than L2 (no flush)"},
        "mass_conservation_rel_err": r["mass_err"],
        "roofline": roof,
        "e2e": {"value": n / (r["e2e_ms"] / 1e3), "unit": "particles/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 8 * r["npix"]},
        "gpu_launches": r["launches"], "clocks": r["clocks"], "cpu_baseline": r["cpu"],
    }


def batch_line(args, wl, r):
    peaks, peak_kind = load_peaks()
    sizes = wl["sizes"]
    value = r["P"] * args.steps / (r["ms"] / 1000.0)
    fp64 = r["fp64_ms_per_plane"]
    fp64_total = 0.0
    fp64_ok = True
    for ns, L in sizes:
        v = fp64.get(f"{ns}/{L}")
        if isinstance(v, float):
            fp64_total += v
        else:
            fp64_ok = False
    # Rooflines of the three largest stages (HBM-bound; algorithmic bytes):
    # tensor-core analysis = FP16 hi + lo table once per class; tensor-core
    # synthesis = the table again + the FP32 Legendre sums G written (3
    # quantities x 8 B per (m, ring) per plane); ring synthesis = G read + six
    # FP64 output maps written.
    stage = r["info"]["stage_ms"]
    tab_bytes = g_bytes = out_bytes = 0
    for ns, L in sorted(set(sizes)):
        rows = sum(((L + 1 - m - p) // 2 + 1 + 63) // 64 * 64 for m in range(L + 1) for p in (0, 1)
                   if m + p <= L + 1)
        nplanes = sizes.count((ns, L))
        nclass = -(-nplanes // 21)
        tab_bytes += nclass * 2 * 2 * rows * 2 * ns
        g_bytes += nplanes * 3 * 8 * (L + 1) * (4 * ns - 1)
        out_bytes += nplanes * 6 * 8 * 12 * ns * ns
    pk = peaks.get("hbm_gbs", 6800.0)
    models = [("k_tc_ring_synthesis", 5, g_bytes + out_bytes), ("k_tc_synthesis", 4, tab_bytes + g_bytes),
              ("k_tc_analysis", 2, tab_bytes)]
    roofs = []
    for name, k, nbytes in models:
        ach = nbytes / (stage[k] / 1e3) / 1e9
        roofs.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                      "traffic": None, "stage_ms": stage[k],
                      "peak_source": f"HBM copy, {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"})
    roofs.sort(key=lambda e: -e["stage_ms"])
    return {
        "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x3+f32 (Legendre), f32 (FFT), f64 (tables)", "data": "synthetic",
        "config": {"workload": args.workload, "planes": r["P"],
                   "sizes": {f"{a}/{b}": sizes.count((a, b)) for a, b in sorted(set(sizes))},
                   "outputs": "psi, alpha, U at every pixel", "l2": "inputs larger than L2 (no flush)"},
        "plan": {"launch_shape": r["info"]["shape"], "tuned_stage_ms": [round(x, 3) for x in stage],
                 "device_bytes": r["info"]["device_bytes"], "setup_s": round(r["setup_s"], 2)},
        "fp64_gpu_ms_per_plane": fp64,
        "fp64_gpu_planes_per_s": (len(sizes) / (fp64_total / 1e3)) if fp64_ok and fp64_total > 0 else None,
        "errors_vs_fp64": r["errors"],
        "roofline": roofs[0],
        "roofline_all": roofs,
        "e2e": {"value": r["P"] / (r["e2e_ms"] / 1000.0), "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }


def run_lightcone(args, wl):
    """40 shells of 50 Mpc/h (flat LCDM, Om = 0.25), each a seeded lognormal
    plane scaled by the linear growth factor and Poisson-sampled to
    `particles`; one timed step traces every ray of the Nside grid through all
    planes (binning, kappa, SHT+MG solve, ray step per plane) and takes the
    spectra of the final Jacobians (carried to the image basis)."""
    import paper_1210_3069_gb300 as clc
    clc.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = clc.Context(0)
    N, nf = wl["nplanes"], wl["nside"]
    npix = 12 * nf * nf
    pl = cosmology.lens_planes(N, wl["dchi"])
    chi = pl["chi"]
    parts = [synthetic.lognormal_particles(wl["particles"], wl["seed"] + m, device=dev, growth=pl["growth"][m])
             for m in range(N)]
    prec = {"fp32": clc.FP32, "fp64": clc.FP64, "mixed": clc.MIXED}[args.precision]
    P = clc.mg_params(wl["nside_sht"], wl["lmax"], wl["nside_bundle"], ncell=wl["ncell"], tol=wl["tol"],
                      precision=prec)
    sol = ctx.solution(nf, P)
    rays = ctx.rays(npix)
    counts = torch.zeros(npix, dtype=torch.int32, device=dev)
    kappa = torch.empty(npix, dtype=torch.float64, device=dev)
    cycles = []

    def traverse():
        ctx.rays_init_pixels(rays, nf, chi[0], wl["nside_bundle"])
        for m in range(N):
            z, phi = parts[m]
            counts.zero_()
            ctx.bin_particles(z, phi, nf, counts=counts)
            ctx.counts_to_kappa(counts, nf, z.numel() / npix, pl["scale"][m], kappa=kappa)
            ctx.poisson_shtmg(kappa, nf, sol, check=False)
            cycles.append(sol.info()[0])
            ctx.ray_step(rays, chi[m - 1] if m else 0.0, chi[m], chi[m + 1], sol=sol)
        return ctx.lensing_spectra(rays.A, nf, wl["spectra_lmax"], x=rays.x)

    for _ in range(max(1, args.warmup)):
        traverse()
    torch.cuda.synchronize()
    cycles.clear()
    launches0 = ctx.launch_count()
    ctx.profile(True)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            cl = traverse()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    prof = {k: ctx.profile_query(k) for k in KERNELS}
    ctx.profile(False)
    sol.close()
    return dict(ms=ms, launches=launches, clocks=clocks.summary(), cycles=cycles, cl={k: v.cpu() for k, v in cl.items()},
                prof=prof, npix=npix)


def lightcone_line(args, wl, r):
    nf, N = wl["nside"], wl["nplanes"]
    ms_step = r["ms"] / args.steps
    cl = r["cl"]
    L = wl["spectra_lmax"]
    l = torch.arange(L + 1, dtype=torch.float64)
    s_l = torch.where(l >= 2, (l + 2) * (l - 1) / torch.where(l > 0, l * (l + 1), torch.ones_like(l)),
                      torch.zeros_like(l))
    bands = []
    lo = 8
    while lo < L:
        hi = min(4 * lo, L + 1)
        sel = (l >= lo) & (l < hi)
        bands.append({"l": [lo, hi - 1],
                      "E_over_s_kappa": float(cl["E"][sel].sum() / (s_l[sel] * cl["kappa"][sel]).sum()),
                      "B_over_s_omega": float(cl["B"][sel].sum() / (s_l[sel] * cl["omega"][sel]).sum()),
                      "B_over_E": float(cl["B"][sel].sum() / cl["E"][sel].sum())})
        lo = hi
    return {
        "metric": LIGHTCONE_METRIC, "value": r["npix"] / (ms_step / 1000.0), "unit": "rays/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, **{k: v for k, v in wl.items() if k != "seed"}, "rays": r["npix"],
                   "precision": args.precision, "l2": "inputs larger than L2 (no flush)"},
        "ray_plane_steps_per_s": r["npix"] * N / (ms_step / 1000.0),
        "planes_per_s": N / (ms_step / 1000.0),
        "mg_cycles": sorted(set(r["cycles"])),
        "spectra_bands": bands,
        "stage_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in r["prof"].items()},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "e2e": None,
        "e2e_note": "the light cone's particles (16 B each, all planes) stay resident; the default workload's line "
                    "carries the end-to-end number",
    }


# ---------------------------------------------------------------------------
# the FP64 oracle on a bounded sample of the same workload

def oracle_plane_estimate(cfg, sample_patches=4, sample_rays=20_000, sample_particles=2_000_000, sht_mcols=16,
                          cycles=None, seed=0):
    """Seconds the oracle would take for one plane of `cfg`, from timed
    samples: binning of sample_particles (scaled to all particles), the SHT
    with the Legendre sums restricted to m < sht_mcols (scaled by the number
    of (l, m) pairs) plus all ring FFTs, the MG set-up and V-cycles on
    sample_patches patches (scaled to all patches) and one ray step of
    sample_rays rays (scaled to all rays)."""
    from oracle import binning, healpix as hp, mg as omg, rays as orays, sht
    nf, ns, L, nb, ncell = cfg["nside"], cfg["nside_sht"], cfg["lmax"], cfg["nside_bundle"], cfg["ncell"]
    npix = 12 * nf * nf
    parts = {}
    z, phi = synthetic.lognormal_particles(sample_particles, cfg["seed"] + seed)
    t = time.perf_counter()
    counts = binning.bin_counts(nf, z, phi)
    kap = binning.kappa_from_counts(counts, z.numel() / npix, 1.0)
    parts["bin"] = (time.perf_counter() - t) * cfg["particles"] / z.numel()
    # SHT (analysis + synthesis of psi) on the SHT grid
    ks = torch.randn(12 * ns * ns, dtype=torch.float64, generator=torch.Generator().manual_seed(seed))
    rt = hp.ring_table(ns)
    t = time.perf_counter()
    F = sht.ring_fourier(ns, ks, L)
    G = torch.zeros_like(F)
    for m, lam in sht.legendre_columns(L, rt["z"], rt["sin_theta"], mmax=sht_mcols - 1):
        a = lam.to(torch.complex128) @ F[:, m]
        G[:, m] = lam.T.to(torch.complex128) @ a
    t_leg = time.perf_counter()
    sht.ring_inverse_fourier(ns, G, L)
    t_fft = time.perf_counter() - t_leg
    pairs_all = (L + 1) * (L + 2) / 2
    pairs_s = sum(L - m + 1 for m in range(sht_mcols))
    parts["sht"] = (t_leg - t) * pairs_all / pairs_s + 2 * t_fft
    # MG on a sample of patches
    psi_s = sht.ring_inverse_fourier(ns, G, L)
    bundles = torch.arange(sample_patches) * (12 * nb * nb // sample_patches)
    t = time.perf_counter()
    R, h, u, f, ghosts = omg.setup_patches(kap, nf, psi_s, ns, nb, bundles, ncell=ncell)
    S = omg.PatchSolver(ncell, h, ghosts, nu1=cfg["nu1"], nu2=cfg["nu2"])
    ncyc = cycles if cycles else 10
    S.solve(u, f, fixed_cycles=ncyc)
    parts["mg"] = (time.perf_counter() - t) * (12 * nb * nb) / sample_patches
    # one ray step
    sol = {"R": R, "h": h, "partials": omg.fd_partials(u[:, 1:-1, 1:-1], h), "bundles": bundles}
    pix = torch.randint(0, npix, (sample_rays,), generator=torch.Generator().manual_seed(seed + 1))
    n0 = hp.pix2vec_ring(nf, pix)
    home = bundles[torch.randint(0, sample_patches, (sample_rays,), generator=torch.Generator().manual_seed(2))]
    # rays placed at their patch centres so every lookup is valid
    cen = torch.einsum("bji,j->bi", R, torch.tensor([1.0, 0.0, 0.0], dtype=torch.float64))
    lookup = {int(b): k for k, b in enumerate(bundles.tolist())}
    n0 = cen[torch.tensor([lookup[int(b)] for b in home.tolist()])] + 1e-4 * n0
    n0 = n0 / torch.linalg.vector_norm(n0, dim=-1, keepdim=True)
    t = time.perf_counter()
    st = orays.init_rays(n0, 1000.0)
    orays.step(st, lambda n: omg.fields_at(sol, nb, n, home), 950.0, 1000.0, 1050.0)
    parts["rays"] = (time.perf_counter() - t) * npix / sample_rays
    return sum(parts.values()), parts


# V-cycles the GPU path needs to reach the 1e-10 tolerance on the Nside-2048
# plane (its line's mg_cycles); the reference arm runs the oracle at this count
ORACLE_CYCLES = 10


def cpu_baseline(cfg, cycles, seed=0, small=False):
    kw = dict(sample_patches=2, sample_rays=5_000, sample_particles=500_000, sht_mcols=8) if small else {}
    t0 = time.perf_counter()
    secs, parts = oracle_plane_estimate(cfg, cycles=cycles, seed=seed, **kw)
    wall = time.perf_counter() - t0
    s = dict(sample_patches=2, sample_rays=5000, sample_particles=500000, sht_mcols=8) if small else \
        dict(sample_patches=4, sample_rays=20000, sample_particles=2000000, sht_mcols=16)
    sample = (f"oracle timed on {s['sample_particles']} particles (binning), Legendre columns m<{s['sht_mcols']} "
              f"of the SHT plus all ring FFTs, {s['sample_patches']} MG patches x {cycles} V-cycles, "
              f"{s['sample_rays']} ray steps; each part scaled to the full plane")
    return {"value": 1.0 / secs, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": sample, "seconds_per_plane": secs, "parts_s": {k: round(v, 3) for k, v in parts.items()},
            "wall_s": round(wall, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed"],
                    help="MG arithmetic: fp64, fp32, or mixed (FP32 V-cycles on an FP64 residual equation)")
    ap.add_argument("--workload", default="shtmg_plane_nside2048",
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + sorted(ADJOINT_WORKLOADS)
                    + sorted(SMOOTH_WORKLOADS) + sorted(IMAGE_WORKLOADS) + sorted(LIGHTCONE_WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refine-cycles", type=int, default=0,
                    help="mixed precision: FP32 V-cycles per float-float residual refinement (0: the library's 2)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed steps of the plain FP64 solver on the same plane after the main run (0: skip)")
    args = ap.parse_args()
    if args.workload in ADJOINT_WORKLOADS:
        if args.impl == "reference" or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": args.impl, "metric": ADJOINT_METRIC,
                                  "unavailable": "the adjoint workload runs on one GPU"}))
            return
        wl = ADJOINT_WORKLOADS[args.workload]
        print(json.dumps(adjoint_line(args, wl, run_adjoint(args, wl))))
        return
    if args.workload in LIGHTCONE_WORKLOADS:
        if args.impl == "reference" or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": args.impl, "metric": LIGHTCONE_METRIC,
                                  "unavailable": "the light-cone workload runs on one GPU; the oracle's per-plane "
                                                 "cost is in the default workload's cpu_baseline"}))
            return
        wl = LIGHTCONE_WORKLOADS[args.workload]
        print(json.dumps(lightcone_line(args, wl, run_lightcone(args, wl))))
        return
    if args.workload in SMOOTH_WORKLOADS:
        if args.impl == "reference" or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": args.impl, "metric": SMOOTH_METRIC,
                                  "unavailable": "the smoothing workload runs on one GPU (its oracle sample is in "
                                                 "the GPU line's cpu_baseline)"}))
            return
        wl = SMOOTH_WORKLOADS[args.workload]
        print(json.dumps(smooth_line(args, wl, run_smooth(args, wl))))
        return
    if args.workload in IMAGE_WORKLOADS:
        if args.impl == "reference" or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": args.impl, "metric": IMAGE_METRIC,
                                  "unavailable": "the image-search workload runs on one GPU (its oracle sample is "
                                                 "in the GPU line's cpu_baseline)"}))
            return
        wl = IMAGE_WORKLOADS[args.workload]
        print(json.dumps(images_line(args, wl, run_images(args, wl))))
        return
    if args.workload in BATCH_WORKLOADS:
        if args.impl == "reference" or int(os.environ.get("WORLD_SIZE", "1")) > 1:
            if int(os.environ.get("RANK", "0")) == 0:
                print(json.dumps({"impl": args.impl, "metric": BATCH_METRIC,
                                  "unavailable": "the batch workload runs on one GPU, mixed precision only"}))
            return
        wl = BATCH_WORKLOADS[args.workload]
        print(json.dumps(batch_line(args, wl, run_batch(args, wl))))
        return
    cfg = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    config = {"workload": args.workload, **{k: v for k, v in cfg.items() if k != "seed"},
              "rays": 12 * cfg["nside"] ** 2, "precision": args.precision,
              "refine_cycles": args.refine_cycles or 2,
              "l2": "inputs larger than L2 (no flush)", "planes_per_rank_per_step": 1}

    if args.impl == "reference":
        if rank != 0:
            return
        # the FP64 oracle on the GPU line's cpu_baseline sample, at the V-cycle
        # count the GPU path needs on this plane; each step times one sample
        # and extrapolates it to a whole plane
        est, walls = [], []
        for s in range(args.warmup + args.steps):
            t = time.perf_counter()
            e = cpu_baseline(cfg, cycles=ORACLE_CYCLES, seed=s)
            if s >= args.warmup:
                est.append(e)
                walls.append(time.perf_counter() - t)
        secs = statistics.median(e["seconds_per_plane"] for e in est)
        parts = {k: round(statistics.median(e["parts_s"][k] for e in est), 3) for k in est[0]["parts_s"]}
        value = 1.0 / secs
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * secs, "extrapolated": True,
                "sample_wall_ms_per_step": 1000.0 * statistics.median(walls), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "impl": "reference",
                "cpu_baseline": {"kind": "oracle", "cores": est[0]["cores"], "sample": est[0]["sample"],
                                 "value": value, "unit": UNIT, "parts_s": parts},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        torch.distributed.init_process_group("nccl")
    r = run_gpu(args, cfg, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, peak_kind = load_peaks()
    value = whole_job_rate(world, args.steps, r["ms"])
    roof = roofline(r["prof"], kernel_models(cfg, args.precision, r["cycles"], args.steps), peaks, peak_kind,
                    traffic={k: band_traffic(k, cfg, args.precision) for k in BAND_DRAM_PER_PATCH_CYCLE})
    top = max(r["prof"].items(), key=lambda kv: kv[1][1])[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f32+f64"}[args.precision], "data": "synthetic",
        "config": config,
        "rays_per_s": whole_job_rate(world, r["npix"] * args.steps, r["ms"]),
        "mg_cycles": r["cycles"],
        "top_kernel": top,
        "roofline": roof[0] if roof else None,
        "roofline_all": roof,
        "stage_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in r["prof"].items()},
        "e2e": {"value": whole_job_rate(world, 1, r["e2e_ms"]), "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    if r.get("fp64"):
        line["fp64"] = r["fp64"]
        line["speedup_vs_fp64"] = value / (world * r["fp64"]["value"])
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(cfg, cycles=max(r["cycles"]) if r["cycles"] else 10)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
