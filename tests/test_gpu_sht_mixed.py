"""GPU parity of the mixed-precision (split FP16 hi + lo on the tensor cores,
FP32 accumulation) pure-SHT Poisson solve, single plane and batched (paper
Sec. 3.2 transforms).  Every output field agrees with the FP64 oracle to
<= 1e-5 relative L2; the batched call equals per-plane calls of the same
precision's single-plane entry point within the same bound, and the FP64
batch equals per-plane FP64 solves."""
import pytest
import torch

from oracle import binning, healpix as hp, sht
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5
FIELDS = ("psi", "a_th", "a_ph", "u_tt", "u_pp", "u_tp")


def _planes(nside, P, seed0=100):
    """P convergence maps of clumpy particle sets (uniform background plus
    Gaussian clumps of varying size), binned at nside."""
    out = []
    for i in range(P):
        s = seed0 + i
        z, phi = synthetic.uniform_sphere(40_000, s)
        z2, p2 = synthetic.gaussian_clumps(10 + i % 7, 1500, 0.02 + 0.01 * (i % 5), s)
        z = torch.cat([z, z2])
        phi = torch.cat([phi, p2])
        c = binning.bin_counts(nside, z, phi)
        out.append(binning.kappa_from_counts(c, z.numel() / hp.npix(nside), 1.0))
    return torch.stack(out)


def _check_oracle(got, kappa, i, nside, lmax, fields=FIELDS):
    want = sht.poisson_sht(kappa[i], nside, lmax)
    for k in fields:
        e = rel_l2(got[k][i], want[k])
        assert e < TOL_MIXED, (i, k, e)


@pytest.mark.parametrize("nside,lmax", [(64, 128), (64, 100), (64, 256)])
def test_mixed_batch_matches_oracle(nside, lmax):
    """Three planes in one tensor-core batch; lmax 100 leaves ragged row tiles,
    lmax = 4 nside is the largest band limit the entry point accepts."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    kappa = _planes(nside, 3)
    got = c.poisson_sht_batch(kappa.cuda(), nside, lmax, precision=clc.MIXED)
    c.sync()
    for i in range(3):
        _check_oracle(got, kappa, i, nside, lmax)


def test_mixed_single_plane_entry():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 64, 128
    kappa = _planes(nside, 1, seed0=7)
    got = c.poisson_sht(kappa[0].cuda(), nside, lmax, precision=clc.MIXED)
    c.sync()
    got = {k: v[None] for k, v in got.items()}
    _check_oracle(got, kappa, 0, nside, lmax)


def test_mixed_batches_split_with_derivatives():
    """23 planes with derivatives: one full batch of 21 and a batch of 2."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 128, 256
    kappa = _planes(nside, 23, seed0=300)
    got = c.poisson_sht_batch(kappa.cuda(), nside, lmax, precision=clc.MIXED)
    ref = c.poisson_sht_batch(kappa.cuda(), nside, lmax, precision=clc.FP64)
    c.sync()
    for i in range(23):
        for k in FIELDS:
            assert rel_l2(got[k][i], ref[k][i]) < TOL_MIXED, (i, k)
    for i in (0, 22):
        _check_oracle(got, kappa, i, nside, lmax)


def test_mixed_psi_only_many_planes():
    """66 planes, potential only: one batch of 64 and a batch of 2."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 64, 128
    kappa = _planes(nside, 66, seed0=500)
    got = c.poisson_sht_batch(kappa.cuda(), nside, lmax, precision=clc.MIXED, derivatives=False)
    c.sync()
    assert set(got) == {"psi"}
    for i in (0, 63, 64, 65):
        _check_oracle(got, kappa, i, nside, lmax, fields=("psi",))


def test_fp64_batch_equals_single_planes():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 64, 128
    kappa = _planes(nside, 2, seed0=900).cuda()
    got = c.poisson_sht_batch(kappa, nside, lmax, precision=clc.FP64)
    for i in range(2):
        one = c.poisson_sht(kappa[i], nside, lmax, precision=clc.FP64)
        c.sync()
        for k in FIELDS:
            assert torch.equal(got[k][i], one[k]), k


def test_mixed_large_against_fp64():
    """Nside 512, lmax 1024 (the SHT grid of the SHT+MG plane), a full batch of
    21 planes with derivatives against the FP64 path (itself checked against
    the oracle at this size on sampled pixels)."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 512, 1024
    g = torch.Generator().manual_seed(4)
    P = 21
    base = _planes(nside, 3, seed0=40)
    kappa = (base[torch.arange(P) % 3] * (1.0 + 0.1 * torch.randn(P, 1, dtype=torch.float64, generator=g))).cuda()
    got = c.poisson_sht_batch(kappa, nside, lmax, precision=clc.MIXED)
    ref = c.poisson_sht_batch(kappa[:4], nside, lmax, precision=clc.FP64)
    c.sync()
    for i in range(4):
        for k in FIELDS:
            assert rel_l2(got[k][i], ref[k][i]) < TOL_MIXED, (i, k)


@pytest.mark.parametrize("nside,lmax", [(512, 1024), (1024, 2048)])
def test_mixed_lognormal_full_band(nside, lmax):
    """Lognormal density contrast of a C_l ~ l^-2 Gaussian field with power up
    to l ~ 2 nside (the light-cone planes of the batched workload): every
    field within 1e-5 of the FP64 path, which is itself checked against the
    oracle.  High-l power is where FP32 accumulation error shows first."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    z, phi = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    maps = []
    for i in range(3):
        modes = synthetic.random_field_modes(256, 2.0, 2.0 * nside, 77 + i)
        maps.append(synthetic.lognormal_density(z, phi, modes).double() - 1.0)
    kappa = torch.stack(maps).cuda()
    got = c.poisson_sht_batch(kappa, nside, lmax, precision=clc.MIXED)
    for i in range(3):
        ref = c.poisson_sht(kappa[i], nside, lmax, precision=clc.FP64)
        c.sync()
        for k in FIELDS:
            assert rel_l2(got[k][i], ref[k]) < TOL_MIXED, (i, k, rel_l2(got[k][i], ref[k]))


def test_mixed_rejects_bad_arguments():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    k = torch.zeros(2, 12 * 32 * 32, dtype=torch.float64, device="cuda")
    with pytest.raises(clc.CalclensError) as e:
        c.poisson_sht_batch(k, 32, 64, precision=clc.MIXED)
    assert e.value.code == clc.EINVAL
    k = torch.zeros(2, 12 * 64 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(clc.CalclensError) as e:
        c.poisson_sht_batch(k, 64, 257, precision=clc.MIXED)
    assert e.value.code == clc.EINVAL
    with pytest.raises(clc.CalclensError) as e:
        c.poisson_sht_batch(k, 64, 128, precision=clc.FP32)
    assert e.value.code == clc.EINVAL


def test_plan_mixed_sizes_graph_and_tuning():
    """One plan over three (nside, lmax) classes, autotuned and replayed as a
    CUDA graph twice with different maps; every plane checked."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    sizes = [(64, 128), (128, 256), (64, 128), (64, 100), (128, 256), (64, 100), (64, 128)]
    plan = c.sht_plan([s[0] for s in sizes], [s[1] for s in sizes], derivatives=True, graph=True, tune=True)
    for rep in range(2):
        kappas = [_planes(ns, 1, seed0=1000 + 10 * rep + i)[0] for i, (ns, _) in enumerate(sizes)]
        outs = [{k: torch.empty(hp.npix(ns), dtype=torch.float64, device="cuda") for k in FIELDS} for ns, _ in sizes]
        plan.execute([k.cuda() for k in kappas], outs)
        c.sync()
        for i, (ns, L) in enumerate(sizes):
            ref = c.poisson_sht(kappas[i].cuda(), ns, L, precision=clc.FP64)
            c.sync()
            for k in FIELDS:
                assert rel_l2(outs[i][k], ref[k]) < TOL_MIXED, (rep, i, k)
        if rep == 0:
            want = sht.poisson_sht(kappas[3], 64, 100)
            for k in FIELDS:
                assert rel_l2(outs[3][k], want[k]) < TOL_MIXED, k
    info = plan.info()
    assert all(v > 0 for v in info["stage_ms"]) and info["device_bytes"] > 0
    plan.close()


@pytest.mark.parametrize("order", ["narrow_first", "wide_first"])
def test_plan_classes_of_different_widths_match_single_planes(order):
    """A class of few planes with long contractions (8 planes, 48 operand
    columns) beside a class of many planes with short ones (21 planes, 128
    columns): the work lists interleave items of both widths on each CTA.
    Every plane must come out exactly as the single-plane tensor-core solve
    gives it: the per-column arithmetic is the same, only the batching
    differs."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    narrow, wide = [(512, 1024)] * 8, [(256, 512)] * 21
    sizes = narrow + wide if order == "narrow_first" else wide + narrow
    kappas = [_planes(ns, 1, seed0=3000 + i)[0].cuda() for i, (ns, _) in enumerate(sizes)]
    outs = [{k: torch.empty(hp.npix(ns), dtype=torch.float64, device="cuda") for k in FIELDS} for ns, _ in sizes]
    plan = c.sht_plan([s[0] for s in sizes], [s[1] for s in sizes], derivatives=True)
    plan.execute(kappas, outs)
    c.sync()
    plan.close()
    for i in sorted({0, 7, 8, 20, len(sizes) - 1}):
        ns, L = sizes[i]
        ref = c.poisson_sht(kappas[i], ns, L, precision=clc.MIXED)
        c.sync()
        for k in FIELDS:
            assert rel_l2(outs[i][k], ref[k]) <= 1e-13, (order, i, k, rel_l2(outs[i][k], ref[k]))


def test_plan_splits_large_classes():
    """23 planes of one size with derivatives: two classes (21 + 2) in one plan."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    plan = c.sht_plan([64] * 23, [128] * 23, derivatives=True, graph=True)
    kappa = _planes(64, 23, seed0=2000)
    outs = [{k: torch.empty(hp.npix(64), dtype=torch.float64, device="cuda") for k in FIELDS} for _ in range(23)]
    plan.execute([k.cuda() for k in kappa], outs)
    c.sync()
    for i in (0, 20, 21, 22):
        want = sht.poisson_sht(kappa[i], 64, 128)
        for k in FIELDS:
            assert rel_l2(outs[i][k], want[k]) < TOL_MIXED, (i, k)
    plan.close()


def test_plan_potential_only_without_graph():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    sizes = [(64, 128)] * 5
    plan = c.sht_plan([s[0] for s in sizes], [s[1] for s in sizes], derivatives=False, graph=False, tune=False)
    kappa = _planes(64, 5, seed0=77)
    outs = [{"psi": torch.empty(hp.npix(64), dtype=torch.float64, device="cuda")} for _ in sizes]
    plan.execute([k.cuda() for k in kappa], outs)
    c.sync()
    for i in (0, 4):
        want = sht.poisson_sht(kappa[i], 64, 128)
        assert rel_l2(outs[i]["psi"], want["psi"]) < TOL_MIXED
    plan.close()


def test_plan_rejects_bad_batches():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    with pytest.raises(clc.CalclensError) as e:
        c.sht_plan([64] * 9, [100 + i for i in range(9)])
    assert e.value.code == clc.EINVAL
    with pytest.raises(clc.CalclensError) as e:
        c.sht_plan([32], [64])
    assert e.value.code == clc.EINVAL
    with pytest.raises(clc.CalclensError) as e:
        c.sht_plan([64] * (8 * 21 + 1), [128] * (8 * 21 + 1), derivatives=True)
    assert e.value.code == clc.EINVAL
