"""GPU parity of binning and the SHT Poisson solve against the oracle
(paper Sec. 3.1, Sec. 3.2).  Integer work is bit-exact; FP64 SHT results
agree to <= 1e-10 relative L2."""
import math

import pytest
import torch

from oracle import binning, healpix as hp, sht
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _edge_points():
    z = torch.tensor([1.0, -1.0, 2.0 / 3.0, -2.0 / 3.0, 0.0, 0.5, 0.999999, -0.3333333333333333],
                     dtype=torch.float64)
    phi = torch.tensor([0.0, 1.0, 0.0, math.nextafter(2 * math.pi, 0.0), 2 * math.pi, 3.0, 6.0, math.pi / 2],
                       dtype=torch.float64)
    return z, phi


@pytest.mark.parametrize("nside", [1, 2, 64, 2048, 8192])
@pytest.mark.parametrize("nest", [False, True])
def test_bin_counts_bit_exact(nside, nest):
    c = ctx()
    import paper_1210_3069_gb300 as clc
    z, phi = synthetic.point_clump_config(seed=1210001)
    ze, pe = _edge_points()
    z = torch.cat([z, ze])
    phi = torch.cat([phi, pe])
    # pixel centres and ring / face boundaries of this nside as extra cases
    if nside <= 64:
        zc, pc = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
        z = torch.cat([z, zc])
        phi = torch.cat([phi, pc])
    want = binning.bin_counts(nside, z, phi, nest=nest)
    got = c.bin_particles(z.cuda(), phi.cuda(), nside, clc.NEST if nest else clc.RING)
    c.sync()
    assert torch.equal(got.cpu().long(), want)


def test_bin_empty_and_accumulate():
    c = ctx()
    z, phi = synthetic.uniform_sphere(1000, 3)
    counts = torch.zeros(12 * 16 * 16, dtype=torch.int32, device="cuda")
    c.bin_particles(z[:0].cuda(), phi[:0].cuda(), 16, counts=counts)
    c.bin_particles(z[:500].cuda(), phi[:500].cuda(), 16, counts=counts)
    c.bin_particles(z[500:].cuda(), phi[500:].cuda(), 16, counts=counts)
    c.sync()
    assert torch.equal(counts.cpu().long(), binning.bin_counts(16, z, phi))


def test_bad_arguments_are_rejected():
    c = ctx()
    import paper_1210_3069_gb300 as clc
    z, phi = synthetic.uniform_sphere(10, 3)
    with pytest.raises(clc.CalclensError) as e:
        c.bin_particles(z.cuda(), phi.cuda(), 48)
    assert e.value.code == clc.EINVAL
    with pytest.raises(clc.CalclensError):
        c.sht_analysis(torch.zeros(12 * 64, dtype=torch.float64, device="cuda"), 8, 33)


def test_kappa_and_degrade_bit_exact():
    c = ctx()
    z, phi = synthetic.point_clump_config(seed=1210001)
    nf, ns = 64, 16
    counts = binning.bin_counts(nf, z, phi)
    nbar = z.numel() / hp.npix(nf)
    want = binning.kappa_from_counts(counts, nbar, 1.7)
    got = c.counts_to_kappa(counts.to(torch.int32).cuda(), nf, nbar, 1.7)
    deg = c.degrade(got, nf, ns)
    c.sync()
    assert torch.equal(got.cpu(), want)
    assert torch.equal(deg.cpu(), binning.degrade_ring(want, nf, ns))


def _random_alm(L, seed):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    for l in range(L + 1):
        i = sht.alm_index(L, l, 0)
        a[i] = complex(a[i].real.item(), 0.0)
    return a


@pytest.mark.parametrize("nside,lmax", [(1, 4), (2, 8), (8, 32), (16, 20), (64, 128)])
def test_sht_analysis_and_synthesis(nside, lmax):
    c = ctx()
    g = torch.Generator().manual_seed(nside + lmax)
    m = torch.randn(hp.npix(nside), dtype=torch.float64, generator=g)
    want = sht.analysis(m, nside, lmax)
    got = c.sht_analysis(m.cuda(), nside, lmax)
    a = _random_alm(lmax, 7)
    want_map = sht.synthesis(a, nside, lmax)
    got_map = c.sht_synthesis(a.cuda(), nside, lmax)
    c.sync()
    assert rel_l2(got, want) < TOL
    assert rel_l2(got_map, want_map) < TOL


@pytest.mark.parametrize("nside,lmax", [(8, 24), (64, 128)])
def test_poisson_sht_fields(nside, lmax):
    """Point-clump plane (the single-plane SHT workload at Nside 64, lmax 128)."""
    c = ctx()
    z, phi = synthetic.point_clump_config(seed=1210001)
    counts = binning.bin_counts(nside, z, phi)
    kappa = binning.kappa_from_counts(counts, z.numel() / hp.npix(nside), 1.0)
    want = sht.poisson_sht(kappa, nside, lmax)
    got = c.poisson_sht(kappa.cuda(), nside, lmax)
    c.sync()
    for k in ("psi", "a_th", "a_ph", "u_tt", "u_pp", "u_tp"):
        assert rel_l2(got[k], want[k]) < TOL, k


def test_sht_large_sampled():
    """Nside 512, lmax 1024 (the SHT grid of the SHT+MG plane): synthesis of a
    random band-limited alm checked at sampled pixels against the oracle's
    direct per-pixel sum; analysis of that map against the oracle on a
    sample of (l, m)."""
    c = ctx()
    nside, L = 512, 1024
    a = _random_alm(L, 11) * torch.exp(-torch.arange(sht.nalm(L)) * 0.0)
    got = c.sht_synthesis(a.cuda(), nside, L)
    c.sync()
    g = torch.Generator().manual_seed(5)
    pix = torch.randint(0, hp.npix(nside), (24,), generator=g)
    pix = torch.cat([pix, torch.tensor([0, 3, hp.npix(nside) - 1, 2 * nside * (nside - 1)])])
    z, phi = hp.pix2ang_ring(nside, pix)
    s = torch.sqrt((1 - z) * (1 + z))
    want = torch.zeros(pix.numel(), dtype=torch.float64)
    for m, lam in sht.legendre_columns(L, z, s):
        i0 = sht.alm_index(L, m, m)
        col = lam.T.to(torch.complex128) @ a[i0:i0 + L - m + 1]
        fac = 1.0 if m == 0 else 2.0
        want += fac * (col * torch.exp(1j * m * phi)).real
    assert rel_l2(got.cpu()[pix], want) < TOL


@pytest.mark.parametrize("nside,lmax", [(16, 40), (64, 128)])
def test_eb_analysis_matches_oracle(nside, lmax):
    """Spin-2 E/B analysis of a random shear map (paper Sec. 5)."""
    from oracle import spectra
    c = ctx()
    g = torch.Generator().manual_seed(nside)
    g1 = torch.randn(hp.npix(nside), dtype=torch.float64, generator=g)
    g2 = torch.randn(hp.npix(nside), dtype=torch.float64, generator=g)
    E, B = c.eb_analysis(g1.cuda(), g2.cuda(), nside, lmax)
    c.sync()
    wE, wB = spectra.eb_analysis(g1, g2, nside, lmax)
    assert rel_l2(E, wE) < TOL and rel_l2(B, wB) < TOL


def test_lensing_spectra_match_oracle():
    from oracle import spectra
    c = ctx()
    nside, lmax = 32, 64
    g = torch.Generator().manual_seed(9)
    A = torch.eye(2, dtype=torch.float64).expand(hp.npix(nside), 2, 2) + \
        0.01 * torch.randn(hp.npix(nside), 2, 2, dtype=torch.float64, generator=g)
    soa = A.reshape(-1, 4).T.contiguous()
    got = c.lensing_spectra(soa.cuda(), nside, lmax)
    c.sync()
    want = spectra.spectra_from_A(A, nside, lmax)
    for k in ("kappa", "E", "B", "omega"):
        assert rel_l2(got[k], want[k]) < TOL, k


def test_lensing_spectra_in_image_basis_match_oracle():
    """A given in the basis at the rays' source-sphere positions x: the call
    carries it to the pixel centres (Appendix B transport) before the
    spectra, as the oracle's image_basis does."""
    from oracle import rays as orays, spectra
    c = ctx()
    nside, lmax = 32, 64
    g = torch.Generator().manual_seed(10)
    npx = hp.npix(nside)
    A = torch.eye(2, dtype=torch.float64).expand(npx, 2, 2) + \
        0.01 * torch.randn(npx, 2, 2, dtype=torch.float64, generator=g)
    n0 = hp.pix2vec_ring(nside, torch.arange(npx))
    x = 700.0 * (n0 + 0.02 * torch.randn(npx, 3, dtype=torch.float64, generator=g))
    nx = x / torch.linalg.vector_norm(x, dim=-1, keepdim=True)
    got = c.lensing_spectra(A.reshape(-1, 4).T.contiguous().cuda(), nside, lmax, x=x.T.contiguous().cuda())
    c.sync()
    want = spectra.spectra_from_A(orays.image_basis(A, nx, n0), nside, lmax)
    for k in ("kappa", "E", "B", "omega"):
        assert rel_l2(got[k], want[k]) < TOL, k


def test_fp64_sht_in_order_ranges_is_identical():
    """With the FP64 Legendre table limited to a fraction of its size the SHT
    runs over order ranges; every result is bit-identical to the whole-table
    run (each order's sums do not depend on the others)."""
    c = ctx()
    nside, lmax = 64, 128
    z, phi = synthetic.point_clump_config(seed=1210001)
    counts = binning.bin_counts(nside, z, phi)
    kappa = binning.kappa_from_counts(counts, z.numel() / hp.npix(nside), 1.0).cuda()
    whole = c.poisson_sht(kappa, nside, lmax)
    alm = c.sht_analysis(kappa, nside, lmax)
    m = c.sht_synthesis(alm, nside, lmax)
    c.sync()
    try:
        c.set_table_budget(2 << 20)   # about a quarter of the 8.7 MB table
        part = c.poisson_sht(kappa, nside, lmax)
        alm2 = c.sht_analysis(kappa, nside, lmax)
        m2 = c.sht_synthesis(alm2, nside, lmax)
        c.sync()
    finally:
        c.set_table_budget(0)
    for k in whole:
        assert torch.equal(whole[k], part[k]), k
    assert torch.equal(alm, alm2) and torch.equal(m, m2)
