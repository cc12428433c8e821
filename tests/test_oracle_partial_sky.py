"""Partial-sky mode of the SHT+MG solver (Sec. 3.4), oracle side.

The paper fills the sky outside a light cone's domain with matter at the
mean density of the universe, so that rays crossing it are not deflected,
and runs the SHT over the full sky but MG only on the domain's bundles.
Pins: the partial-sky source has zero monopole; for an axisymmetric source in
a polar cap, Gauss's law on the sphere gives alpha = 0 everywhere outside the
cap and alpha_theta(theta) = -(1 / sin theta) int_0^theta kappa sin inside,
which the oracle's solution reproduces (and a source referred to the
full-sky mean does not); the domain's patches of a masked plane equal those
of the full-sky solve of the same source."""
import math

import pytest
import torch
from scipy.integrate import quad

from oracle import binning, healpix as hp, mg as omg, sht
from workloads import synthetic

F64 = torch.float64


def _counts(nf=32):
    z, phi = synthetic.point_clump_config(seed=1210001, n_uniform=20000, nclumps=10, per_clump=500)
    return binning.bin_counts(nf, z, phi), z, phi


def test_partial_sky_source_has_zero_monopole_and_mean_density_outside():
    nf = 32
    counts, z, phi = _counts(nf)
    zp, _ = hp.pix2ang_ring(nf, torch.arange(hp.npix(nf)))
    covered = zp > 0.2
    k = omg.partial_sky_kappa(counts, covered, 2.5)
    assert float(k[~covered].abs().max()) == 0.0
    assert abs(float(k.sum())) < 1e-12 * float(k.abs().sum())
    # a light cone that holds only the covered sky's particles, binned with
    # its own mean density, gives the same source inside
    inside = hp.ang2pix_ring(nf, z, phi)
    keep = covered[inside]
    c_in = binning.bin_counts(nf, z[keep], phi[keep])
    nbar = keep.sum().double() / covered.sum()
    want = binning.kappa_from_counts(c_in, nbar, 2.5)
    assert torch.allclose(k[covered], want[covered], rtol=0, atol=1e-13)


def test_axisymmetric_cap_gauss_law():
    """No deflection outside a covered polar cap whose density depends on
    the colatitude only; Gauss's law inside (Sec. 3.4: matter at the mean
    density outside the domain does not deflect rays)."""
    nside, L, zc = 32, 96, 0.2
    z, _ = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    rho = 1.0 + 0.5 * torch.sin(6.0 * z)
    cov = z > zc
    k = omg.partial_sky_kappa(rho, cov, 1.0)
    a = sht.poisson_sht(k, nside, L)["a_th"]
    nbar = float(rho[cov].mean())
    tc = math.acos(zc)

    def kap(t):
        return (1.0 + 0.5 * math.sin(6.0 * math.cos(t))) / nbar - 1.0 if t < tc else 0.0

    def gauss(t):
        return -quad(lambda x: kap(x) * math.sin(x), 0.0, min(t, tc), limit=200)[0] / math.sin(t)

    th = torch.arccos(z)
    far_out = z < zc - 0.15
    far_in = z > zc + 0.15
    amax = float(a.abs().max())
    assert float(a[far_out].abs().max()) < 2e-3 * amax
    want = torch.tensor([gauss(float(t)) for t in th[far_in]], dtype=F64)
    assert float((a[far_in] - want).abs().max()) < 5e-3 * amax
    # referred to the full-sky mean, the source keeps a monopole and the
    # exterior is deflected: the pin above tells the two apart
    k_wrong = torch.where(cov, rho / rho.mean() - 1.0, torch.zeros_like(rho))
    a_wrong = sht.poisson_sht(k_wrong, nside, L)["a_th"]
    assert float(a_wrong[far_out].abs().max()) > 0.05 * amax


def test_domain_patches_equal_the_full_sky_solve():
    nf, ns, lmax, nb, ncell = 32, 8, 16, 4, 32
    counts, _, _ = _counts(nf)
    zp, _ = hp.pix2ang_ring(nf, torch.arange(hp.npix(nf)))
    kappa = omg.partial_sky_kappa(counts, zp > -0.3, 1.0)
    full = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, fixed_cycles=4)
    dom = omg.domain_bundles(nb, torch.tensor([0.3, 0.5, math.sqrt(1 - 0.34)], dtype=F64), 0.6)
    assert 0 < dom.numel() < 12 * nb * nb
    part = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, fixed_cycles=4, bundles=dom)
    assert torch.allclose(part["u"], full["u"][dom], rtol=0, atol=1e-14)
    # and the fields at the domain's pixel centres
    p = torch.arange(hp.npix(nf))
    home = omg.home_bundle(nf, nb, hp.ring2nest(nf, p))
    sel = torch.isin(home, dom)
    n = hp.pix2vec_ring(nf, p[sel])
    a = omg.fields_at(part, nb, n, home[sel])
    b = omg.fields_at(full, nb, n, home[sel])
    for k in a:
        assert torch.allclose(a[k], b[k], rtol=0, atol=1e-12)
