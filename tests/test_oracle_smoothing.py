"""Pins of the Epanechnikov smoothing oracle (paper Sec. 3.2): exact mass
conservation, reduction to plain binning when the kernel is below the pixel
scale, symmetry about the pole, the kernel's shape against an independent
(haversine) angular distance, and the HEALPix quadrature of the kernel
normalised on the sphere."""
import math

import torch

from oracle import binning, healpix as hp, smoothing as sm
from workloads import synthetic

F64 = torch.float64


def test_mass_is_conserved_exactly():
    z, phi = synthetic.uniform_sphere(300, 41)
    for nside, sigma in ((8, 0.4), (32, 0.05), (32, 0.01)):
        m = sm.smooth_particles(nside, z, phi, sigma)
        assert abs(float(m.sum()) - 300.0) < 1e-11
        assert float(m.min()) >= 0.0


def test_tiny_kernel_is_plain_binning():
    """No pixel centre within sigma: every particle lands on its own pixel."""
    nside = 16
    z, phi = synthetic.uniform_sphere(500, 42)
    m = sm.smooth_particles(nside, z, phi, 1e-9)
    assert torch.equal(m, binning.bin_counts(nside, z, phi).to(F64))


def test_particle_at_the_pole_spreads_symmetrically():
    """A particle at z = 1: the four pixels of each polar ring sit at the same
    distance and receive equal shares."""
    nside = 16
    m = sm.smooth_particles(nside, torch.tensor([1.0], dtype=F64), torch.tensor([0.3], dtype=F64), 0.25)
    for i in range(1, 4):
        first = 2 * i * (i - 1)
        vals = m[first:first + 4 * i]
        assert float(vals.max() - vals.min()) <= 1e-15 * float(vals.max())
        assert float(vals.max()) > 0.0


def test_kernel_shape_against_haversine_distance():
    """Deposit of a particle at a pixel centre: value_q / value_centre =
    1 - (theta_q / sigma)^2 with theta from the haversine formula."""
    nside, sigma = 32, 0.12
    p0 = 3000
    z0, ph0 = hp.pix2ang_ring(nside, torch.tensor([p0]))
    m = sm.smooth_particles(nside, z0, ph0, sigma)
    zq, phq = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    th0, thq = torch.arccos(z0), torch.arccos(zq)
    hav = torch.sin((thq - th0) / 2) ** 2 + torch.sin(th0) * torch.sin(thq) * torch.sin((phq - ph0) / 2) ** 2
    theta = 2 * torch.arcsin(torch.sqrt(hav))
    inside = theta < sigma - 1e-9
    ratio = m[inside] / m[p0]
    assert torch.allclose(ratio, 1.0 - (theta[inside] / sigma) ** 2, rtol=0, atol=1e-12)
    assert float(m[theta > sigma + 1e-9].abs().max()) == 0.0


def test_kernel_normalisation_by_healpix_quadrature():
    """sum_q K(theta_q) Omega_pix -> 1 for a kernel much wider than the pixels
    (the N(sigma) of Sec. 3.2 normalises the kernel on the sphere)."""
    nside, sigma = 256, 0.6
    zq, phq = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    a = hp.vec_from_zphi(zq, phq)
    pole = torch.tensor([0.0, 0.0, 1.0], dtype=F64).expand_as(a)
    q = float(sm.kernel(sm.angular_distance(pole, a), sigma).sum()) * 4 * math.pi / hp.npix(nside)
    assert abs(q - 1.0) < 2e-5, q


def test_density_to_kappa():
    rho = torch.tensor([0.0, 2.0, 4.5], dtype=F64)
    assert torch.equal(sm.kappa_from_density(rho, 2.0, 3.0), torch.tensor([-3.0, 0.0, 3.75], dtype=F64))
