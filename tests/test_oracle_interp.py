"""Pins of the oracle's HEALPix ring-bilinear interpolation (the four-pixel
interpolation of Sec. 3.2 and 3.3: patch boundary values and starting guess,
patch sources, the pure-SHT ray lookup, the image matrices): exact at pixel
centres, exact for fields linear in theta between two rings and linear in
phi along a ring, continuous across the first ring's pole blend and across
phi = 0 / 2 pi, equal to the ring-1 mean at the pole, and second-order
accurate on a spherical harmonic."""
import math

import numpy as np
import pytest
import scipy.special as sp
import torch

from oracle import healpix as hp, interp

F64 = torch.float64


@pytest.mark.parametrize("nside", [1, 2, 8])
def test_exact_at_pixel_centres(nside):
    g = torch.Generator().manual_seed(nside)
    m = torch.randn(hp.npix(nside), dtype=F64, generator=g)
    p = torch.arange(hp.npix(nside))
    ring, _ = hp.pix2ring(nside, p)
    _, phi = hp.pix2ang_ring(nside, p)
    got = interp.interpolate(nside, m, interp.ring_theta(nside)[ring - 1], phi)
    assert torch.allclose(got, m, rtol=0, atol=1e-13)   # rounding of the longitude fraction


def test_linear_in_theta_between_rings():
    """A map a + b theta_ring is reproduced exactly at any point between the
    first and the last ring (the two bracketing rings, linear weights)."""
    nside = 8
    p = torch.arange(hp.npix(nside))
    ring, _ = hp.pix2ring(nside, p)
    th_r = interp.ring_theta(nside)
    m = 0.3 + 1.7 * th_r[ring - 1]
    g = torch.Generator().manual_seed(1)
    th = th_r[0] + (th_r[-1] - th_r[0]) * torch.rand(500, generator=g, dtype=F64)
    ph = 2 * math.pi * torch.rand(500, generator=g, dtype=F64)
    got = interp.interpolate(nside, m, th, ph)
    assert torch.allclose(got, 0.3 + 1.7 * th, rtol=0, atol=1e-13)


@pytest.mark.parametrize("ring", [1, 3, 8, 15, 30])
def test_linear_in_phi_along_a_ring(ring):
    """On a ring's colatitude, a map equal to c phi_p on that ring is
    reproduced at every phi between its first and last pixel (no wrap)."""
    nside = 8
    rt = hp.ring_table(nside)
    r = ring - 1
    n, first = int(rt["npix"][r]), int(rt["first"][r])
    _, phi_p = hp.pix2ang_ring(nside, torch.arange(first, first + n))
    m = torch.full((hp.npix(nside),), 99.0, dtype=F64)
    m[first:first + n] = 2.5 * phi_p
    th = interp.ring_theta(nside)[r].expand(200)
    g = torch.Generator().manual_seed(ring)
    ph = phi_p[0] + (phi_p[-1] - phi_p[0]) * torch.rand(200, generator=g, dtype=F64)
    got = interp.interpolate(nside, m, th, ph)
    assert torch.allclose(got, 2.5 * ph, rtol=0, atol=1e-13)


def test_continuous_across_first_ring_pole_and_phi_wrap():
    nside = 8
    g = torch.Generator().manual_seed(2)
    m = torch.randn(hp.npix(nside), dtype=F64, generator=g)
    th_r = interp.ring_theta(nside)
    ph = 2 * math.pi * torch.rand(50, generator=g, dtype=F64)
    eps = 1e-9
    for t in (th_r[0], th_r[-1], th_r[3], th_r[nside]):
        a = interp.interpolate(nside, m, (t - eps).expand(50), ph)
        b = interp.interpolate(nside, m, (t + eps).expand(50), ph)
        assert float((a - b).abs().max()) < 1e-6
    th = th_r[0] + (th_r[-1] - th_r[0]) * torch.rand(50, generator=g, dtype=F64)
    a = interp.interpolate(nside, m, th, torch.full((50,), eps, dtype=F64))
    b = interp.interpolate(nside, m, th, torch.full((50,), 2 * math.pi - eps, dtype=F64))
    assert float((a - b).abs().max()) < 1e-6
    # at either pole every longitude gives the mean of the nearest ring
    rt = hp.ring_table(nside)
    north = interp.interpolate(nside, m, torch.zeros(50, dtype=F64), ph)
    south = interp.interpolate(nside, m, torch.full((50,), math.pi, dtype=F64), ph)
    last = int(rt["first"][-1])
    assert torch.allclose(north, m[:4].mean().expand(50), rtol=0, atol=1e-14)
    assert torch.allclose(south, m[last:last + 4].mean().expand(50), rtol=0, atol=1e-14)


def test_second_order_on_a_spherical_harmonic():
    """Error on Re Y_43 sampled at pixel centres and interpolated at random
    points away from the poles falls by about four per doubling of Nside."""
    g = torch.Generator().manual_seed(3)
    z = 1.6 * torch.rand(400, generator=g, dtype=F64) - 0.8
    ph = 2 * math.pi * torch.rand(400, generator=g, dtype=F64)
    th = torch.arccos(z)
    exact = torch.from_numpy(sp.sph_harm_y(4, 3, th.numpy(), ph.numpy()).real.copy())
    errs = []
    for nside in (16, 32, 64):
        zp, pp = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
        m = torch.from_numpy(sp.sph_harm_y(4, 3, np.arccos(zp.numpy()), pp.numpy()).real.copy())
        errs.append(float((interp.interpolate(nside, m, th, ph) - exact).abs().max()))
    for a, b in zip(errs, errs[1:]):
        assert 3.3 < a / b < 4.7, errs
