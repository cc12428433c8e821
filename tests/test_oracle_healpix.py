"""Pins of the oracle's HEALPix geometry and binning (Gorski et al. 2005;
paper Sec. 3, Sec. 3.1, Sec. 3.2)."""
import math

import pytest
import torch

from oracle import binning, healpix as hp
from workloads import synthetic


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32, 64])
def test_pixel_centres_round_trip(nside):
    p = torch.arange(hp.npix(nside))
    z, phi = hp.pix2ang_ring(nside, p)
    assert torch.equal(hp.ang2pix_ring(nside, z, phi), p)
    zn, pn = hp.pix2ang_nest(nside, p)
    assert torch.equal(hp.ang2pix_nest(nside, zn, pn), p)
    r = hp.nest2ring(nside, p)
    assert torch.equal(torch.sort(r).values, p)          # a permutation
    assert torch.equal(hp.ang2pix_ring(nside, zn, pn), r)
    assert torch.equal(hp.ring2nest(nside, r), p)


def test_base_layout_by_hand():
    # Nside = 1: four pixels on z = 2/3 at phi = pi/4 + k pi/2, four on the
    # equator at phi = k pi/2, four on z = -2/3 (Gorski et al. 2005, Fig. 3)
    z, phi = hp.pix2ang_ring(1, torch.arange(12))
    assert torch.allclose(z, torch.tensor([2 / 3] * 4 + [0.0] * 4 + [-2 / 3] * 4, dtype=torch.float64))
    k = torch.arange(4, dtype=torch.float64)
    exp_phi = torch.cat([math.pi / 4 + k * math.pi / 2, k * math.pi / 2, math.pi / 4 + k * math.pi / 2])
    assert torch.allclose(phi, exp_phi)
    # Nside = 2: ring lengths 4, 8, 8, 8, 8, 8, 4 and the northmost / southmost
    # children of base face 0 are RING pixels 0 and 13
    rt = hp.ring_table(2)
    assert rt["npix"].tolist() == [4, 8, 8, 8, 8, 8, 4]
    assert hp.nest2ring(2, torch.tensor([3, 0])).tolist() == [0, 13]
    assert hp.nest2ring(2, torch.arange(16)).tolist() == [13, 5, 4, 0, 15, 7, 6, 1, 17, 9, 8, 2, 19, 11, 10, 3]


def test_ring_nest_agree_on_random_points():
    z, phi = synthetic.uniform_sphere(200_000, 11)
    for nside in (1, 8, 64, 2048):
        r = hp.ang2pix_ring(nside, z, phi)
        n = hp.ang2pix_nest(nside, z, phi)
        if nside <= 64:
            assert torch.equal(hp.nest2ring(nside, n), r)
        assert int(r.min()) >= 0 and int(r.max()) < hp.npix(nside)
        assert int(n.min()) >= 0 and int(n.max()) < hp.npix(nside)


def test_pixels_are_equal_area():
    z, phi = synthetic.uniform_sphere(2_000_000, 12)
    nside = 8
    c = binning.bin_counts(nside, z, phi).double()
    mu = c.sum() / hp.npix(nside)
    chi2 = ((c - mu) ** 2 / mu).sum()
    dof = hp.npix(nside) - 1
    assert abs(float(chi2) - dof) < 6 * math.sqrt(2 * dof)


def test_edges_and_poles():
    # exact poles, phi = 0, phi just below 2 pi, and the z = +-2/3 transition
    z = torch.tensor([1.0, -1.0, 2.0 / 3.0, -2.0 / 3.0, 0.0, 0.5, 0.999999], dtype=torch.float64)
    phi = torch.tensor([0.0, 1.0, 0.0, math.nextafter(2 * math.pi, 0.0), 2 * math.pi, 3.0, 6.0], dtype=torch.float64)
    for nside in (1, 4, 256):
        r = hp.ang2pix_ring(nside, z, phi)
        n = hp.ang2pix_nest(nside, z, phi)
        assert int(r.min()) >= 0 and int(r.max()) < hp.npix(nside)
        if nside <= 64:
            assert torch.equal(hp.nest2ring(nside, n), r)


def test_binning_conserves_mass_and_zero_monopole():
    z, phi = synthetic.point_clump_config(seed=5, n_uniform=20_000, nclumps=5, per_clump=300)
    nside = 16
    c = binning.bin_counts(nside, z, phi)
    assert int(c.sum()) == z.numel()                     # exact mass conservation
    nbar = z.numel() / hp.npix(nside)
    k = binning.kappa_from_counts(c, nbar, 1.0)
    assert abs(float(k.sum())) < 1e-9 * hp.npix(nside)
    cn = binning.bin_counts(nside, z, phi, nest=True)
    assert torch.equal(cn[hp.ring2nest(nside, torch.arange(hp.npix(nside)))], c)


def test_degrade_equals_coarse_binning():
    z, phi = synthetic.uniform_sphere(50_000, 13)
    nf, ns = 32, 8
    kf = binning.kappa_from_counts(binning.bin_counts(nf, z, phi), z.numel() / hp.npix(nf), 2.0)
    ks = binning.kappa_from_counts(binning.bin_counts(ns, z, phi), z.numel() / hp.npix(ns), 2.0)
    assert torch.allclose(binning.degrade_ring(kf, nf, ns), ks, atol=1e-12, rtol=0)
