"""Partial-sky mode of the SHT+MG solver (Sec. 3.4), oracle side: the SHT
runs over the full sky and MG only on the bundles of a domain; since every
patch is solved from the same full-sky SHT solution, the domain's patches
equal those of the full-sky solve (same V-cycle count), and a light cone
that covers only part of the sky has kappa = 0 (mean density) outside."""
import math

import torch

from oracle import binning, healpix as hp, mg as omg
from workloads import synthetic

F64 = torch.float64


def _plane(nf=32):
    z, phi = synthetic.point_clump_config(seed=1210001, n_uniform=20000, nclumps=10, per_clump=500)
    return binning.kappa_from_counts(binning.bin_counts(nf, z, phi), z.numel() / hp.npix(nf), 1.0)


def test_domain_patches_equal_the_full_sky_solve():
    nf, ns, lmax, nb, ncell = 32, 8, 16, 4, 32
    kappa = _plane(nf)
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


def test_uncovered_sky_is_at_mean_density():
    nf = 16
    kappa = _plane(nf)
    z, _ = hp.pix2ang_ring(nf, torch.arange(hp.npix(nf)))
    covered = z > 0.2
    k = omg.partial_sky_kappa(kappa, nf, covered)
    assert torch.equal(k[covered], kappa[covered])
    assert float(k[~covered].abs().max()) == 0.0
