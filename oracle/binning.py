"""Particle binning and the plane source (oracle; test infrastructure).

Sec. 3.2 of the paper builds the convergence source of each lens plane by
depositing particle mass on the HEALPix map with exact mass conservation;
Eq. lenspoisson defines the source kappa^(m) as the projected overdensity
times Omega_m (3 H0^2 / c^2) r(chi_m) / a(chi_m) (twice the standard
convergence).  With equal-mass particles and plain (unsmoothed) binning this
is kappa_p = s * (counts_p / nbar - 1), nbar = N_particles / Npix.
"""
import torch

from . import healpix as hp

F64 = torch.float64


def bin_counts(nside, z, phi, nest=False):
    """Integer particle counts per pixel (Sec. 3.2; exact mass conservation:
    the counts sum to the number of particles)."""
    f = hp.ang2pix_nest if nest else hp.ang2pix_ring
    pix = f(nside, z, phi)
    return torch.bincount(pix, minlength=hp.npix(nside))


def kappa_from_counts(counts, nbar, scale):
    """Plane source kappa_p = scale * (counts_p / nbar - 1) (Eq. lenspoisson),
    each operation rounded separately in this order."""
    c = counts.to(F64)
    return scale * (c / nbar - 1.0)


def degrade_ring(kappa_fine, nside_fine, nside_coarse):
    """Mean of the (Nf/Ns)^2 NEST children of every coarse pixel, RING in and
    out.  For a map linear in the counts this equals binning the particles at
    the coarse Nside (exact mass conservation, Sec. 3.2)."""
    k = (nside_fine // nside_coarse) ** 2
    npc = hp.npix(nside_coarse)
    parents_nest = hp.ring2nest(nside_coarse, torch.arange(npc))
    acc = torch.zeros(npc, dtype=F64)
    for c in range(k):                       # children summed in NEST order
        child_ring = hp.nest2ring(nside_fine, parents_nest * k + c)
        acc = acc + kappa_fine[child_ring]
    return acc * (1.0 / k)
