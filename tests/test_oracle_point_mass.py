"""Point-mass tests of the SHT+MG Poisson solver (Sec. 4.1,
Fig. 2), on the oracle at a reduced scale.

A unit mass smoothed by the Epanechnikov kernel (Appendix E, sigma = 3
pixels, sampled at the pixel centres and normalised to unit mass as the
mass-conserving deposit of Sec. 3.2 does) minus the mean density is solved
with SHT+MG on the bundles around it; the deflection's radial component and
the tangential shear at the pixel centres between 8 pixels and 0.25 rad
from the mass are compared with the closed forms of Appendices A and E.
The paper reports, at its resolutions, RMS fractional errors of 1-2 %, a
bias below 0.1 % and maxima below 5 %, smaller errors for a finer SHT grid,
and errors that fall with the MG convergence until they reach the
truncation error.  Here: Nside 256 fine map and MG cells of one fine pixel
(patches of 64 cells for bundles of Nside 16), SHT on Nside 64 or 128."""
import math

import numpy as np
import pytest
import torch

from oracle import geometry, healpix as hp, mg as omg
from tests.test_oracle_sht import ep_alpha_gamma, ep_kernel

F64 = torch.float64


def _point_mass_errors(nside_sht, lmax, fixed_cycles=None, nf=256, nb=16, ncell=64, sig_pix=3.0, rmax=0.25,
                       seed=0, stop="residual", eps=0.1):
    npx = hp.npix(nf)
    h = math.sqrt(4 * math.pi / npx)
    c = hp.pix2vec_ring(nf, torch.arange(npx))
    p0 = int(torch.randint(0, npx, (1,), generator=torch.Generator().manual_seed(seed)))
    c0 = c[p0]
    sig = sig_pix * h
    d = torch.arccos((c @ c0).clamp(-1, 1))
    w = ep_kernel(d.numpy(), sig)
    kappa = torch.from_numpy(w / w.sum() * npx / (4 * math.pi) - 1 / (4 * math.pi))
    zb, pb = hp.pix2ang_nest(nb, torch.arange(12 * nb * nb))
    bund = torch.nonzero(torch.arccos((hp.vec_from_zphi(zb, pb) @ c0).clamp(-1, 1)) < rmax + 0.1).flatten()
    sol = omg.solve_plane(kappa, nf, nside_sht, lmax, nb, ncell=ncell, tol=1e-10, bundles=bund,
                          fixed_cycles=fixed_cycles, stop=stop, eps=eps)
    home = omg.home_bundle(nf, nb, hp.ring2nest(nf, torch.arange(npx)))
    idx = torch.nonzero((d > 8 * h) & (d < rmax) & torch.isin(home, bund)).flatten()
    n = c[idx]
    f = omg.fields_at(sol, nb, n, home[idx])
    t, q = geometry.basis(n)
    er = n * (n @ c0)[:, None] - c0                      # tangent direction away from the mass
    er = er / torch.linalg.vector_norm(er, dim=-1, keepdim=True)
    a_r = ((f["a_th"][:, None] * t + f["a_ph"][:, None] * q) * er).sum(-1)
    cb, sb = (er * t).sum(-1), (er * q).sum(-1)
    g_t = 0.5 * (f["u_tt"] - f["u_pp"]) * (cb * cb - sb * sb) + f["u_tp"] * (2 * cb * sb)
    a_ref, g_ref = (torch.from_numpy(v) for v in ep_alpha_gamma(d[idx].numpy(), sig))
    out = {}
    for name, got, ref in (("alpha", a_r, a_ref), ("gamma_t", g_t, g_ref)):
        e = (got - ref) / ref.abs()
        out[name] = (float(e.mean()), float(e.pow(2).mean().sqrt()), float(e.abs().max()))
    out["cycles"] = sol["cycles"]
    return out


@pytest.fixture(scope="module")
def errors():
    return {"ns128": _point_mass_errors(128, 256), "ns64": _point_mass_errors(64, 128),
            "one_cycle": _point_mass_errors(64, 128, fixed_cycles=1),
            "eps0.1": _point_mass_errors(128, 256, stop="tau", eps=0.1),
            "eps0.01": _point_mass_errors(128, 256, stop="tau", eps=0.01)}


def test_point_mass_error_envelope(errors):
    for name in ("alpha", "gamma_t"):
        bias, rms, mx = errors["ns128"][name]
        assert abs(bias) < 2e-3 and rms < 1e-2 and mx < 5e-2, (name, bias, rms, mx)


def test_finer_sht_grid_reduces_the_errors(errors):
    for name in ("alpha", "gamma_t"):
        assert errors["ns64"][name][1] > 1.5 * errors["ns128"][name][1], name


def test_errors_fall_with_convergence_to_the_truncation_level(errors):
    assert errors["one_cycle"]["gamma_t"][1] > 2.0 * errors["ns64"]["gamma_t"][1]
    assert errors["ns64"]["gamma_t"][1] < 2e-2


def test_tau_rule_reaches_the_truncation_level_in_few_cycles(errors):
    """The paper's stopping rule ||r|| < eps ||tau||: eps = 0.1 stops after a
    few V-cycles (a 1e-10 residual needs about ten) with errors already at
    the converged (truncation) level, and eps = 0.01 no further from it."""
    conv, e1, e2 = errors["ns128"], errors["eps0.1"], errors["eps0.01"]
    assert e1["cycles"] <= e2["cycles"] < conv["cycles"]
    for name in ("alpha", "gamma_t"):
        assert abs(e1[name][1] - conv[name][1]) < 0.02 * conv[name][1], (name, e1[name], conv[name])
        assert abs(e2[name][1] - conv[name][1]) <= abs(e1[name][1] - conv[name][1]) + 1e-12, name


def _radial_centroid(nb, ncell, nf=256, ns=128, lmax=256, rmax=0.25):
    """Centroid in distance from the mass of the squared fractional
    deflection error (the radius where the errors sit)."""
    npx = hp.npix(nf)
    h = math.sqrt(4 * math.pi / npx)
    c = hp.pix2vec_ring(nf, torch.arange(npx))
    c0 = c[int(torch.randint(0, npx, (1,), generator=torch.Generator().manual_seed(0)))]
    sig = 3.0 * h
    d = torch.arccos((c @ c0).clamp(-1, 1))
    w = ep_kernel(d.numpy(), sig)
    kappa = torch.from_numpy(w / w.sum() * npx / (4 * math.pi) - 1 / (4 * math.pi))
    zb, pb = hp.pix2ang_nest(nb, torch.arange(12 * nb * nb))
    bund = torch.nonzero(torch.arccos((hp.vec_from_zphi(zb, pb) @ c0).clamp(-1, 1)) < rmax + 0.1).flatten()
    sol = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, tol=1e-10, bundles=bund)
    home = omg.home_bundle(nf, nb, hp.ring2nest(nf, torch.arange(npx)))
    idx = torch.nonzero((d > 8 * h) & (d < rmax) & torch.isin(home, bund)).flatten()
    n = c[idx]
    f = omg.fields_at(sol, nb, n, home[idx])
    t, q = geometry.basis(n)
    er = n * (n @ c0)[:, None] - c0
    er = er / torch.linalg.vector_norm(er, dim=-1, keepdim=True)
    a_r = ((f["a_th"][:, None] * t + f["a_ph"][:, None] * q) * er).sum(-1)
    a_ref = torch.from_numpy(ep_alpha_gamma(d[idx].numpy(), sig)[0])
    e2 = ((a_r - a_ref) / a_ref.abs()) ** 2
    return float((e2 * d[idx]).sum() / e2.sum())


def test_larger_bundles_move_the_errors_outwards():
    """Sec. 4.1: with larger bundle cells (and patches, at the same MG cell
    size) the radius at which the errors are largest moves out accordingly."""
    small = _radial_centroid(16, 64)
    large = _radial_centroid(8, 128)
    assert large > 1.3 * small, (small, large)

