"""Point-mass tests of the SHT+MG Poisson solver (Sec. 4.1,
Fig. 2) on the GPU path: the measurement of `test_oracle_point_mass.py`
(an Epanechnikov-smoothed unit mass, sigma = 3 pixels, normalised to unit
mass; deflection and tangential shear 8 pixels to 0.25 rad from it against
the Appendix A/E closed forms) through clc_poisson_shtmg in mixed precision
on every patch of the sphere, with the oracle's envelope and the paper's
SHT-order trend."""
import math

import pytest
import torch

from oracle import geometry, healpix as hp
from tests.gpu_util import ctx
from tests.test_oracle_sht import ep_alpha_gamma, ep_kernel

pytestmark = pytest.mark.gpu
F64 = torch.float64


def smoothed_point_mass(nf, sig_pix=3.0, seed=0):
    npx = hp.npix(nf)
    h = math.sqrt(4 * math.pi / npx)
    c = hp.pix2vec_ring(nf, torch.arange(npx))
    p0 = int(torch.randint(0, npx, (1,), generator=torch.Generator().manual_seed(seed)))
    d = torch.arccos((c @ c[p0]).clamp(-1, 1))
    w = ep_kernel(d.numpy(), sig_pix * h)
    kappa = torch.from_numpy(w / w.sum() * npx / (4 * math.pi) - 1 / (4 * math.pi))
    return kappa, c, c[p0], d, sig_pix * h, h


def point_mass_errors(fields, c, c0, d, sig, h, rmax=0.25):
    """(bias, rms, max) of the fractional errors of the radial deflection and
    the tangential shear at the pixel centres 8 pixels to rmax from the mass;
    fields: the five lens fields at every pixel centre."""
    idx = torch.nonzero((d > 8 * h) & (d < rmax)).flatten()
    n = c[idx]
    t, q = geometry.basis(n)
    er = n * (n @ c0)[:, None] - c0
    er = er / torch.linalg.vector_norm(er, dim=-1, keepdim=True)
    f = {k: v[idx] for k, v in fields.items()}
    a_r = ((f["a_th"][:, None] * t + f["a_ph"][:, None] * q) * er).sum(-1)
    cb, sb = (er * t).sum(-1), (er * q).sum(-1)
    g_t = 0.5 * (f["u_tt"] - f["u_pp"]) * (cb * cb - sb * sb) + f["u_tp"] * (2 * cb * sb)
    a_ref, g_ref = (torch.from_numpy(v) for v in ep_alpha_gamma(d[idx].numpy(), sig))
    out = {}
    for name, got, ref in (("alpha", a_r, a_ref), ("gamma_t", g_t, g_ref)):
        e = (got - ref) / ref.abs()
        out[name] = (float(e.mean()), float(e.pow(2).mean().sqrt()), float(e.abs().max()))
    return out


def _gpu_fields(c, kappa, nf, ns, lmax, nb=16, ncell=64):
    import paper_1210_3069_gb300 as clc
    sol = c.solution(nf, clc.mg_params(ns, lmax, nb, ncell=ncell, tol=1e-10, precision=clc.MIXED))
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    sol.close()
    return {k: got[k].cpu() for k in ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")}


def test_point_mass_errors_on_the_gpu_path():
    c = ctx()
    nf = 256
    kappa, cen, c0, d, sig, h = smoothed_point_mass(nf)
    fine = point_mass_errors(_gpu_fields(c, kappa, nf, 128, 256), cen, c0, d, sig, h)
    coarse = point_mass_errors(_gpu_fields(c, kappa, nf, 64, 128), cen, c0, d, sig, h)
    for name in ("alpha", "gamma_t"):
        bias, rms, mx = fine[name]
        assert abs(bias) < 2e-3 and rms < 1e-2 and mx < 5e-2, (name, fine[name])
        assert coarse[name][1] > 1.5 * rms, (name, coarse[name], fine[name])
