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


def test_point_mass_trends_at_nside2048():
    """The Sec. 4.1 / Fig. 2 measurements at the throughput configuration's
    scale: a smoothed unit mass on the Nside-2048 sphere solved by SHT+MG on
    every patch (mixed precision), deflection and tangential shear against the
    closed forms.  Trends: a finer SHT grid (nside_sht 1024 against 512)
    lowers the errors; larger bundles (Nside 16 with 512-cell patches against
    Nside 32 with 256, the same MG cell) move the errors outwards; the paper's
    stopping rule with eps = 0.1 and 0.01 stops after a few V-cycles at the
    converged solution's errors."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf = 2048
    kappa, cen, c0, d, sig, h = smoothed_point_mass(nf, seed=1)
    idx = torch.nonzero((d > 8 * h) & (d < 0.25)).flatten()
    kd = kappa.cuda()
    idx_d = idx.cuda()

    def run(ns, lmax, nb, ncell, **kw):
        # tol 1e-9: the mixed solver's float-float residual bottoms out near
        # 1.2e-10 on this source (a 3-pixel mass of peak kappa 3e5); errors of
        # the measurement sit at 1e-3
        kw.setdefault("tol", 1e-9)
        sol = c.solution(nf, clc.mg_params(ns, lmax, nb, ncell=ncell, precision=clc.MIXED, **kw))
        got = c.poisson_shtmg(kd, nf, sol, derivatives=True)
        c.sync()
        cyc = sol.info()[0]
        sol.close()
        sel = {k: v[idx_d].cpu() for k, v in got.items()}
        # point_mass_errors indexes full maps: hand it maps that hold the selected values
        maps = {}
        for k, v in sel.items():
            m = torch.zeros(d.numel(), dtype=F64)
            m[idx] = v
            maps[k] = m
        out = point_mass_errors(maps, cen, c0, d, sig, h)
        a_ref = torch.from_numpy(ep_alpha_gamma(d[idx].numpy(), sig)[0])
        t, q = geometry.basis(cen[idx])
        er = cen[idx] * (cen[idx] @ c0)[:, None] - c0
        er = er / torch.linalg.vector_norm(er, dim=-1, keepdim=True)
        a_r = ((sel["a_th"][:, None] * t + sel["a_ph"][:, None] * q) * er).sum(-1)
        e2 = ((a_r - a_ref) / a_ref.abs()) ** 2
        out["centroid"] = float((e2 * d[idx]).sum() / e2.sum())
        out["cycles"] = cyc
        return out

    base = run(512, 1024, 32, 256)
    fine_sht = run(1024, 2048, 32, 256)
    big = run(512, 1024, 16, 512)
    e1 = run(512, 1024, 32, 256, stop_rule=clc.STOP_TAU, eps=0.1, refine_cycles=1)
    e2 = run(512, 1024, 32, 256, stop_rule=clc.STOP_TAU, eps=0.01, refine_cycles=1)
    for tag, r in (("base", base), ("sht1024", fine_sht), ("nb16", big), ("eps0.1", e1), ("eps0.01", e2)):
        print("point mass Nside 2048", tag, r)
    # measured on GB300: RMS alpha 0.064 %, gamma_t 0.089 %, max 0.9 % / 1.9 %, |bias| < 0.01 %; the
    # finer SHT grid takes gamma_t's RMS to 0.077 % and alpha's to 0.063 %; eps = 0.1 stops after 3
    # V-cycles (gamma_t RMS 7.5 % above the converged 12-cycle solution's), eps = 0.01 after 4 at it
    for name in ("alpha", "gamma_t"):
        bias, rms, mx = base[name]
        assert abs(bias) < 1e-3 and rms < 1e-2 and mx < 5e-2, (name, base[name])
        assert fine_sht[name][1] < base[name][1], (name, fine_sht[name], base[name])
        assert abs(e1[name][1] - base[name][1]) < 0.1 * base[name][1], (name, e1[name], base[name])
        assert abs(e2[name][1] - base[name][1]) < 0.01 * base[name][1], (name, e2[name], base[name])
        assert abs(e2[name][1] - base[name][1]) <= abs(e1[name][1] - base[name][1]) + 1e-12, name
    assert fine_sht["gamma_t"][1] < 0.9 * base["gamma_t"][1]
    assert e1["cycles"] < e2["cycles"] < base["cycles"]
    assert big["centroid"] > 1.3 * base["centroid"], (big["centroid"], base["centroid"])
