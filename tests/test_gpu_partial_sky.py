"""Partial sky on the GPU (paper Sec. 3.4): the light cone's source with the
uncovered sky at the mean density, the SHT over the full sky and MG patches
only for the bundles of a domain.  Against the oracle (same domain), against
the full-sky GPU solve on the domain's pixels (bit for bit at a fixed cycle
count: every patch is solved independently), and the ray step with rays
outside the domain left undeflected and counted."""
import math

import pytest
import torch

import oracle.rays as orays
from oracle import binning, healpix as hp, mg as omg
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
KEYS = ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")
NF, NS, LMAX, NB, NCELL = 64, 16, 32, 4, 32
CENTRE = torch.tensor([0.3, 0.5, math.sqrt(1 - 0.34)], dtype=torch.float64)


def _plane(seed=31):
    z, phi = synthetic.lognormal_particles(300_000, seed)
    counts = binning.bin_counts(NF, z, phi)
    zp, _ = hp.pix2ang_ring(NF, torch.arange(hp.npix(NF)))
    covered = zp > -0.2
    return counts, covered


def _domain_pixels(dom):
    p = torch.arange(hp.npix(NF))
    home = omg.home_bundle(NF, NB, hp.ring2nest(NF, p))
    inside = torch.isin(home, dom)
    return p, home, inside


def test_masked_source_is_bit_exact():
    c = ctx()
    counts, covered = _plane()
    got = c.counts_to_kappa_masked(counts.to(torch.int32).cuda(), covered.cuda(), NF, 2.5)
    c.sync()
    want = omg.partial_sky_kappa(counts, covered, 2.5)
    assert torch.equal(got.cpu(), want)


def test_domain_solve_matches_oracle_and_full_sky():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    counts, covered = _plane()
    kappa = omg.partial_sky_kappa(counts, covered, 1.0)
    dom = omg.domain_bundles(NB, CENTRE, 0.6)
    assert 0 < dom.numel() < 12 * NB * NB
    P = clc.mg_params(NS, LMAX, NB, ncell=NCELL, fixed_cycles=3)
    sd = c.solution(NF, P, domain=dom.tolist())
    got = c.poisson_shtmg(kappa.cuda(), NF, sd, derivatives=True)
    c.sync()
    assert sd.domain() == (dom.numel(), int((~_domain_pixels(dom)[2]).sum()))   # pixels outside: lookups counted
    sf = c.solution(NF, P)
    full = c.poisson_shtmg(kappa.cuda(), NF, sf, derivatives=True)
    c.sync()
    p, home, inside = _domain_pixels(dom)
    ref = omg.solve_plane(kappa, NF, NS, LMAX, NB, ncell=NCELL, fixed_cycles=3, bundles=dom)
    want = omg.fields_at(ref, NB, hp.pix2vec_ring(NF, p[inside]), home[inside])
    for k in KEYS:
        g = got[k].cpu()
        assert rel_l2(g[inside], want[k]) < 1e-10, k
        assert torch.equal(g[inside], full[k].cpu()[inside]), k      # patch by patch identical
        assert float(g[~inside].abs().max()) == 0.0, k               # no patch: no deflection
    sd.close()
    sf.close()


def test_domain_solve_mixed_converged():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    counts, covered = _plane(32)
    kappa = omg.partial_sky_kappa(counts, covered, 1.0)
    dom = omg.domain_bundles(NB, CENTRE, 0.8)
    sd = c.solution(NF, clc.mg_params(NS, LMAX, NB, ncell=NCELL, tol=1e-10, precision=clc.MIXED), domain=dom.tolist())
    got = c.poisson_shtmg(kappa.cuda(), NF, sd, derivatives=True)
    c.sync()
    assert sd.info()[1] < 1e-10
    p, home, inside = _domain_pixels(dom)
    ref = omg.solve_plane(kappa, NF, NS, LMAX, NB, ncell=NCELL, tol=1e-12, bundles=dom)
    want = omg.fields_at(ref, NB, hp.pix2vec_ring(NF, p[inside]), home[inside])
    for k in KEYS:
        assert rel_l2(got[k].cpu()[inside], want[k]) < 1e-8, k
    sd.close()


def test_rays_on_a_partial_sky():
    """One ray step on the domain solution: rays of the domain's bundles
    follow the oracle; rays outside see zero lens fields (straight on, A = I)
    and are counted."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    counts, covered = _plane(33)
    kappa = 0.05 * omg.partial_sky_kappa(counts, covered, 1.0)
    dom = omg.domain_bundles(NB, CENTRE, 0.6)
    P = clc.mg_params(NS, LMAX, NB, ncell=NCELL, fixed_cycles=4)
    sd = c.solution(NF, P, domain=dom.tolist())
    c.poisson_shtmg(kappa.cuda(), NF, sd)
    chi = [200.0, 300.0]
    rs = c.rays(hp.npix(NF))
    c.rays_init_pixels(rs, NF, chi[0], NB)
    c.ray_step(rs, 0.0, chi[0], chi[1], sol=sd)
    c.sync()
    p, home, inside = _domain_pixels(dom)
    assert sd.domain()[1] == int((~inside).sum())
    ref = omg.solve_plane(kappa, NF, NS, LMAX, NB, ncell=NCELL, fixed_cycles=4, bundles=dom)
    n0 = hp.pix2vec_ring(NF, p[inside])
    st = orays.trace(n0, chi, [lambda n: omg.fields_at(ref, NB, n, home[inside])])
    x = rs.x.T.cpu()
    assert rel_l2(x[inside], st["x"]) < 1e-10
    assert rel_l2(rs.A.T.cpu()[inside].reshape(-1, 2, 2), st["A"]) < 1e-10
    out = ~inside
    n_out = hp.pix2vec_ring(NF, p[out])
    assert float((x[out] - chi[1] * n_out).abs().max()) < 1e-12 * chi[1]
    eye = torch.tensor([1.0, 0.0, 0.0, 1.0], dtype=torch.float64)
    assert float((rs.A.T.cpu()[out] - eye).abs().max()) < 1e-14
    sd.close()


def test_bad_domains_are_rejected():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    P = clc.mg_params(NS, LMAX, NB, ncell=NCELL)
    with pytest.raises(clc.CalclensError):
        c.solution(NF, P, domain=[0, 0])                  # repeated bundle
    with pytest.raises(clc.CalclensError):
        c.solution(NF, P, domain=[12 * NB * NB])          # beyond the sphere
