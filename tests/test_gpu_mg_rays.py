"""GPU parity of the SHT+MG solver, the lens-field lookup and the ray
recursion against the oracle (paper Sec. 2.2, Sec. 3.2, Appendix A, B)."""
import math

import pytest
import torch

import oracle.rays as orays
from oracle import binning, geometry, healpix as hp, mg as omg, sht
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-10
KEYS = ("a_th", "a_ph", "u_tt", "u_pp", "u_tp")


def _kappa(nside, seed, n=200_000):
    z, phi = synthetic.lognormal_particles(n, seed)
    c = binning.bin_counts(nside, z, phi)
    return binning.kappa_from_counts(c, z.numel() / hp.npix(nside), 1.0)


def _params(clc, ns, lmax, nb, ncell, fixed=0, tol=1e-10, nu1=2, nu2=2, prec=0, max_cycles=60):
    return clc.mg_params(ns, lmax, nb, ncell=ncell, nu1=nu1, nu2=nu2, fixed_cycles=fixed, tol=tol, precision=prec,
                         max_cycles=max_cycles)


def _pixel_home(nf, nb):
    p = torch.arange(hp.npix(nf))
    nest = hp.ring2nest(nf, p)
    return omg.home_bundle(nf, nb, nest), hp.pix2vec_ring(nf, p)


@pytest.mark.parametrize("nf,ns,lmax,nb,ncell,cycles,nu1,nu2", [
    (64, 16, 32, 4, 32, 3, 2, 2),
    (32, 8, 16, 2, 64, 2, 2, 2),
    # several 64 x 64 blocks per patch on the two finest levels, unequal
    # halos (2 nu1 + 1 = 7 before, 2 nu2 = 2 after the coarse step)
    (64, 16, 32, 2, 256, 2, 3, 1),
    # no pre-smoothing (restriction only) / no post-smoothing
    (32, 8, 16, 2, 128, 2, 0, 2),
    (32, 8, 16, 2, 128, 2, 2, 0),
    # finest level wider than a row band: square blocks there, bands below
    (64, 16, 32, 2, 512, 1, 2, 2),
    # 8 sweeps: the FP64 row band would not fit in shared memory, square blocks
    (32, 8, 16, 2, 256, 1, 8, 1),
])
def test_shtmg_fixed_cycles_matches_oracle(nf, ns, lmax, nb, ncell, cycles, nu1, nu2):
    import paper_1210_3069_gb300 as clc
    c = ctx()
    kappa = _kappa(nf, 21)
    P = _params(clc, ns, lmax, nb, ncell, fixed=cycles, nu1=nu1, nu2=nu2)
    sol = c.solution(nf, P)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, nu1=nu1, nu2=nu2, fixed_cycles=cycles)
    home, nv = _pixel_home(nf, nb)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        assert rel_l2(got[k], want[k]) < TOL, k
    cyc, res = sol.info()
    assert cyc == cycles
    assert abs(res - ref["residual"]) <= 1e-6 * ref["residual"] + 1e-14
    sol.close()


def test_shtmg_converges_like_oracle():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 32
    kappa = _kappa(nf, 22)
    P = _params(clc, ns, lmax, nb, ncell, tol=1e-10)
    sol = c.solution(nf, P)
    g = torch.Generator().manual_seed(3)
    zq, pq = synthetic.uniform_sphere(500, 4)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol)
    pts = c.lens_derivs(sol, zq.cuda(), pq.cuda())
    c.sync()
    cyc, res = sol.info()
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, tol=1e-10)
    assert res < 1e-10 and abs(cyc - ref["cycles"]) <= 1
    nv = geometry_vec(zq, pq)
    home = hp.ang2pix_nest(nb, zq, pq)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        # both solutions converged to 1e-10 relative residual: agreement is
        # bounded by the residual times the operator's conditioning, not 1e-10
        assert rel_l2(pts[k], want[k]) < 1e-7, k
    sol.close()


def geometry_vec(z, phi):
    s = torch.sqrt((1 - z) * (1 + z))
    return torch.stack([s * torch.cos(phi), s * torch.sin(phi), z], -1)


def test_shtmg_mixed_precision_converges_to_fp64_solution():
    """CLC_MIXED: FP32 V-cycles on the FP64 residual equation reach the same
    1e-10 relative residual and the same solution as the FP64 oracle."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 32
    kappa = _kappa(nf, 24)
    P = _params(clc, ns, lmax, nb, ncell, tol=1e-10, prec=clc.MIXED)
    sol = c.solution(nf, P)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    cyc, res = sol.info()
    assert res < 1e-10
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, tol=1e-12)
    home, nv = _pixel_home(nf, nb)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        assert rel_l2(got[k], want[k]) < 1e-7, k
    sol.close()


def test_shtmg_fp32_path():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 32
    kappa = _kappa(nf, 23)
    P = _params(clc, ns, lmax, nb, ncell, fixed=6, prec=clc.FP32)
    sol = c.solution(nf, P)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, fixed_cycles=6)
    home, nv = _pixel_home(nf, nb)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        assert rel_l2(got[k], want[k]) < 1e-4, k
    sol.close()


def _sht_lens_maps(kappa, nside, lmax):
    return sht.poisson_sht(kappa, nside, lmax)


def test_rays_sht_path_matches_oracle():
    """Three pure-SHT planes at Nside 16, rays from all pixel centres."""
    c = ctx()
    import paper_1210_3069_gb300 as clc
    nside, lmax = 16, 32
    chi = [100.0, 200.0, 300.0, 350.0]
    kap = [5e-2 * _kappa(nside, 30 + m, n=50_000) for m in range(3)]
    p = torch.arange(hp.npix(nside))
    z, phi = hp.pix2ang_ring(nside, p)
    rs = c.rays(p.numel())
    c.rays_init(rs, z.cuda(), phi.cuda(), chi[0])
    lenses = []
    for m in range(3):
        maps = c.poisson_sht(kap[m].cuda(), nside, lmax, psi=False)
        c.ray_step(rs, chi[m - 1] if m else 0.0, chi[m], chi[m + 1], maps=maps, nside_maps=nside)
        lenses.append(orays.map_lens(nside, _sht_lens_maps(kap[m], nside, lmax)))
    c.sync()
    n0 = hp.pix2vec_ring(nside, p)
    st = orays.trace(n0, chi, lenses)
    assert rel_l2(rs.x.T, st["x"]) < TOL
    assert rel_l2(rs.beta.T, st["beta"]) < TOL
    assert rel_l2(rs.A.T.reshape(-1, 2, 2), st["A"]) < TOL
    assert rel_l2(rs.Ap.T.reshape(-1, 2, 2), st["Ap"]) < TOL
    # the multi-plane entry point (clc_raytrace_planes) gives the same state
    rs2 = c.rays(p.numel())
    c.rays_init(rs2, z.cuda(), phi.cuda(), chi[0])
    c.raytrace_planes(clc.SOLVER_SHT, clc.mg_params(nside, lmax, 1), [k.cuda() for k in kap], nside, chi, rs2)
    c.sync()
    assert torch.allclose(rs2.A, rs.A, rtol=0, atol=1e-13)


@pytest.mark.parametrize("nside,nb", [(8, 1), (64, 4), (256, 16)])
def test_rays_at_pixel_centres(nside, nb):
    """Rays started at every RING pixel centre: positions chi0 n_p, unit
    directions, identity Jacobians, and the bundle = the pixel's NEST index at
    the bundle resolution (exact)."""
    c = ctx()
    chi0 = 123.0
    rs = c.rays(hp.npix(nside))
    c.rays_init_pixels(rs, nside, chi0, nb)
    c.sync()
    p = torch.arange(hp.npix(nside))
    nv = hp.pix2vec_ring(nside, p)
    # a few units in the last place: sincospi against the oracle's cos / sin
    assert float((rs.x.T.cpu() - chi0 * nv).abs().max()) <= 4e-15 * chi0
    assert float((rs.beta.T.cpu() - nv).abs().max()) <= 4e-15
    eye = torch.tensor([1.0, 0.0, 0.0, 1.0], dtype=torch.float64)
    assert torch.equal(rs.A.T.cpu(), eye.expand(p.numel(), 4)) and torch.equal(rs.Ap.T.cpu(), eye.expand(p.numel(), 4))
    shift = 2 * (hp.nside_order(nside) - hp.nside_order(nb))
    assert torch.equal(rs.bundle.cpu().long(), hp.ring2nest(nside, p) >> shift)


def test_rays_mg_path_matches_oracle():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 32
    chi = [150.0, 250.0, 400.0]
    kap = [5e-2 * _kappa(nf, 40 + m, n=100_000) for m in range(2)]
    g = torch.Generator().manual_seed(8)
    pix = torch.randint(0, hp.npix(nf), (3000,), generator=g)
    z, phi = hp.pix2ang_ring(nf, pix)
    rs = c.rays(pix.numel())
    c.rays_init(rs, z.cuda(), phi.cuda(), chi[0], nside_bundle=nb)
    P = _params(clc, ns, lmax, nb, ncell, fixed=3)
    sol = c.solution(nf, P)
    lenses = []
    home = hp.ang2pix_nest(nb, z, phi)
    for m in range(2):
        c.poisson_shtmg(kap[m].cuda(), nf, sol)
        c.ray_step(rs, chi[m - 1] if m else 0.0, chi[m], chi[m + 1], sol=sol)
        c.sync()
        ref = omg.solve_plane(kap[m], nf, ns, lmax, nb, ncell=ncell, fixed_cycles=3)
        lenses.append(lambda n, ref=ref: omg.fields_at(ref, nb, n, home))
    assert torch.equal(rs.bundle.cpu().long(), home)
    st = orays.trace(hp.pix2vec_ring(nf, pix), chi, lenses)
    assert rel_l2(rs.x.T, st["x"]) < TOL
    assert rel_l2(rs.A.T.reshape(-1, 2, 2), st["A"]) < TOL
    assert rel_l2(rs.Ap.T.reshape(-1, 2, 2), st["Ap"]) < TOL
    sol.close()


def test_invalid_mg_parameters():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    with pytest.raises(clc.CalclensError):
        c.solution(64, _params(clc, 16, 100, 4, 32))      # lmax > 4 nside_sht
    with pytest.raises(clc.CalclensError):
        c.solution(64, _params(clc, 16, 32, 4, 48))       # ncell not a power of two
    with pytest.raises(clc.CalclensError):
        c.solution(64, _params(clc, 16, 32, 4, 32, nu1=9))  # more sweeps than the block halo allows


@pytest.mark.parametrize("eps", [0.1, 0.01])
def test_tau_stopping_rule_matches_oracle(eps):
    """The paper's rule ||r|| < eps ||tau|| (Sec. 3.2) in FP64: the GPU stops
    after the same number of V-cycles as the oracle, with the same fields."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 32
    kappa = _kappa(nf, 25)
    P = clc.mg_params(ns, lmax, nb, ncell=ncell, stop_rule=clc.STOP_TAU, eps=eps, precision=clc.FP64)
    sol = c.solution(nf, P)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    cyc, ratio = sol.info()
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, stop="tau", eps=eps)
    assert cyc == ref["cycles"] and ratio < eps
    assert abs(ratio - ref["residual"]) <= 1e-8 * ref["residual"]
    home, nv = _pixel_home(nf, nb)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        assert rel_l2(got[k], want[k]) < TOL, k
    sol.close()


def test_tau_stopping_rule_mixed_precision():
    """CLC_MIXED with the tau rule checked after every V-cycle
    (refine_cycles = 1): the same cycle count as the FP64 oracle and its
    fields at that count to the mixed path's level."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 64
    kappa = _kappa(nf, 26)
    P = clc.mg_params(ns, lmax, nb, ncell=ncell, stop_rule=clc.STOP_TAU, eps=0.1, precision=clc.MIXED,
                      refine_cycles=1)
    sol = c.solution(nf, P)
    got = c.poisson_shtmg(kappa.cuda(), nf, sol, derivatives=True)
    c.sync()
    cyc, ratio = sol.info()
    ref = omg.solve_plane(kappa, nf, ns, lmax, nb, ncell=ncell, stop="tau", eps=0.1)
    assert cyc == ref["cycles"] and ratio < 0.1
    home, nv = _pixel_home(nf, nb)
    want = omg.fields_at(ref, nb, nv, home)
    for k in KEYS:
        assert rel_l2(got[k], want[k]) < 1e-7, k
    sol.close()
