"""GPU galaxy shears through SHT+MG planes and the SHT+MG adjoint (paper
Sec. 3.2, Sec. 2.2, Appendix B, D): forward shears against the oracle's
SHT+MG chain, the adjoint gradient (adjoint patch solve L^T lambda = ubar,
transposed interpolations, SHT Poisson adjoint, transposed degrade) against
the oracle's autograd gradient over every pixel and against central finite
differences of the GPU forward."""
import pytest
import torch

from oracle import binning, healpix as hp, rays
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
F64 = torch.float64
CYC = 20   # fixed V-cycles: the forward converged to rounding on both sides


def _case(seed, nf, nplanes, ngal, amp=0.02):
    kappas = []
    for m in range(nplanes):
        z, phi = synthetic.lognormal_particles(20 * hp.npix(nf), seed + m)
        c = binning.bin_counts(nf, z, phi)
        kappas.append(amp * binning.kappa_from_counts(c, z.numel() / hp.npix(nf), 1.0))
    g = torch.Generator().manual_seed(seed)
    chi = [100.0 + 100.0 * k for k in range(nplanes + 1)]
    gz, gphi = synthetic.uniform_sphere(ngal, seed + 11)
    gchi = 80.0 + (chi[-1] - 80.0) * torch.rand(ngal, dtype=F64, generator=g)
    return torch.stack(kappas), chi, gz, gphi, gchi


def _params(clc, ns, lmax, nb, ncell):
    return clc.mg_params(ns, lmax, nb, ncell=ncell, nu1=2, nu2=2, fixed_cycles=CYC, precision=clc.FP64)


def _gpu(c, clc, kappas, nf, P, chi, gz, gphi, gchi):
    return clc.galaxy_shear(c, kappas, nf, P, chi, gz.cuda(), gphi.cuda(), gchi.cuda())


GEOM = [(32, 8, 16, 2, 32), (64, 16, 32, 4, 64)]


@pytest.mark.parametrize("nf,ns,lmax,nb,ncell", GEOM)
def test_mg_forward_matches_oracle(nf, ns, lmax, nb, ncell):
    import paper_1210_3069_gb300 as clc
    c = ctx()
    kappas, chi, gz, gphi, gchi = _case(5, nf, 3, 400)
    P = _params(clc, ns, lmax, nb, ncell)
    got = _gpu(c, clc, kappas.cuda(), nf, P, chi, gz, gphi, gchi)
    c.sync()
    want = rays.galaxy_shear_mg(list(kappas), nf, ns, lmax, nb, ncell, chi, gz, gphi, gchi, cycles=CYC)
    assert rel_l2(got, want) < 1e-10


@pytest.mark.parametrize("nf,ns,lmax,nb,ncell", GEOM)
def test_mg_adjoint_matches_oracle_gradient(nf, ns, lmax, nb, ncell):
    import paper_1210_3069_gb300 as clc
    c = ctx()
    kappas, chi, gz, gphi, gchi = _case(7, nf, 2, 300)
    P = _params(clc, ns, lmax, nb, ncell)
    args = (nf, ns, lmax, nb, ncell, chi, gz, gphi, gchi)
    target = 0.5 * rays.galaxy_shear_mg(list(kappas), *args, cycles=CYC).detach()
    ko = [k.clone().requires_grad_(True) for k in kappas]
    lo = ((rays.galaxy_shear_mg(ko, *args, cycles=CYC) - target) ** 2).sum()
    lo.backward()
    kg = kappas.clone().cuda().requires_grad_(True)
    lg = ((_gpu(c, clc, kg, nf, P, chi, gz, gphi, gchi) - target.cuda()) ** 2).sum()
    lg.backward()
    c.sync()
    assert abs(float(lg.detach()) - float(lo.detach())) <= 1e-10 * abs(float(lo.detach()))
    errs = [rel_l2(kg.grad[m], ko[m].grad) for m in range(kappas.shape[0])]
    print("mg gradient vs oracle", errs)
    for e in errs:
        # the oracle differentiates its 20 V-cycles, the GPU solves the
        # adjoint patch problem to 1e-12: both are the converged solve's
        # gradient up to the iteration's residual (measured 1.2e-11 on GB300)
        assert e < 1e-10, errs


def test_mg_adjoint_matches_finite_differences():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nf, ns, lmax, nb, ncell = 64, 16, 32, 4, 64
    kappas, chi, gz, gphi, gchi = _case(11, nf, 3, 3000)
    P = _params(clc, ns, lmax, nb, ncell)
    kappas = kappas.cuda()
    with torch.no_grad():
        target = 0.5 * _gpu(c, clc, kappas, nf, P, chi, gz, gphi, gchi)

    def loss(k):
        return float(((_gpu(c, clc, k, nf, P, chi, gz, gphi, gchi) - target) ** 2).sum())

    kg = kappas.clone().requires_grad_(True)
    L0 = ((_gpu(c, clc, kg, nf, P, chi, gz, gphi, gchi) - target) ** 2).sum()
    L0.backward()
    grad = kg.grad
    h = 1e-6
    fd_floor = 1e-15 * float(L0.detach()) * (2 * gz.numel()) ** 0.5 / (2 * h)
    gen = torch.Generator().manual_seed(3)
    for m in range(kappas.shape[0]):
        gmax = float(grad[m].abs().max())
        pix = torch.cat([grad[m].abs().topk(2).indices.cpu(), torch.randint(0, hp.npix(nf), (2,), generator=gen)])
        for p in pix.tolist():
            kp = kappas.clone()
            km = kappas.clone()
            kp[m, p] += h
            km[m, p] -= h
            fd = (loss(kp) - loss(km)) / (2 * h)
            ad = float(grad[m, p])
            assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-8 * gmax + fd_floor, (m, p, fd, ad, fd_floor)


def test_mg_trace_rejects_non_fp64_parameters():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    kappas, chi, gz, gphi, gchi = _case(12, 32, 1, 10)
    P = clc.mg_params(8, 16, 2, ncell=32, precision=clc.MIXED)
    with pytest.raises(clc.CalclensError):
        c.gal_trace_mg(kappas.cuda(), 32, P, chi, gz.cuda(), gphi.cuda(), gchi.cuda())
