"""GPU galaxy shears through pure-SHT planes and their adjoint (paper Sec. 2.2,
Sec. 3.2, Appendix B, Appendix D): the forward shears match the oracle
(<= 1e-10 relative), the adjoint gradient matches the oracle's autograd
gradient over every pixel and central finite differences of the GPU forward
(step 1e-6) to <= 1e-6 relative."""
import pytest
import torch

from oracle import healpix as hp, rays
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
F64 = torch.float64


def _case(seed, nside, lmax, nplanes, ngal, amp=0.02):
    g = torch.Generator().manual_seed(seed)
    kappas = torch.stack([amp * torch.randn(hp.npix(nside), dtype=F64, generator=g) for _ in range(nplanes)])
    chi = [100.0 + 100.0 * k for k in range(nplanes + 1)]
    gz, gphi = synthetic.uniform_sphere(ngal, seed + 1)
    gchi = 80.0 + (chi[-1] - 80.0) * torch.rand(ngal, dtype=F64, generator=g)
    return kappas, chi, gz, gphi, gchi


def _gpu(c, kappas, nside, lmax, chi, gz, gphi, gchi):
    import paper_1210_3069_gb300 as clc
    return clc.galaxy_shear(c, kappas, nside, lmax, chi, gz.cuda(), gphi.cuda(), gchi.cuda())


def test_forward_matches_oracle():
    c = ctx()
    nside, lmax = 16, 32
    kappas, chi, gz, gphi, gchi = _case(5, nside, lmax, 3, 300)
    got = _gpu(c, kappas.cuda(), nside, lmax, chi, gz, gphi, gchi)
    c.sync()
    want = rays.galaxy_shear(list(kappas), nside, lmax, chi, gz, gphi, gchi)
    assert rel_l2(got, want) < 1e-10
    # galaxies in front of the first plane see no lensing
    front = gchi < chi[0]
    assert front.any() and float(got.cpu()[:, front].abs().max()) == 0.0


def test_zero_convergence_gives_zero_shear_and_gradient_is_finite():
    c = ctx()
    nside, lmax = 16, 32
    kappas, chi, gz, gphi, gchi = _case(6, nside, lmax, 2, 100)
    k = torch.zeros_like(kappas).cuda().requires_grad_(True)
    g = _gpu(c, k, nside, lmax, chi, gz, gphi, gchi)
    assert float(g.detach().abs().max()) < 1e-14
    g.sum().backward()
    assert torch.isfinite(k.grad).all()


def test_adjoint_matches_oracle_gradient():
    c = ctx()
    nside, lmax = 16, 32
    kappas, chi, gz, gphi, gchi = _case(7, nside, lmax, 3, 400)
    target = 0.5 * rays.galaxy_shear(list(kappas), nside, lmax, chi, gz, gphi, gchi).detach()
    ko = [k.clone().requires_grad_(True) for k in kappas]
    lo = ((rays.galaxy_shear(ko, nside, lmax, chi, gz, gphi, gchi) - target) ** 2).sum()
    lo.backward()
    kg = kappas.clone().cuda().requires_grad_(True)
    lg = ((_gpu(c, kg, nside, lmax, chi, gz, gphi, gchi) - target.cuda()) ** 2).sum()
    lg.backward()
    c.sync()
    assert abs(float(lg.detach()) - float(lo.detach())) <= 1e-10 * abs(float(lo.detach()))
    for m in range(3):
        assert rel_l2(kg.grad[m], ko[m].grad) < 1e-10, m


@pytest.mark.parametrize("nside,lmax,nplanes,ngal", [(16, 32, 3, 400), (64, 128, 4, 20000)])
def test_adjoint_matches_finite_differences(nside, lmax, nplanes, ngal):
    c = ctx()
    kappas, chi, gz, gphi, gchi = _case(11, nside, lmax, nplanes, ngal)
    kappas = kappas.cuda()
    with torch.no_grad():
        target = 0.5 * _gpu(c, kappas, nside, lmax, chi, gz, gphi, gchi)

    def loss(k):
        return float(((_gpu(c, k, nside, lmax, chi, gz, gphi, gchi) - target) ** 2).sum())

    kg = kappas.clone().requires_grad_(True)
    L0 = ((_gpu(c, kg, nside, lmax, chi, gz, gphi, gchi) - target) ** 2).sum()
    L0.backward()
    grad = kg.grad
    h = 1e-6
    # rounding floor of the central difference itself: the loss (a sum of
    # 2 ngal squares, each from a long FP64 chain) carries ~1e-15 relative
    # error per term, accumulated over sqrt(2 ngal) terms, divided by 2h
    fd_floor = 1e-15 * float(L0) * (2 * ngal) ** 0.5 / (2 * h)
    gen = torch.Generator().manual_seed(3)
    for m in range(nplanes):
        gmax = float(grad[m].abs().max())
        pix = torch.cat([grad[m].abs().topk(2).indices.cpu(), torch.randint(0, hp.npix(nside), (2,), generator=gen)])
        for p in pix.tolist():
            kp = kappas.clone()
            km = kappas.clone()
            kp[m, p] += h
            km[m, p] -= h
            fd = (loss(kp) - loss(km)) / (2 * h)
            ad = float(grad[m, p])
            assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-8 * gmax + fd_floor, (m, p, fd, ad, fd_floor)


def test_mixed_precision_forward_and_gradient_are_close():
    """The same chain with the tensor-core SHT: shears and gradient within
    the mixed path's error of the FP64 ones."""
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside, lmax = 64, 128
    kappas, chi, gz, gphi, gchi = _case(13, nside, lmax, 2, 5000)
    k64 = kappas.clone().cuda().requires_grad_(True)
    kmx = kappas.clone().cuda().requires_grad_(True)
    g64 = clc.galaxy_shear(c, k64, nside, lmax, chi, gz.cuda(), gphi.cuda(), gchi.cuda(), precision=clc.FP64)
    gmx = clc.galaxy_shear(c, kmx, nside, lmax, chi, gz.cuda(), gphi.cuda(), gchi.cuda(), precision=clc.MIXED)
    assert rel_l2(gmx, g64) < 1e-5
    (g64 ** 2).sum().backward()
    (gmx ** 2).sum().backward()
    assert rel_l2(kmx.grad, k64.grad) < 1e-4
