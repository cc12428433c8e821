"""The oracle's galaxy-shear chain (pure-SHT planes, ray recursion, Appendix D
interpolation) and its autograd gradient, pinned by central finite
differences of the oracle itself: a gradient that dropped a term (the
position dependence of the lens lookup, the transport, the SHT adjoint)
would miss the finite difference by far more than the tolerance."""
import torch

from oracle import healpix as hp, rays
from workloads import synthetic

F64 = torch.float64


def _case(seed=3, nside=8, lmax=16, nplanes=3, ngal=40):
    g = torch.Generator().manual_seed(seed)
    kappas = [0.02 * torch.randn(hp.npix(nside), dtype=F64, generator=g) for _ in range(nplanes)]
    chi = [100.0 + 100.0 * k for k in range(nplanes + 1)]
    gz, gphi = synthetic.uniform_sphere(ngal, seed + 1)
    gchi = 80.0 + (chi[-1] - 80.0) * torch.rand(ngal, dtype=F64, generator=g)
    return kappas, nside, lmax, chi, gz, gphi, gchi


def test_galaxy_bins_and_interpolation_limits():
    chi = [100.0, 200.0, 300.0]
    b = rays.galaxy_bins(chi, torch.tensor([50.0, 100.0, 150.0, 200.0, 299.0, 300.0], dtype=F64))
    assert b.tolist() == [-1, 0, 0, 1, 1, 1]
    # at chi_g = chi_n the galaxy takes A_n, at chi_{n+1} it takes A_{n+1}
    A0, A1 = torch.eye(2, dtype=F64)[None] * 2.0, torch.eye(2, dtype=F64)[None] * 3.0
    assert torch.allclose(rays.galaxy_interp(A0, A1, torch.tensor([1.0]), torch.tensor([2.0]), torch.tensor([1.0])), A0)
    assert torch.allclose(rays.galaxy_interp(A0, A1, torch.tensor([1.0]), torch.tensor([2.0]), torch.tensor([2.0])), A1)


def test_no_lensing_gives_zero_shear():
    kappas, nside, lmax, chi, gz, gphi, gchi = _case()
    zero = [torch.zeros_like(k) for k in kappas]
    g = rays.galaxy_shear(zero, nside, lmax, chi, gz, gphi, gchi)
    assert float(g.abs().max()) < 1e-14


def test_oracle_gradient_matches_finite_differences():
    kappas, nside, lmax, chi, gz, gphi, gchi = _case()
    target = 0.5 * rays.galaxy_shear(kappas, nside, lmax, chi, gz, gphi, gchi).detach()
    ks = [k.clone().requires_grad_(True) for k in kappas]

    def loss(kk):
        g = rays.galaxy_shear(kk, nside, lmax, chi, gz, gphi, gchi)
        return ((g - target) ** 2).sum()

    L = loss(ks)
    L.backward()
    h = 1e-6
    gen = torch.Generator().manual_seed(9)
    for m in range(len(kappas)):
        gmax = float(ks[m].grad.abs().max())
        pix = torch.cat([ks[m].grad.abs().topk(2).indices, torch.randint(0, hp.npix(nside), (2,), generator=gen)])
        for p in pix.tolist():
            kp = [k.detach().clone() for k in kappas]
            km = [k.detach().clone() for k in kappas]
            kp[m][p] += h
            km[m][p] -= h
            with torch.no_grad():
                fd = (loss(kp) - loss(km)) / (2 * h)
            ad = ks[m].grad[p]
            # the finite difference itself carries ~1e-14 relative rounding of the loss over 2h
            assert abs(float(fd - ad)) <= 1e-6 * abs(float(ad)) + 1e-8 * gmax, (m, p, float(fd), float(ad))


def _case_mg(seed=5, nf=16, ns=8, lmax=16, nb=2, ncell=16, nplanes=2, ngal=30):
    from oracle import binning
    kappas = []
    for m in range(nplanes):
        z, phi = synthetic.lognormal_particles(60_000, seed + m)
        c = binning.bin_counts(nf, z, phi)
        kappas.append(0.02 * binning.kappa_from_counts(c, z.numel() / hp.npix(nf), 1.0))
    g = torch.Generator().manual_seed(seed)
    chi = [100.0 + 100.0 * k for k in range(nplanes + 1)]
    gz, gphi = synthetic.uniform_sphere(ngal, seed + 11)
    gchi = 120.0 + (chi[-1] - 120.0) * torch.rand(ngal, dtype=F64, generator=g)
    return kappas, nf, ns, lmax, nb, ncell, chi, gz, gphi, gchi


def test_oracle_mg_gradient_matches_finite_differences():
    """The same pin for the SHT+MG chain: autograd through the patch set-up
    (interpolation of the SHT potential and of kappa), the V-cycles, the
    finite-difference lookup and the degrade to the SHT grid."""
    kappas, nf, ns, lmax, nb, ncell, chi, gz, gphi, gchi = _case_mg()
    args = (nf, ns, lmax, nb, ncell, chi, gz, gphi, gchi)
    target = 0.5 * rays.galaxy_shear_mg(kappas, *args).detach()
    ks = [k.clone().requires_grad_(True) for k in kappas]

    def loss(kk):
        g = rays.galaxy_shear_mg(kk, *args)
        return ((g - target) ** 2).sum()

    L = loss(ks)
    L.backward()
    h = 1e-6
    for m in range(len(kappas)):
        gmax = float(ks[m].grad.abs().max())
        assert gmax > 0
        for p in ks[m].grad.abs().topk(3).indices.tolist():
            kp = [k.detach().clone() for k in kappas]
            km = [k.detach().clone() for k in kappas]
            kp[m][p] += h
            km[m][p] -= h
            with torch.no_grad():
                fd = (loss(kp) - loss(km)) / (2 * h)
            ad = ks[m].grad[p]
            assert abs(float(fd - ad)) <= 1e-6 * abs(float(ad)) + 1e-8 * gmax, (m, p, float(fd), float(ad))
