"""GPU Epanechnikov smoothing (paper Sec. 3.2) against the oracle: the
smoothed particle-number map element by element (FP64 atomics: rounding
only), exact mass conservation, the tiny-kernel limit equal to binning, and
per-particle smoothing lengths; at Nside 2048 mass conservation and the
support of a single kernel."""
import math

import pytest
import torch

from oracle import binning, healpix as hp, smoothing as sm
from tests.gpu_util import ctx, rel_l2
from workloads import synthetic

pytestmark = pytest.mark.gpu
F64 = torch.float64


def _particles(n, seed, extra=True):
    z, phi = synthetic.uniform_sphere(n, seed)
    if extra:   # both poles, longitude 0 and just below 2 pi, the polar-cap / belt boundary
        z = torch.cat([z, torch.tensor([1.0, -1.0, 0.3, 2.0 / 3.0, -2.0 / 3.0], dtype=F64)])
        phi = torch.cat([phi, torch.tensor([0.7, 5.1, 0.0, 2 * math.pi - 1e-12, 1.0], dtype=F64)])
    return z, phi


@pytest.mark.parametrize("nside,n,sig_pix", [(16, 300, 6.0), (64, 400, 2.5), (64, 300, 0.3), (128, 200, 1.2)])
def test_smoothing_matches_oracle(nside, n, sig_pix):
    c = ctx()
    sigma = sig_pix * math.sqrt(4 * math.pi / hp.npix(nside))
    z, phi = _particles(n, 61 + nside)
    got = c.smooth_particles(z.cuda(), phi.cuda(), nside, sigma)
    c.sync()
    want = sm.smooth_particles(nside, z, phi, sigma)
    assert rel_l2(got, want) < 1e-12
    assert float((got.cpu() - want).abs().max()) < 1e-12
    assert abs(float(got.sum()) - z.numel()) < 1e-9


def test_per_particle_smoothing_lengths():
    c = ctx()
    nside = 32
    z, phi = _particles(250, 7)
    g = torch.Generator().manual_seed(8)
    sig = 0.02 + 0.2 * torch.rand(z.numel(), generator=g, dtype=F64)
    got = c.smooth_particles(z.cuda(), phi.cuda(), nside, sigma_each=sig.cuda())
    c.sync()
    want = torch.zeros(hp.npix(nside), dtype=F64)
    for k in range(z.numel()):
        want += sm.smooth_particles(nside, z[k:k + 1], phi[k:k + 1], float(sig[k]))
    assert rel_l2(got, want) < 1e-12


def test_tiny_kernel_is_binning_and_kappa():
    c = ctx()
    nside = 64
    z, phi = _particles(5000, 9, extra=False)
    rho = c.smooth_particles(z.cuda(), phi.cuda(), nside, 1e-9)
    c.sync()
    counts = binning.bin_counts(nside, z, phi)
    assert torch.equal(rho.cpu(), counts.to(F64))
    nbar = z.numel() / hp.npix(nside)
    k = c.density_to_kappa(rho, nside, nbar, 0.7)
    c.sync()
    assert torch.equal(k.cpu(), sm.kappa_from_density(counts.to(F64), nbar, 0.7))


def test_full_size_mass_and_support():
    """Nside 2048: 1e6 particles keep their mass; one particle's deposit lies
    within sigma and has the kernel's shape (checked on the pixels it touched)."""
    c = ctx()
    nside = 2048
    sigma = 2.5 * math.sqrt(4 * math.pi / hp.npix(nside))
    z, phi = synthetic.uniform_sphere(1_000_000, 12, device="cuda")
    rho = c.smooth_particles(z, phi, nside, sigma)
    c.sync()
    assert abs(float(rho.sum()) - 1e6) < 1e-6
    z1, p1 = torch.tensor([0.123456], dtype=F64), torch.tensor([2.5], dtype=F64)
    one = c.smooth_particles(z1.cuda(), p1.cuda(), nside, sigma)
    c.sync()
    idx = one.nonzero().flatten().cpu()
    assert 10 < idx.numel() < 40 and abs(float(one.sum()) - 1.0) < 1e-14
    zq, phq = hp.pix2ang_ring(nside, idx)
    th = sm.angular_distance(hp.vec_from_zphi(zq, phq), hp.vec_from_zphi(z1, p1).expand(idx.numel(), 3))
    assert float(th.max()) < sigma
    w = 1.0 - (th / sigma) ** 2
    assert rel_l2(one.cpu()[idx], w / w.sum()) < 1e-12


def test_bad_arguments():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    z = torch.zeros(4, dtype=F64, device="cuda")
    with pytest.raises(clc.CalclensError):
        c.smooth_particles(z, z, 16, 0.0)
    with pytest.raises(clc.CalclensError):
        c.smooth_particles(z, z, 16, 0.7)
    with pytest.raises(clc.CalclensError):
        c.smooth_particles(z, z, 12, 0.1)
