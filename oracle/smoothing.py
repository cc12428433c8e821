"""Adaptive Epanechnikov smoothing of particles onto a HEALPix map (oracle;
test infrastructure).

Sec. 3.2 of the paper smooths the mass of every N-body particle with the
Epanechnikov kernel normalised on the sphere, K(theta; sigma) =
[1 - (theta / sigma)^2] / N(sigma), N(sigma) = 2 pi (sinc^2(sigma / 2 pi)
- 2 sinc(sigma / pi) + 1), sinc(x) = sin(pi x) / (pi x), with a smoothing
length sigma per particle (the larger of a few softening lengths and a few
ray spacings), bins the kernel over the HEALPix map and enforces exact mass
conservation.

Reading taken here: a particle's mass goes to the pixels whose centres lie at
angular distance theta < sigma, in proportion to K at the pixel centre, the
weights divided by their sum so that the particle's whole mass is deposited
(on a grid of equal-area pixels this is the binned kernel made exactly
mass-conserving; N(sigma) cancels).  A particle with no pixel centre inside
its kernel (sigma below the pixel scale) deposits its mass on the pixel that
contains it.

Plain definition, no blocking: every particle is compared with every pixel
centre, the angular distance being atan2(|n_p x n_q|, n_p . n_q).
"""
import math

import torch

from . import healpix as hp

F64 = torch.float64


def sinc(x):
    """sin(pi x) / (pi x), 1 at x = 0."""
    return 1.0 if x == 0 else math.sin(math.pi * x) / (math.pi * x)


def kernel_norm(sigma):
    """N(sigma) of the Epanechnikov kernel on the sphere (Sec. 3.2)."""
    return 2.0 * math.pi * (sinc(sigma / (2.0 * math.pi)) ** 2 - 2.0 * sinc(sigma / math.pi) + 1.0)


def kernel(theta, sigma):
    """K(theta; sigma), zero for theta >= sigma (Sec. 3.2)."""
    t = torch.as_tensor(theta, dtype=F64)
    return torch.where(t < sigma, (1.0 - (t / sigma) ** 2) / kernel_norm(sigma), torch.zeros_like(t))


def angular_distance(a, b):
    """Angle between unit vectors a [..., 3] and b [..., 3]."""
    cr = torch.linalg.cross(a, b, dim=-1)
    return torch.atan2(torch.linalg.vector_norm(cr, dim=-1), (a * b).sum(-1))


def smooth_particles(nside, z, phi, sigma, mass=1.0):
    """FP64 RING map of the deposited mass of particles at (z, phi) with
    smoothing length sigma (a number, or one per particle), each particle
    of mass `mass`."""
    z = torch.as_tensor(z, dtype=F64)
    phi = torch.as_tensor(phi, dtype=F64)
    n = z.numel()
    sig = torch.as_tensor(sigma, dtype=F64).expand(n)
    nv = hp.vec_from_zphi(z, phi)                              # [n, 3]
    centres = hp.pix2vec_ring(nside, torch.arange(hp.npix(nside)))  # [npix, 3]
    own = hp.ang2pix_ring(nside, z, phi)
    out = torch.zeros(hp.npix(nside), dtype=F64)
    for k in range(n):
        th = angular_distance(nv[k].expand_as(centres), centres)
        s = float(sig[k])
        w = kernel(th, s)
        tot = float(w.sum())
        if tot > 0.0:
            out += mass * (w / tot)
        else:
            out[own[k]] += mass
    return out


def kappa_from_density(rho, nbar, scale):
    """Plane source kappa_p = scale * (rho_p / nbar - 1) (Eq. lenspoisson) for
    a smoothed particle-number map rho, each operation rounded separately."""
    return scale * (torch.as_tensor(rho, dtype=F64) / nbar - 1.0)
