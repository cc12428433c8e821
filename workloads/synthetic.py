"""Seeded particle, density-field and galaxy generators (torch, any device).

All positions are returned as (z = cos theta, phi) in float64 with phi in
[0, 2 pi).  Random numbers come from a torch.Generator seeded explicitly, so
a (seed, device) pair always yields the same arrays.
"""
import math

import torch

F64 = torch.float64


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _wrap_phi(phi):
    phi = torch.remainder(phi, 2 * math.pi)
    return torch.where(phi >= 2 * math.pi, phi - 2 * math.pi, phi)


def uniform_sphere(n, seed, device="cpu"):
    """n points uniform on the unit sphere."""
    g = _gen(seed, device)
    u = torch.rand(n, generator=g, dtype=F64, device=device)
    v = torch.rand(n, generator=g, dtype=F64, device=device)
    return 2.0 * u - 1.0, 2.0 * math.pi * v


def gaussian_clumps(nclumps, per_clump, sigma_rad, seed, device="cpu"):
    """nclumps centres uniform on the sphere; around each, per_clump points
    with 2D Gaussian tangent-plane offsets (std sigma_rad per axis) mapped to
    the sphere along geodesics (exponential map)."""
    g = _gen(seed, device)
    zc = 2.0 * torch.rand(nclumps, generator=g, dtype=F64, device=device) - 1.0
    pc = 2.0 * math.pi * torch.rand(nclumps, generator=g, dtype=F64, device=device)
    dx = sigma_rad * torch.randn(nclumps, per_clump, generator=g, dtype=F64, device=device)
    dy = sigma_rad * torch.randn(nclumps, per_clump, generator=g, dtype=F64, device=device)
    sc = torch.sqrt((1 - zc) * (1 + zc))
    c = torch.stack([sc * torch.cos(pc), sc * torch.sin(pc), zc], -1)[:, None, :]
    t = torch.stack([zc * torch.cos(pc), zc * torch.sin(pc), -sc], -1)[:, None, :]
    p = torch.stack([-torch.sin(pc), torch.cos(pc), torch.zeros_like(pc)], -1)[:, None, :]
    r = torch.sqrt(dx * dx + dy * dy)
    dirn = (dx[..., None] * t + dy[..., None] * p) / torch.where(r > 0, r, 1.0)[..., None]
    v = torch.cos(r)[..., None] * c + torch.sin(r)[..., None] * dirn
    v = v.reshape(-1, 3)
    v = v / torch.linalg.vector_norm(v, dim=-1, keepdim=True)
    z = v[:, 2].clamp(-1.0, 1.0)
    phi = _wrap_phi(torch.atan2(v[:, 1], v[:, 0]))
    return z, phi


def point_clump_config(seed=1210001, device="cpu", n_uniform=200_000, nclumps=50,
                       per_clump=2000, sigma_deg=1.0):
    """Uniform background plus Gaussian clumps (the single-plane SHT case)."""
    zu, pu = uniform_sphere(n_uniform, seed, device)
    zc, pc = gaussian_clumps(nclumps, per_clump, math.radians(sigma_deg), seed + 7919, device)
    return torch.cat([zu, zc]), torch.cat([pu, pc])


def random_field_modes(nmodes, kmin, kmax, seed, device="cpu"):
    """Wave vectors (log-uniform |k|, isotropic directions) and phases of a
    sum-of-plane-waves Gaussian field; equal variance per octave of |k|
    gives an angular power close to C_l ~ l^-2."""
    g = _gen(seed, device)
    lk = math.log(kmin) + (math.log(kmax) - math.log(kmin)) * torch.rand(nmodes, generator=g, dtype=F64, device=device)
    kz = 2 * torch.rand(nmodes, generator=g, dtype=F64, device=device) - 1
    kp = 2 * math.pi * torch.rand(nmodes, generator=g, dtype=F64, device=device)
    ks = torch.sqrt((1 - kz) * (1 + kz))
    k = torch.exp(lk)[:, None] * torch.stack([ks * torch.cos(kp), ks * torch.sin(kp), kz], -1)
    ph = 2 * math.pi * torch.rand(nmodes, generator=g, dtype=F64, device=device)
    return k, ph


def lognormal_density(z, phi, modes, sigma2=math.log(2.0), chunk=1 << 20):
    """1 + delta = exp(g - sigma^2 / 2) with g = sqrt(2 sigma^2 / M) sum cos(k.n + ph)
    (unit-variance lognormal for sigma^2 = ln 2), evaluated in float32."""
    k, ph = modes
    k32, ph32 = k.float(), ph.float()
    amp = math.sqrt(2.0 * sigma2 / k.shape[0])
    out = torch.empty(z.shape, dtype=torch.float32, device=z.device)
    for s in range(0, z.numel(), chunk):
        zz = z[s:s + chunk]
        pp = phi[s:s + chunk]
        sn = torch.sqrt((1 - zz) * (1 + zz))
        n = torch.stack([sn * torch.cos(pp), sn * torch.sin(pp), zz], -1).float()
        arg = n @ k32.T + ph32
        gf = amp * torch.cos(arg).sum(-1)
        out[s:s + chunk] = torch.exp(gf - 0.5 * sigma2)
    return out


def lognormal_particles(n_mean, seed, device="cpu", nz=None, nphi=None, nmodes=256,
                        kmin=2.0, kmax=4096.0, growth=1.0):
    """Poisson-sampled particles of a lognormal density field on an
    equal-area (z, phi) grid of nz x nphi cells: each cell draws a Poisson
    count with mean n_mean (1 + growth * delta) / ncell and places its
    particles uniformly inside the cell."""
    if nz is None:
        ncell = max(64, int(n_mean))
        nz = max(4, int(math.sqrt(ncell / 3.0)))
        nphi = 3 * nz
    modes = random_field_modes(nmodes, kmin, kmax, seed, device)
    g = _gen(seed + 1, device)
    zc = -1.0 + (torch.arange(nz, dtype=F64, device=device) + 0.5) * (2.0 / nz)
    pc = (torch.arange(nphi, dtype=F64, device=device) + 0.5) * (2 * math.pi / nphi)
    Z = zc[:, None].expand(nz, nphi).reshape(-1)
    P = pc[None, :].expand(nz, nphi).reshape(-1)
    rho = lognormal_density(Z, P, modes)
    rho = (1.0 + growth * (rho.double() - 1.0)).clamp(min=0.0)
    lam = rho * (n_mean / rho.numel())
    counts = torch.poisson(lam, generator=g).long()
    cell = torch.repeat_interleave(torch.arange(rho.numel(), device=device), counts)
    iz = cell // nphi
    ip = cell % nphi
    u = torch.rand(cell.numel(), generator=g, dtype=F64, device=device)
    v = torch.rand(cell.numel(), generator=g, dtype=F64, device=device)
    z = -1.0 + (iz.double() + u) * (2.0 / nz)
    phi = (ip.double() + v) * (2 * math.pi / nphi)
    return z.clamp(-1.0, 1.0), _wrap_phi(phi)


def galaxies(n, z_lo, z_hi, seed, device="cpu"):
    """n galaxies uniform on the sphere with redshift uniform in [z_lo, z_hi]."""
    zz, pp = uniform_sphere(n, seed, device)
    g = _gen(seed + 3, device)
    red = z_lo + (z_hi - z_lo) * torch.rand(n, generator=g, dtype=F64, device=device)
    return zz, pp, red


def cored_lens_map(n, centre, b, s):
    """Source-sphere directions of rays seen at unit vectors n [..., 3] through
    an axisymmetric lens at unit vector `centre`: a ray at angle theta from the
    centre is moved along its great circle to theta - alpha(theta), with the
    cored isothermal deflection alpha = b (sqrt(theta^2 + s^2) - s) / theta
    tapered by ((1 + cos theta) / 2)^2 so that the map stays smooth at the
    antipode (one image for b / (2 s) < 1, three near the centre above).
    Also returns alpha(theta) as a function for root finding."""
    def alpha(th):
        th = torch.as_tensor(th, dtype=F64)
        a = b * (torch.sqrt(th * th + s * s) - s) / torch.where(th == 0, torch.ones_like(th), th)
        a = torch.where(th == 0, torch.zeros_like(th), a)
        return a * ((1.0 + torch.cos(th)) / 2.0) ** 2

    c = torch.as_tensor(centre, dtype=F64, device=n.device)
    ct = (n @ c).clamp(-1.0, 1.0)
    th = torch.arccos(ct)
    e = n - ct[..., None] * c
    en = torch.linalg.vector_norm(e, dim=-1, keepdim=True)
    e = e / torch.where(en > 0, en, torch.ones_like(en))
    beta = th - alpha(th)
    return torch.cos(beta)[..., None] * c + torch.sin(beta)[..., None] * e, alpha


def random_jacobians(n, amp, seed, device="cpu"):
    """[n, 2, 2] matrices I + amp * (standard normal entries)."""
    g = _gen(seed, device)
    return torch.eye(2, dtype=F64, device=device) + amp * torch.randn(n, 2, 2, generator=g, dtype=F64, device=device)
