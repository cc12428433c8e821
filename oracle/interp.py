"""HEALPix ring-bilinear interpolation (oracle; test infrastructure).

Sec. 3.2 interpolates the SHT potential onto the multigrid patches with the
linear interpolation of the public HEALPix package, and Sec. 3.3 uses the
same four-pixel interpolation to carry ray quantities to galaxy images.
Reading used here (the paper gives no formula): between the two rings that
bracket the point's colatitude theta the value is linear in theta; on each
ring it is linear in phi between the two pixels that bracket phi.  Above the
first ring (below the last) ring 1 (ring 4 Nside - 1) is blended, linearly in
theta, with a pole value equal to the mean of that ring's four pixels.  The
result is continuous in position everywhere.
"""
import math

import torch

from . import healpix as hp

F64 = torch.float64
I64 = torch.int64


def ring_theta(nside):
    rt = hp.ring_table(nside)
    return torch.atan2(rt["sin_theta"], rt["z"])


def _ring_pixels(rt, r, phi):
    """Two pixels of ring index r (0-based) bracketing phi and their weights."""
    n = rt["npix"][r]
    t = (phi - rt["phi0"][r]) * n.to(F64) / (2.0 * math.pi)
    j0 = torch.floor(t)
    f = t - j0
    j0 = j0.to(I64)
    p0 = rt["first"][r] + torch.remainder(j0, n)
    p1 = rt["first"][r] + torch.remainder(j0 + 1, n)
    return p0, p1, 1.0 - f, f


def interp_weights(nside, theta, phi):
    """Pixel indices [..., 8] and weights [..., 8] (sum 1) of the
    ring-bilinear interpolation at (theta, phi); unused slots have weight 0."""
    rt = hp.ring_table(nside)
    th_r = ring_theta(nside)
    nr = th_r.numel()
    theta = torch.as_tensor(theta, dtype=F64).contiguous()
    phi = torch.as_tensor(phi, dtype=F64)
    # ring index r1 (0-based) with th_r[r1] <= theta < th_r[r1 + 1]; -1 above the first ring
    r1 = torch.searchsorted(th_r, theta, right=True) - 1
    north = r1 < 0
    south = r1 >= nr - 1
    ra = r1.clamp(0, nr - 1)
    rb = (r1 + 1).clamp(0, nr - 1)
    ta = th_r[ra]
    tb = th_r[rb]
    w = torch.where(north, theta / th_r[0],
                    torch.where(south, (math.pi - theta) / (math.pi - th_r[-1]),
                                (theta - ta) / torch.where(tb > ta, tb - ta, 1.0)))
    pa0, pa1, wa0, wa1 = _ring_pixels(rt, ra, phi)
    pb0, pb1, wb0, wb1 = _ring_pixels(rt, rb, phi)
    # interior: (1 - w) ring a + w ring b.  North: w ring 1 + (1 - w) pole.
    # South: w ring last + (1 - w) pole.
    wring_a = torch.where(north, w, torch.where(south, w, 1.0 - w))
    wring_b = torch.where(north | south, torch.zeros_like(w), w)
    pole_w = torch.where(north | south, (1.0 - w) * 0.25, torch.zeros_like(w))
    pole_first = torch.where(north, rt["first"][0], rt["first"][nr - 1])
    idx = torch.stack([pa0, pa1, pb0, pb1] + [pole_first + k for k in range(4)], -1)
    wts = torch.stack([wring_a * wa0, wring_a * wa1, wring_b * wb0, wring_b * wb1] + [pole_w] * 4, -1)
    return idx, wts


def interpolate(nside, maps, theta, phi):
    """Interpolate map(s) [..., Npix] (last axis pixels) at (theta, phi)."""
    idx, wts = interp_weights(nside, theta, phi)
    return (maps[..., idx] * wts).sum(-1)
