"""HEALPix geometry in plain FP64 / int64 torch ops (oracle; test infrastructure).

The paper places rays on HEALPix cell centres, groups them into NEST-ordered
bundle cells by bit shifts and runs its SHT over HEALPix rings (Sec. 3,
Sec. 3.1, footnote of Sec. 4.1: pixel area 4 pi / (12 Nside^2)).  The
pixelisation itself is the one published by Gorski et al. (2005, ApJ 622,
759, Sec. 4-5); every formula below restates that publication.

Bit-exactness contract: ``ang2pix_ring`` and ``ang2pix_nest`` use only
IEEE-correctly-rounded +, -, *, sqrt and truncation, each rounded separately,
in the order written here.  Inputs are (z = cos theta, phi) in FP64, with
phi in [0, 2 pi]; tt = phi * (2/pi) is wrapped once into [0, 4).
"""
import math

import torch

F64 = torch.float64
I64 = torch.int64

TWO_OVER_PI = 2.0 / math.pi      # the double nearest 2/pi
TWO_THIRDS = 2.0 / 3.0           # the double nearest 2/3


def npix(nside):
    """Number of pixels, 12 Nside^2 (Gorski et al. 2005, Sec. 4)."""
    return 12 * nside * nside


def nside_order(nside):
    order = int(nside).bit_length() - 1
    if nside < 1 or (1 << order) != nside:
        raise ValueError("nside must be a power of two")
    return order


def _isqrt(x):
    """Exact integer square root of an int64 tensor (floor)."""
    r = torch.floor(torch.sqrt(x.to(F64))).to(I64)
    r = torch.where(r * r > x, r - 1, r)
    r = torch.where((r + 1) * (r + 1) <= x, r + 1, r)
    return r


def ring_table(nside):
    """Per-ring geometry for rings i = 1 .. 4 Nside - 1 (index i - 1).

    Returns a dict of tensors: ``z`` (cos theta of the ring), ``sin_theta``,
    ``npix`` (pixels in the ring: 4i in the polar caps, 4 Nside in the
    equatorial belt), ``first`` (RING index of the ring's first pixel) and
    ``phi0`` (longitude of that first pixel; pixel j sits at
    phi0 + 2 pi j / npix).  Gorski et al. (2005), Eq. 4-9.
    """
    n = nside
    i = torch.arange(1, 4 * n, dtype=I64)
    north = i < n
    south = i > 3 * n
    ip = torch.where(south, 4 * n - i, i)            # ring counted from nearest pole
    polar = north | south
    a = ip.to(F64) * ip.to(F64) / (3.0 * n * n)       # 1 - |z| in the caps
    z_cap = 1.0 - a
    z_eq = (4.0 / 3.0) - (2.0 * i.to(F64)) / (3.0 * n)
    z = torch.where(polar, torch.where(north, z_cap, -z_cap), z_eq)
    sin_cap = torch.sqrt(a * (2.0 - a))
    sin_eq = torch.sqrt((1.0 - z_eq) * (1.0 + z_eq))
    sin_theta = torch.where(polar, sin_cap, sin_eq)
    nring = torch.where(polar, 4 * ip, torch.full_like(i, 4 * n))
    ncap = 2 * n * (n - 1)
    first = torch.where(north, 2 * i * (i - 1),
                        torch.where(south, npix(n) - 2 * ip * (ip + 1),
                                    ncap + (i - n) * 4 * n))
    # polar rings and equatorial rings with (i - Nside) even are offset by half a pixel
    half = polar | (((i - n) % 2) == 0)
    phi0 = torch.where(half, math.pi / nring.to(F64), torch.zeros_like(z))
    return {"z": z, "sin_theta": sin_theta, "npix": nring, "first": first, "phi0": phi0}


def pix2ring(nside, pix):
    """Ring number (1-based) and position j (0-based) of RING pixels."""
    n = nside
    pix = torch.as_tensor(pix, dtype=I64)
    ncap = 2 * n * (n - 1)
    np_ = npix(n)
    i_n = (1 + _isqrt(1 + 2 * pix)) // 2
    j_n = pix - 2 * i_n * (i_n - 1)
    q = pix - ncap
    i_e = q // (4 * n) + n
    j_e = q % (4 * n)
    qs = np_ - pix
    i_s = (1 + _isqrt((2 * qs - 1).clamp(min=0))) // 2
    j_s = pix - (np_ - 2 * i_s * (i_s + 1))
    is_n = pix < ncap
    is_s = pix >= np_ - ncap
    ring = torch.where(is_n, i_n, torch.where(is_s, 4 * n - i_s, i_e))
    j = torch.where(is_n, j_n, torch.where(is_s, j_s, j_e))
    return ring, j


def pix2ang_ring(nside, pix):
    """(z, phi) of RING pixel centres (Gorski et al. 2005, Eq. 4-9)."""
    rt = ring_table(nside)
    ring, j = pix2ring(nside, pix)
    r = ring - 1
    z = rt["z"][r]
    phi = rt["phi0"][r] + (2.0 * math.pi) * j.to(F64) / rt["npix"][r].to(F64)
    return z, phi


def _tt(phi):
    tt = phi * TWO_OVER_PI
    return torch.where(tt >= 4.0, tt - 4.0, tt)


def ang2pix_ring(nside, z, phi):
    """RING index of the pixel containing (z, phi) (Gorski et al. 2005, Sec. 5)."""
    n = nside
    nd = float(n)
    z = torch.as_tensor(z, dtype=F64)
    phi = torch.as_tensor(phi, dtype=F64)
    za = torch.abs(z)
    tt = _tt(phi)
    # equatorial belt: the two families of pixel-edge lines
    t1 = nd * (0.5 + tt)
    t2 = nd * (0.75 * z)
    jp = torch.trunc(t1 - t2).to(I64)
    jm = torch.trunc(t1 + t2).to(I64)
    ir = n + 1 + jp - jm
    kshift = 1 - (ir & 1)
    ipe = (jp + jm - n + kshift + 1) // 2
    ipe = torch.remainder(ipe, 4 * n)
    pix_eq = 2 * n * (n - 1) + (ir - 1) * 4 * n + ipe
    # polar caps
    tp = tt - torch.trunc(tt)
    tmp = nd * torch.sqrt(3.0 * (1.0 - za))
    jpp = torch.trunc(tp * tmp).to(I64)
    jmp = torch.trunc((1.0 - tp) * tmp).to(I64)
    irp = jpp + jmp + 1
    ipp = torch.trunc(tt * irp.to(F64)).to(I64)
    ipp = torch.remainder(ipp, 4 * irp)
    pix_n = 2 * irp * (irp - 1) + ipp
    pix_s = npix(n) - 2 * irp * (irp + 1) + ipp
    pix_p = torch.where(z > 0, pix_n, pix_s)
    return torch.where(za <= TWO_THIRDS, pix_eq, pix_p)


def _spread_bits(v, order):
    out = torch.zeros_like(v)
    for b in range(order):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def _compress_bits(v, order):
    out = torch.zeros_like(v)
    for b in range(order):
        out |= ((v >> (2 * b)) & 1) << b
    return out


def ang2pix_nest(nside, z, phi):
    """NEST index of the pixel containing (z, phi) (Gorski et al. 2005, Sec. 5)."""
    n = nside
    order = nside_order(n)
    nd = float(n)
    z = torch.as_tensor(z, dtype=F64)
    phi = torch.as_tensor(phi, dtype=F64)
    za = torch.abs(z)
    tt = _tt(phi)
    # equatorial belt
    t1 = nd * (0.5 + tt)
    t2 = nd * (0.75 * z)
    jp = torch.trunc(t1 - t2).to(I64)
    jm = torch.trunc(t1 + t2).to(I64)
    # phi rounded up to 2 pi: both edge indices past 4 Nside -> wrap both
    wrap = (jp >= 4 * n) & (jm >= 4 * n)
    jp = torch.where(wrap, jp - 4 * n, jp)
    jm = torch.where(wrap, jm - 4 * n, jm)
    ifp = jp >> order
    ifm = jm >> order
    face_eq = torch.where(ifp == ifm, torch.where(ifp == 4, torch.full_like(ifp, 4), ifp + 4),
                          torch.where(ifp < ifm, ifp, ifm + 8))
    ix_eq = jm & (n - 1)
    iy_eq = n - (jp & (n - 1)) - 1
    # polar caps
    ntt = torch.clamp(torch.trunc(tt).to(I64), max=3)
    tp = tt - ntt.to(F64)
    tmp = nd * torch.sqrt(3.0 * (1.0 - za))
    jpp = torch.clamp(torch.trunc(tp * tmp).to(I64), max=n - 1)
    jmp = torch.clamp(torch.trunc((1.0 - tp) * tmp).to(I64), max=n - 1)
    north = z >= 0
    face_p = torch.where(north, ntt, ntt + 8)
    ix_p = torch.where(north, n - jmp - 1, jpp)
    iy_p = torch.where(north, n - jpp - 1, jmp)
    eq = za <= TWO_THIRDS
    face = torch.where(eq, face_eq, face_p)
    ix = torch.where(eq, ix_eq, ix_p)
    iy = torch.where(eq, iy_eq, iy_p)
    return face * n * n + _spread_bits(ix, order) + (_spread_bits(iy, order) << 1)


# base-face coordinates: ring of the face's lowest corner (in units of Nside)
# and the longitude index of its centre (in units of pi/4), Gorski et al. 2005
_JRLL = torch.tensor([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4], dtype=I64)
_JPLL = torch.tensor([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7], dtype=I64)


def nest2ring(nside, pix):
    """RING index of NEST pixels (face, x, y -> ring, position)."""
    n = nside
    order = nside_order(n)
    pix = torch.as_tensor(pix, dtype=I64)
    face = pix >> (2 * order)
    ipf = pix & (n * n - 1)
    ix = _compress_bits(ipf, order)
    iy = _compress_bits(ipf >> 1, order)
    jr = _JRLL[face] * n - ix - iy - 1
    north = jr < n
    south = jr > 3 * n
    nr = torch.where(north, jr, torch.where(south, 4 * n - jr, torch.full_like(jr, n)))
    nbefore = torch.where(north, 2 * nr * (nr - 1),
                          torch.where(south, npix(n) - 2 * nr * (nr + 1),
                                      2 * n * (n - 1) + (jr - n) * 4 * n))
    kshift = torch.where(north | south, torch.zeros_like(jr), (jr - n) & 1)
    jp = (_JPLL[face] * nr + ix - iy + 1 + kshift) // 2
    jp = torch.where(jp > 4 * n, jp - 4 * n, jp)
    jp = torch.where(jp < 1, jp + 4 * n, jp)
    return nbefore + jp - 1


def ring2nest(nside, pix):
    """NEST index of RING pixels (inverse permutation of ``nest2ring``)."""
    inv = torch.empty(npix(nside), dtype=I64)
    inv[nest2ring(nside, torch.arange(npix(nside), dtype=I64))] = torch.arange(npix(nside), dtype=I64)
    return inv[torch.as_tensor(pix, dtype=I64)]


def pix2ang_nest(nside, pix):
    """(z, phi) of NEST pixel centres."""
    return pix2ang_ring(nside, nest2ring(nside, pix))


def vec_from_zphi(z, phi):
    """Unit 3-vector of (z, phi); sin theta from sqrt((1 - z)(1 + z))."""
    s = torch.sqrt((1.0 - z) * (1.0 + z))
    return torch.stack([s * torch.cos(phi), s * torch.sin(phi), z], dim=-1)


def pix2vec_ring(nside, pix):
    """Unit vectors of RING pixel centres; sin theta from the ring table."""
    rt = ring_table(nside)
    ring, j = pix2ring(nside, pix)
    r = ring - 1
    phi = rt["phi0"][r] + (2.0 * math.pi) * j.to(F64) / rt["npix"][r].to(F64)
    s = rt["sin_theta"][r]
    return torch.stack([s * torch.cos(phi), s * torch.sin(phi), rt["z"][r]], dim=-1)
