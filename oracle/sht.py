"""Spherical-harmonic transforms on HEALPix rings (oracle; test infrastructure).

Sec. 3.2 of the paper solves the plane Poisson equation by an SHT analysis
of the source, psi_lm = -kappa_lm / (l (l + 1)) with the l = 0 term set to
zero, and a synthesis back to the map; the pure-SHT solver synthesises the
derivatives of psi directly from psi_lm.  The transforms run over HEALPix
rings with FFTs along each ring and Legendre sums across rings (Sec. 3.2,
"fast SHT" of Press et al. 2007 Sec. 6.7).

Conventions (readings where the paper is silent):
* Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi}, orthonormal, with the
  Condon-Shortley phase; lambda_mm = (-1)^m sqrt((2m+1)!! / (4 pi (2m)!!))
  sin^m theta and the three-term recurrence in l.
* Analysis is plain uniform quadrature, a_lm = (4 pi / Npix) sum_p f_p
  Y*_lm(p), with no iterative refinement.
* Real fields: only m >= 0 is stored; a_lm is packed m-major with index
  m (2 L + 1 - m) / 2 + l.
* Along a ring of n pixels the Fourier coefficient of order m is the DFT bin
  m mod n (aliasing on short polar rings).

The FFT is torch.fft (a library primitive); every other step is written out.
"""
import math

import torch

from . import healpix as hp

F64 = torch.float64
C128 = torch.complex128


def nalm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def _times_pow2(p, e):
    """p * 2^e for int64 exponents e, with one final rounding: 2^e alone
    underflows FP64 for e < -1074 although p * 2^e may not."""
    lo = e < -1000
    e1 = torch.where(lo, e + 600, e).to(F64)
    return torch.where(lo, torch.ldexp(p, e1) * 2.0 ** -600, torch.ldexp(p, e1))


def legendre_columns(lmax, z, sin_theta, mmax=None, mmin=0):
    """Yield (m, lam) with lam[l - m, r] = lambda_lm(z_r) for l = m .. lmax.

    lambda_mm is carried as mantissa * 2^exponent so that sin^m theta never
    underflows; the l-recurrence runs on the mantissas (it is linear), which
    are renormalised by 2^-400 when they grow, and the result is converted
    with one final rounding (values below the FP64 range become 0 there).
    Columns m < mmin are skipped.
    """
    if mmax is None:
        mmax = lmax
    z = torch.as_tensor(z, dtype=F64)
    s = torch.as_tensor(sin_theta, dtype=F64)
    mant = torch.full_like(z, math.sqrt(1.0 / (4.0 * math.pi)))
    expo = torch.zeros(z.shape, dtype=torch.int64)
    for m in range(0, mmax + 1):
        if m > 0:
            mant = mant * (-math.sqrt((2.0 * m + 1.0) / (2.0 * m))) * s
            fr = torch.frexp(mant)
            mant = fr.mantissa
            expo = expo + fr.exponent.to(torch.int64)
        if m < mmin:
            continue
        nl = lmax - m + 1
        out = torch.empty((nl, z.numel()), dtype=F64)
        e = expo.clone()
        p2 = mant.clone()                      # lambda_{l-2}
        out[0] = _times_pow2(p2, e)
        if nl > 1:
            p1 = math.sqrt(2.0 * m + 3.0) * z * p2   # lambda_{m+1, m}
            out[1] = _times_pow2(p1, e)
            for l in range(m + 2, lmax + 1):
                a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                p0 = a * (z * p1 - b * p2)
                big = torch.abs(p0) > 2.0 ** 400
                if bool(big.any()):
                    sc = torch.where(big, torch.tensor(2.0 ** -400, dtype=F64), torch.tensor(1.0, dtype=F64))
                    p0 = p0 * sc
                    p1 = p1 * sc
                    e = e + torch.where(big, 400, 0)
                out[l - m] = _times_pow2(p0, e)
                p2, p1 = p1, p0
        yield m, out


def eps_lm(l, m):
    """epsilon_lm = sqrt((l^2 - m^2) / (4 l^2 - 1)) (0 for l <= |m|)."""
    l = torch.as_tensor(l, dtype=F64)
    num = l * l - m * m
    return torch.where(num > 0, torch.sqrt(num.clamp(min=0) / (4.0 * l * l - 1.0)), torch.zeros_like(l))


def dtheta_columns(lmax, z, sin_theta):
    """Yield (m, lam, dlam, d2lam) for l = m .. lmax with theta derivatives:
    sin(t) d/dt lambda_lm = l eps_{l+1,m} lambda_{l+1,m} - (l+1) eps_lm lambda_{l-1,m}
    and the Legendre equation
    d2/dt2 lambda_lm = -cot(t) d/dt lambda_lm - (l(l+1) - m^2 / sin^2 t) lambda_lm."""
    z = torch.as_tensor(z, dtype=F64)
    s = torch.as_tensor(sin_theta, dtype=F64)
    for m, lam in legendre_columns(lmax + 1, z, s, mmax=lmax):
        l = torch.arange(m, lmax + 2, dtype=F64)
        nl = lmax - m + 1
        lam_lo = torch.cat([torch.zeros_like(lam[:1]), lam[:-1]], 0)  # lambda_{l-1}
        lam_hi = lam[1:]                                             # lambda_{l+1}
        lv = l[:nl, None]
        sdl = lv * eps_lm(lv + 1, m) * lam_hi - (lv + 1) * eps_lm(lv, m) * lam_lo[:nl]
        dl = sdl / s
        d2l = -(z / s) * dl - (lv * (lv + 1) - (m * m) / (s * s)) * lam[:nl]
        yield m, lam[:nl], dl, d2l


def ring_fourier(nside, f, mmax):
    """F[r, m] = sum_j f_j e^{-i m phi_j} on every ring r (DFT bin m mod n)."""
    rt = hp.ring_table(nside)
    nr = rt["npix"].numel()
    out = torch.zeros((nr, mmax + 1), dtype=C128)
    m = torch.arange(mmax + 1)
    for r in range(nr):
        n = int(rt["npix"][r])
        first = int(rt["first"][r])
        X = torch.fft.fft(f[first:first + n].to(C128))
        phase = torch.exp(-1j * m.to(F64) * float(rt["phi0"][r]))
        out[r] = X[m % n] * phase
    return out


def ring_inverse_fourier(nside, G, mmax):
    """f_j = sum_{m=0}^{mmax} c_m Re(G[r, m] e^{i m phi_j}), c_0 = 1, c_m = 2."""
    rt = hp.ring_table(nside)
    f = torch.empty(hp.npix(nside), dtype=F64)
    m = torch.arange(mmax + 1)
    c = torch.where(m == 0, 1.0, 2.0).to(F64)
    for r in range(G.shape[0]):
        n = int(rt["npix"][r])
        first = int(rt["first"][r])
        H = torch.zeros(n, dtype=C128)
        H.index_add_(0, m % n, c * G[r] * torch.exp(1j * m.to(F64) * float(rt["phi0"][r])))
        f[first:first + n] = (torch.fft.ifft(H) * n).real
    return f


def analysis(f, nside, lmax):
    """a_lm = (4 pi / Npix) sum_p f_p Y*_lm(p), m >= 0 (Sec. 3.2)."""
    rt = hp.ring_table(nside)
    F = ring_fourier(nside, f, lmax)
    w = 4.0 * math.pi / hp.npix(nside)
    alm = torch.zeros(nalm(lmax), dtype=C128)
    for m, lam in legendre_columns(lmax, rt["z"], rt["sin_theta"]):
        i0 = alm_index(lmax, m, m)
        alm[i0:i0 + lmax - m + 1] = w * (lam.to(C128) @ F[:, m])
    return alm


def synthesis(alm, nside, lmax):
    """f_p = sum_lm a_lm Y_lm(p) for a real field (Sec. 3.2)."""
    rt = hp.ring_table(nside)
    G = torch.zeros((rt["z"].numel(), lmax + 1), dtype=C128)
    for m, lam in legendre_columns(lmax, rt["z"], rt["sin_theta"]):
        i0 = alm_index(lmax, m, m)
        G[:, m] = lam.T.to(C128) @ alm[i0:i0 + lmax - m + 1]
    return ring_inverse_fourier(nside, G, lmax)


def synthesis_rings(alm, nside, lmax, rings):
    """The synthesis of `synthesis` on the listed rings only (0-based ring
    indices); every other pixel of the returned map is NaN, so a later use of
    a pixel that was not synthesised shows up as NaN.  The same sums as the
    full synthesis, restricted to fewer rings."""
    rt = hp.ring_table(nside)
    rings = torch.as_tensor(rings, dtype=torch.int64)
    G = torch.zeros((rings.numel(), lmax + 1), dtype=C128)
    for m, lam in legendre_columns(lmax, rt["z"][rings], rt["sin_theta"][rings]):
        i0 = alm_index(lmax, m, m)
        G[:, m] = lam.T.to(C128) @ alm[i0:i0 + lmax - m + 1]
    f = torch.full((hp.npix(nside),), float("nan"), dtype=F64)
    m = torch.arange(lmax + 1)
    c = torch.where(m == 0, 1.0, 2.0).to(F64)
    for k, r in enumerate(rings.tolist()):
        n = int(rt["npix"][r])
        first = int(rt["first"][r])
        H = torch.zeros(n, dtype=C128)
        H.index_add_(0, m % n, c * G[k] * torch.exp(1j * m.to(F64) * float(rt["phi0"][r])))
        f[first:first + n] = (torch.fft.ifft(H) * n).real
    return f


def ell_of_index(lmax):
    ls = []
    for m in range(lmax + 1):
        ls.append(torch.arange(m, lmax + 1))
    return torch.cat(ls)


def poisson(kappa_lm, lmax):
    """psi_lm = -kappa_lm / (l (l + 1)), psi_00 = 0 (Sec. 3.2, the harmonic
    form of Eq. lenspoisson)."""
    l = ell_of_index(lmax).to(F64)
    den = l * (l + 1.0)
    psi = torch.where(l > 0, -kappa_lm / torch.where(l > 0, den, 1.0), torch.zeros_like(kappa_lm))
    return psi


def derivative_synthesis(psi_lm, nside, lmax):
    """psi and its first and second theta/phi partial derivatives at every
    pixel centre, synthesised directly from psi_lm (the pure-SHT solver of
    Sec. 3.2).  Returns a dict of maps: psi, p_t, p_p, p_tt, p_pp, p_tp."""
    rt = hp.ring_table(nside)
    nr = rt["z"].numel()
    G0 = torch.zeros((nr, lmax + 1), dtype=C128)
    G1 = torch.zeros_like(G0)
    G2 = torch.zeros_like(G0)
    for m, lam, dl, d2l in dtheta_columns(lmax, rt["z"], rt["sin_theta"]):
        i0 = alm_index(lmax, m, m)
        a = psi_lm[i0:i0 + lmax - m + 1]
        G0[:, m] = lam.T.to(C128) @ a
        G1[:, m] = dl.T.to(C128) @ a
        G2[:, m] = d2l.T.to(C128) @ a
    im = 1j * torch.arange(lmax + 1).to(F64)
    return {
        "psi": ring_inverse_fourier(nside, G0, lmax),
        "p_t": ring_inverse_fourier(nside, G1, lmax),
        "p_tt": ring_inverse_fourier(nside, G2, lmax),
        "p_p": ring_inverse_fourier(nside, G0 * im, lmax),
        "p_pp": ring_inverse_fourier(nside, G0 * im * im, lmax),
        "p_tp": ring_inverse_fourier(nside, G1 * im, lmax),
    }


def lens_fields_at(psi_lm, lmax, nvec):
    """alpha and U (Appendix A conventions, (theta-hat, phi-hat) basis) of the
    band-limited potential psi_lm at arbitrary unit vectors nvec[M, 3], by
    direct synthesis of psi's partial derivatives there: the fields of the
    pure-SHT solver (Sec. 3.2) without a map grid or an interpolation."""
    from . import geometry
    z = nvec[:, 2].contiguous()
    s = torch.sqrt(nvec[:, 0] ** 2 + nvec[:, 1] ** 2)
    ph = torch.atan2(nvec[:, 1], nvec[:, 0])
    acc = {k: torch.zeros(z.shape, dtype=F64) for k in ("p_t", "p_p", "p_tt", "p_pp", "p_tp")}
    for m, lam, dl, d2l in dtheta_columns(lmax, z, s):
        i0 = alm_index(lmax, m, m)
        a = psi_lm[i0:i0 + lmax - m + 1].to(C128)
        e = torch.exp(1j * m * ph)
        c = 1.0 if m == 0 else 2.0
        g0 = (lam.T.to(C128) @ a) * e
        g1 = (dl.T.to(C128) @ a) * e
        g2 = (d2l.T.to(C128) @ a) * e
        acc["p_t"] += c * g1.real
        acc["p_tt"] += c * g2.real
        acc["p_p"] += c * (1j * m * g0).real
        acc["p_pp"] += c * (-(m * m) * g0).real
        acc["p_tp"] += c * (1j * m * g1).real
    return geometry.lens_fields_from_partials(acc["p_t"], acc["p_p"], acc["p_tt"], acc["p_pp"], acc["p_tp"], s, z)


def pixel_sin_cos(nside):
    """sin theta and cos theta at every RING pixel centre."""
    rt = hp.ring_table(nside)
    ring, _ = hp.pix2ring(nside, torch.arange(hp.npix(nside)))
    return rt["sin_theta"][ring - 1], rt["z"][ring - 1]


def poisson_sht(kappa, nside, lmax, derivatives=True):
    """Full pure-SHT plane solve: analysis of kappa, harmonic Poisson
    solve, synthesis of psi and (optionally) of alpha and U in the
    (theta-hat, phi-hat) basis with the sign conventions of Appendix A."""
    from . import geometry
    klm = analysis(kappa, nside, lmax)
    plm = poisson(klm, lmax)
    if not derivatives:
        return {"psi": synthesis(plm, nside, lmax)}
    d = derivative_synthesis(plm, nside, lmax)
    s, c = pixel_sin_cos(nside)
    out = geometry.lens_fields_from_partials(d["p_t"], d["p_p"], d["p_tt"], d["p_pp"], d["p_tp"], s, c)
    out["psi"] = d["psi"]
    return out
