"""Flat LCDM distances, growth and lens-plane source scalings (host, FP64).

Sec. 2.1: chi(a) = c int_a^1 da' / (a'^2 H(a')), H(a) = H0 sqrt(Om a^-3 + 1 - Om)
(flat, so r(chi) = chi), and the plane source of Eq. lenspoisson,
kappa^(m) = Om (3 H0^2 / c^2) (r(chi_m) / a(chi_m)) int delta dchi', which for a
shell of width dchi and overdensity delta_m gives the scale
s_m = 3 Om (H0 / c)^2 (chi_m / a_m) dchi.  The linear growth factor
D(a) ~ H(a) int_0^a da' / (a' H(a'))^3, D(1) = 1, scales the synthetic
lognormal planes (a standard result, not from the paper).  Distances are in
Mpc/h, so c / H0 = 2997.92458 Mpc/h.
"""
import math

from scipy import integrate, optimize

C_OVER_H0 = 2997.92458


def efunc(z, om):
    return math.sqrt(om * (1 + z) ** 3 + 1 - om)


def chi_of_z(z, om):
    val, _ = integrate.quad(lambda x: 1.0 / efunc(x, om), 0.0, z, epsabs=1e-13, epsrel=1e-13, limit=200)
    return C_OVER_H0 * val


def z_of_chi(chi, om):
    if chi <= 0:
        return 0.0
    return optimize.brentq(lambda z: chi_of_z(z, om) - chi, 0.0, 20.0, xtol=1e-14, rtol=1e-14)


def growth(z, om):
    a = 1.0 / (1.0 + z)

    def d_unnorm(a):
        ha = math.sqrt(om * a ** -3 + 1 - om)
        val, _ = integrate.quad(lambda x: 1.0 / (x * math.sqrt(om * x ** -3 + 1 - om)) ** 3, 0.0, a,
                                epsabs=1e-14, epsrel=1e-12, limit=200)
        return ha * val
    return d_unnorm(a) / d_unnorm(1.0)


def lens_planes(nplanes, dchi, om=0.25):
    """Planes at chi_m = (m + 1/2) dchi, m = 0 .. N-1, source sphere at
    chi_N = N dchi (outer edge of the last shell).  Returns dict with chi
    (N + 1 values), z, a, growth and the source scale s_m of each plane."""
    chi = [(m + 0.5) * dchi for m in range(nplanes)] + [nplanes * dchi]
    zs = [z_of_chi(c, om) for c in chi[:nplanes]]
    a = [1.0 / (1.0 + z) for z in zs]
    D = [growth(z, om) for z in zs]
    scale = [3.0 * om * chi[m] / a[m] * dchi / C_OVER_H0 ** 2 for m in range(nplanes)]
    return {"chi": chi, "z": zs, "a": a, "growth": D, "scale": scale, "om": om}
