"""Pins of the oracle's spherical-harmonic Poisson solver (paper Sec. 3.2,
Appendix A, Appendix E) against libraries, symbolic algebra and the paper's
closed forms."""
import math

import numpy as np
import pytest
import scipy.special as sp
import sympy
import torch

from oracle import geometry, healpix as hp, sht

F64 = torch.float64


def test_legendre_matches_scipy():
    th = torch.tensor([1e-3, 0.02, 0.3, 1.0, 1.5707, 2.0, 3.1, math.pi - 1e-3], dtype=F64)
    L = 60
    for m, lam in sht.legendre_columns(L, torch.cos(th), torch.sin(th)):
        for l in range(m, L + 1):
            ref = sp.sph_harm_y(l, m, th.numpy(), 0.0).real
            assert np.allclose(lam[l - m].numpy(), ref, rtol=1e-11, atol=1e-13), (l, m)


def test_legendre_high_degree_matches_scipy():
    th = torch.tensor([0.05, 0.7, 1.2, 1.55], dtype=F64)
    L = 1000
    want = {(1000, 0), (1000, 17), (900, 400), (1000, 999), (700, 700)}
    import mpmath
    mpmath.mp.dps = 40
    for m, lam in sht.legendre_columns(L, torch.cos(th), torch.sin(th)):
        for (l, mm) in want:
            if mm == m:
                ref = np.array([float(mpmath.re(mpmath.spherharm(l, m, float(t), 0))) for t in th])
                assert np.allclose(lam[l - m].numpy(), ref, rtol=1e-9, atol=1e-12), (l, m)


def test_legendre_through_underflowed_start():
    """sin^m theta underflows FP64 (lambda_mm ~ 1e-317) but lambda_lm grows
    back to order one near the turning point l ~ m / sin theta: the scaled
    recurrence must carry it (checked against mpmath)."""
    import mpmath
    mpmath.mp.dps = 40
    th = torch.tensor([0.3], dtype=F64)
    m, L = 600, 2100
    for mm, lam in sht.legendre_columns(L, torch.cos(th), torch.sin(th), mmax=m, mmin=m):
        for l in (600, 1200, 1800, 2000, 2100):
            ref = float(mpmath.re(mpmath.spherharm(l, m, 0.3, 0)))
            assert abs(float(lam[l - m, 0]) - ref) <= 1e-10 * abs(ref) + 1e-300, (l, ref)
    assert abs(float(lam[2100 - m, 0])) > 1e-3


def test_legendre_no_underflow_garbage():
    # near the pole sin^m theta underflows FP64 for large m; values must be 0
    # or tiny, never NaN / inf, and columns m <= 2 must stay accurate
    z = torch.tensor([1 - 1e-9, 1 - 1e-6], dtype=F64)
    s = torch.sqrt((1 - z) * (1 + z))
    for m, lam in sht.legendre_columns(600, z, s, mmax=600):
        assert torch.isfinite(lam).all()
        assert lam.abs().max() < 100


def _ylm_sym(l, m):
    t, p = sympy.symbols("t p", real=True)
    return t, p, sympy.Ynm(l, m, t, p).expand(func=True)


@pytest.mark.parametrize("l,m", [(1, 0), (2, 0), (2, 1), (3, 1), (3, 3), (4, 2), (5, 4)])
def test_synthesis_and_derivatives_of_single_harmonic(l, m):
    """psi = Re Y_lm (coefficient 1/2 at m > 0, 1 at m = 0): synthesis and the
    pure-SHT derivative synthesis agree with symbolic derivatives of Y_lm."""
    nside, L = 8, 12
    alm = torch.zeros(sht.nalm(L), dtype=torch.complex128)
    alm[sht.alm_index(L, l, m)] = 1.0 if m == 0 else 0.5
    d = sht.derivative_synthesis(alm, nside, L)
    t, p, y = _ylm_sym(l, m)
    z, phi = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    th = np.arccos(z.numpy())
    ph = phi.numpy()
    exprs = {"psi": y, "p_t": sympy.diff(y, t), "p_p": sympy.diff(y, p), "p_tt": sympy.diff(y, t, 2),
             "p_pp": sympy.diff(y, p, 2), "p_tp": sympy.diff(y, t, p)}
    for k, e in exprs.items():
        f = sympy.lambdify((t, p), sympy.re(e), "numpy")
        ref = np.broadcast_to(f(th, ph), th.shape)
        assert np.allclose(d[k].numpy(), ref, atol=1e-12), k
    # the synthesis alone gives the same psi
    assert torch.allclose(sht.synthesis(alm, nside, L), d["psi"], atol=1e-13)
    # the fields synthesised at arbitrary points (off the pixel grid, poles
    # excluded) against the Appendix A formulas on the symbolic partials
    g = torch.Generator().manual_seed(l * 10 + m)
    zr = 1.8 * torch.rand(40, generator=g, dtype=F64) - 0.9
    pr = 2 * math.pi * torch.rand(40, generator=g, dtype=F64)
    sr = torch.sqrt((1 - zr) * (1 + zr))
    nv = torch.stack([sr * torch.cos(pr), sr * torch.sin(pr), zr], -1)
    got = sht.lens_fields_at(alm, L, nv)
    ev = {k: torch.from_numpy(np.broadcast_to(sympy.lambdify((t, p), sympy.re(e), "numpy")(
        np.arccos(zr.numpy()), pr.numpy()), zr.shape).copy()) for k, e in exprs.items()}
    want = geometry.lens_fields_from_partials(ev["p_t"], ev["p_p"], ev["p_tt"], ev["p_pp"], ev["p_tp"], sr, zr)
    for k in want:
        assert torch.allclose(got[k], want[k], rtol=0, atol=1e-11), k


def test_laplacian_eigen_relation():
    """U from the derivative synthesis has trace -l(l+1) psi (the Y_lm
    eigen-relation), for a random band-limited psi."""
    nside, L = 16, 30
    g = torch.Generator().manual_seed(3)
    alm = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    for l in range(L + 1):
        i = sht.alm_index(L, l, 0)
        alm[i] = complex(alm[i].real.item(), 0.0)
    d = sht.derivative_synthesis(alm, nside, L)
    s, c = sht.pixel_sin_cos(nside)
    lf = geometry.lens_fields_from_partials(d["p_t"], d["p_p"], d["p_tt"], d["p_pp"], d["p_tp"], s, c)
    ell = sht.ell_of_index(L).to(F64)
    lap = sht.synthesis(-ell * (ell + 1) * alm, nside, L)
    assert torch.allclose(lf["u_tt"] + lf["u_pp"], lap, atol=1e-10 * lap.abs().max())


def test_analysis_is_weighted_adjoint_of_synthesis():
    nside, L = 8, 20
    g = torch.Generator().manual_seed(4)
    a = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    f = torch.randn(hp.npix(nside), dtype=F64, generator=g)
    lhs = (sht.synthesis(a, nside, L) * f).sum()
    af = sht.analysis(f, nside, L)
    mm = torch.cat([torch.full((L + 1 - m,), m) for m in range(L + 1)])
    cm = torch.where(mm == 0, 1.0, 2.0).to(F64)
    w = 4 * math.pi / hp.npix(nside)
    # real part of the m = 0 coefficients only enters a real field
    a0 = torch.where(mm == 0, a.real.to(torch.complex128), a)
    lhs = (sht.synthesis(a0, nside, L) * f).sum()
    rhs = (cm * (a0 * af.conj()).real).sum() / w
    assert abs(float(lhs - rhs)) < 1e-11 * float(abs(lhs) + 1)


def test_ring_restricted_synthesis_against_direct_sum():
    """synthesis_rings on a few rings (polar cap, belt, last ring) equals the
    direct sum of a_lm Y_lm (scipy) at those rings' pixel centres; every other
    pixel is NaN."""
    nside, L = 8, 12
    g = torch.Generator().manual_seed(6)
    alm = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    rings = [0, 5, 14, 30]
    f = sht.synthesis_rings(alm, nside, L, rings)
    ring, _ = hp.pix2ring(nside, torch.arange(hp.npix(nside)))
    on = torch.isin(ring - 1, torch.tensor(rings))
    z, phi = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside))[on])
    th = np.arccos(z.numpy())
    want = np.zeros(th.shape)
    for m in range(L + 1):
        for l in range(m, L + 1):
            y = sp.sph_harm_y(l, m, th, phi.numpy())
            a = complex(alm[sht.alm_index(L, l, m)])
            want += (a * y).real if m == 0 else 2.0 * (a * y).real
    assert np.allclose(f[on].numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert bool(torch.isnan(f[~on]).all())


def test_iterated_analysis_recovers_band_limited_map():
    """Jacobi-iterated analysis a <- a + A(f - S a) converges to the exact
    coefficients of a band-limited map (L <= Nside / 2)."""
    nside, L = 16, 8
    g = torch.Generator().manual_seed(5)
    alm = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    for l in range(L + 1):
        i = sht.alm_index(L, l, 0)
        alm[i] = complex(alm[i].real.item(), 0.0)
    f = sht.synthesis(alm, nside, L)
    a = sht.analysis(f, nside, L)
    for _ in range(8):
        a = a + sht.analysis(f - sht.synthesis(a, nside, L), nside, L)
    assert (a - alm).abs().max() < 1e-10


def test_poisson_zero_monopole():
    L = 10
    k = torch.ones(sht.nalm(L), dtype=torch.complex128)
    psi = sht.poisson(k, L)
    assert psi[sht.alm_index(L, 0, 0)] == 0
    assert torch.allclose(psi[sht.alm_index(L, 3, 2)], torch.tensor(-1 / 12, dtype=torch.complex128))


# ---- Appendix E: the Epanechnikov kernel at the north pole ------------------

def sinc(x):
    return np.sinc(x)            # sin(pi x) / (pi x)


def ep_norm(sig):
    return 2 * np.pi * (sinc(sig / 2 / np.pi) ** 2 - 2 * sinc(sig / np.pi) + 1)


def ep_kernel(th, sig):
    return np.where(th < sig, (1 - (th / sig) ** 2) / ep_norm(sig), 0.0)


def ep_h(th, sig):
    return ((th / sig) ** 2 * (-2 * sinc(th / np.pi) + np.cos(th) + sinc(th / 2 / np.pi) ** 2)
            + 1 - np.cos(th)) / (ep_norm(sig) * (1 - np.cos(th))) - 1 / (4 * np.pi)


def ep_alpha_gamma(th, sig):
    """alpha_theta and gamma_1 of the kernel minus its mean (Appendix E);
    outside sigma the point-mass forms of Appendix A."""
    inside = th < sig
    a_in = -ep_h(th, sig) * (1 - np.cos(th)) / np.sin(th)
    a_out = -(1 / (4 * np.pi)) * np.sin(th) / (1 - np.cos(th))
    g_in = -0.5 * (2 * np.cos(th) / (1 + np.cos(th)) * ep_h(th, sig) - ep_kernel(th, sig) + 1 / (4 * np.pi))
    g_out = -(1 / (8 * np.pi)) * (1 + np.cos(th)) / (1 - np.cos(th))
    return np.where(inside, a_in, a_out), np.where(inside, g_in, g_out)


def test_epanechnikov_normalisation():
    for sig in (0.05, 0.5, 1.0):
        th = np.linspace(0, sig, 200001)
        integ = np.trapezoid(2 * np.pi * np.sin(th) * ep_kernel(th, sig), th)
        assert abs(integ - 1) < 1e-8


def test_epanechnikov_closed_form_matches_sht_solution():
    """The oracle's SHT Poisson solve and derivative synthesis of a smooth
    kernel source reproduce the closed-form deflection and shear of
    Appendix E (signs of Appendix A).  Three Jacobi iterations of the
    analysis remove the HEALPix quadrature error, so what is left is the
    band-limit truncation at the kernel's edge."""
    nside, L, sig = 32, 64, 0.6
    z, phi = hp.pix2ang_ring(nside, torch.arange(hp.npix(nside)))
    th = np.arccos(z.numpy())
    kappa = torch.from_numpy(ep_kernel(th, sig) - 1 / (4 * np.pi))
    a = sht.analysis(kappa, nside, L)
    for _ in range(3):
        a = a + sht.analysis(kappa - sht.synthesis(a, nside, L), nside, L)
    d = sht.derivative_synthesis(sht.poisson(a, L), nside, L)
    s, c = sht.pixel_sin_cos(nside)
    out = geometry.lens_fields_from_partials(d["p_t"], d["p_p"], d["p_tt"], d["p_pp"], d["p_tp"], s, c)
    a_ref, g_ref = ep_alpha_gamma(th, sig)
    k, g1, g2 = geometry.kappa_gamma(out["u_tt"], out["u_pp"], out["u_tp"])
    sel = (np.abs(th - sig) > 0.15) & (th > 0.15) & (th < np.pi - 0.15)
    a_err = np.abs(out["a_th"].numpy()[sel] - a_ref[sel]).max() / np.abs(a_ref[sel]).max()
    g_err = np.abs(g1.numpy()[sel] - g_ref[sel]).max() / np.abs(g_ref[sel]).max()
    assert a_err < 1e-3 and g_err < 1e-2, (a_err, g_err)
    assert np.abs(out["a_ph"].numpy()[sel]).max() < 1e-4 * np.abs(a_ref[sel]).max()
    assert np.abs(g2.numpy()[sel]).max() < 1e-4 * np.abs(g_ref[sel]).max()


def test_poisson_solve_against_the_greens_function():
    """Brute force with the Green's function of the sphere's Laplacian,
    G(n, n') = ln(1 - n . n') / 4 pi (the point-mass potential of Appendix A):
    psi_p = (1 / Npix) sum_{q != p} ln(1 - n_p . n_q) kappa_q, plus the own
    pixel's part taken over a disc of equal area.  It agrees with the SHT
    solve of a band-limited kappa up to the discretisation error, which falls
    at second order in the pixel size (constants removed)."""
    errs = []
    for nside in (8, 16):
        L = 3 * nside - 1
        gen = torch.Generator().manual_seed(3)
        a = torch.zeros(sht.nalm(L), dtype=torch.complex128)
        for l in range(1, 7):
            for m in range(0, l + 1):
                re = torch.randn(1, generator=gen, dtype=torch.float64).item()
                im = torch.randn(1, generator=gen, dtype=torch.float64).item() if m > 0 else 0.0
                a[sht.alm_index(L, l, m)] = complex(re, im)
        kappa = sht.synthesis(a, nside, L)
        psi = sht.poisson_sht(kappa, nside, L, derivatives=False)["psi"]
        n = hp.pix2vec_ring(nside, torch.arange(hp.npix(nside)))
        npx = n.shape[0]
        G = torch.log(1.0 - (n @ n.T).clamp(max=1.0))
        G.fill_diagonal_(0.0)
        om = 4 * np.pi / npx
        bf = (G @ kappa) / npx + kappa * om / (4 * np.pi) * (np.log(om / np.pi / 2) - 1)
        d = (bf - bf.mean()) - (psi - psi.mean())
        errs.append(float(d.norm() / (psi - psi.mean()).norm()))
    assert errs[0] < 2e-2 and errs[1] < 5e-3, errs
    assert errs[0] > 3.0 * errs[1], errs
