"""Pins of the oracle's E/B decomposition and spectra (paper Sec. 5)."""
import math

import torch

from oracle import geometry, healpix as hp, sht, spectra

F64 = torch.float64


def _alm(L, seed, lmin=2):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn(sht.nalm(L), dtype=torch.complex128, generator=g)
    for m in range(L + 1):
        for l in range(m, L + 1):
            i = sht.alm_index(L, l, m)
            if l < lmin:
                a[i] = 0
            elif m == 0:
                a[i] = complex(a[i].real.item(), 0.0)
    return a


def _fields(psi_lm, nside, L):
    d = sht.derivative_synthesis(psi_lm, nside, L)
    s, c = sht.pixel_sin_cos(nside)
    return geometry.lens_fields_from_partials(d["p_t"], d["p_p"], d["p_tt"], d["p_pp"], d["p_tp"], s, c)


def _norm(L):
    l = sht.ell_of_index(L).to(F64)
    return torch.sqrt(torch.clamp((l + 2) * (l + 1) * l * (l - 1), min=0.0))


def test_shear_of_a_potential_is_pure_e():
    """gamma = eth^2 psi / 2 (gamma_1 = (U_tt - U_pp)/2, gamma_2 = U_tp) has
    E_lm = N_l psi_lm / 2 and B_lm = 0 (up to the quadrature error of the
    uniform-weight analysis, small for lmax << nside)."""
    nside, L = 32, 12
    psi = _alm(L, 1)
    f = _fields(psi, nside, L)
    k, g1, g2 = geometry.kappa_gamma(f["u_tt"], f["u_pp"], f["u_tp"])
    E, B = spectra.eb_analysis(g1, g2, nside, L)
    want = 0.5 * _norm(L) * psi
    assert (E - want).abs().max() < 2e-3 * want.abs().max()
    assert B.abs().max() < 2e-3 * want.abs().max()


def test_curl_field_is_pure_b():
    """gamma = i eth^2 psi_B / 2 (gamma_1 = -U_tp, gamma_2 = (U_tt - U_pp)/2
    of psi_B) has B_lm = N_l psi_B,lm / 2 and E_lm = 0."""
    nside, L = 32, 12
    psi = _alm(L, 2)
    f = _fields(psi, nside, L)
    k, g1, g2 = geometry.kappa_gamma(f["u_tt"], f["u_pp"], f["u_tp"])
    E, B = spectra.eb_analysis(-g2, g1, nside, L)
    want = 0.5 * _norm(L) * psi
    assert (B - want).abs().max() < 2e-3 * want.abs().max()
    assert E.abs().max() < 2e-3 * want.abs().max()


def test_cl_of_single_harmonic():
    L = 6
    a = torch.zeros(sht.nalm(L), dtype=torch.complex128)
    a[sht.alm_index(L, 4, 0)] = 2.0
    a[sht.alm_index(L, 4, 3)] = 1.0 + 1.0j
    c = spectra.cl(a, L)
    assert abs(float(c[4]) - (4.0 + 2 * 2.0) / 9.0) < 1e-15
    assert float(c.sum() - c[4]) == 0.0


def test_single_plane_spectra_e_equals_kappa_and_no_rotation():
    """One lens plane: A = I - c U with U symmetric, so omega = 0 and B = 0;
    E and kappa spectra of the same potential satisfy
    C^EE_l / C^kk_l = (l+2)(l-1) / (l(l+1)) exactly (Sec. 5's E ~ kappa)."""
    nside, L = 32, 12
    psi = _alm(L, 3)
    f = _fields(psi, nside, L)
    cfac = 0.3
    A = torch.eye(2, dtype=F64).expand(hp.npix(nside), 2, 2).clone()
    A[:, 0, 0] -= cfac * f["u_tt"]
    A[:, 1, 1] -= cfac * f["u_pp"]
    A[:, 0, 1] -= cfac * f["u_tp"]
    A[:, 1, 0] -= cfac * f["u_tp"]
    sp = spectra.spectra_from_A(A, nside, L)
    l = torch.arange(L + 1, dtype=F64)
    ratio = sp["E"][2:] / sp["kappa"][2:]
    want = ((l + 2) * (l - 1) / (l * (l + 1)))[2:]
    assert torch.allclose(ratio, want, rtol=3e-2)   # uniform-quadrature error, largest at l = 2
    assert float(sp["omega"].max()) < 1e-28
    assert float(sp["B"].max()) < 1e-5 * float(sp["E"].max())
