"""Convergence, E/B-mode shear and rotation power spectra (oracle; test
infrastructure).

Sec. 5 of the paper extracts kappa, gamma and omega from the final inverse
magnification matrices (Eq. invmagmat) and measures their full-sky power
spectra, with the shear split into E and B modes.  Conventions used here
(readings; the paper defers to the HEALPix package):

* the shear gamma = gamma_1 + i gamma_2 in the (theta-hat, phi-hat) basis is
  a spin-2 field; with the spin raising operator
  eth f = -(sin t)^s (d_t + i / sin t d_p)[(sin t)^-s f], a potential field
  gives gamma = eth^2 psi / 2 (so gamma_1 = (U_tt - U_pp)/2, gamma_2 = U_tp);
* spin-2 harmonics _{+-2}Y_lm = eth^2 Y_lm / N_l (resp. with eth-bar),
  N_l = sqrt((l+2)! / (l-2)!); acting on Y_lm = lambda_lm e^{i m phi}:
  eth^2 Y_lm = (A_lm - B_lm) e^{i m phi}, eth-bar^2 Y_lm = (A_lm + B_lm) e^{i m phi},
  A_lm = -2 cot t dlambda - (l(l+1) - 2 m^2 / sin^2 t) lambda,
  B_lm = (2 m / sin t)(dlambda - cot t lambda);
* E_lm = (_2a_lm + _-2a_lm)/2 and B_lm = -i (_2a_lm - _-2a_lm)/2 with
  _{+-2}a_lm the quadrature projections of gamma (gamma*) on _{+-2}Y_lm; in
  terms of the ring Fourier coefficients F1, F2 of gamma_1, gamma_2:
  E_lm = (w / N_l) sum_r [A F1 - i B F2],  B_lm = (w / N_l) sum_r [A F2 + i B F1],
  so that gamma = eth^2 psi / 2 gives E_lm = N_l psi_lm / 2 and B_lm = 0;
* C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2 l + 1).
"""
import math

import torch

from . import healpix as hp
from . import sht

F64 = torch.float64
C128 = torch.complex128


def eb_analysis(g1, g2, nside, lmax):
    """E_lm, B_lm (packed like sht.analysis, l < 2 set to zero) of the
    spin-2 field gamma_1 + i gamma_2 given at RING pixel centres."""
    rt = hp.ring_table(nside)
    F1 = sht.ring_fourier(nside, g1, lmax)
    F2 = sht.ring_fourier(nside, g2, lmax)
    w = 4.0 * math.pi / hp.npix(nside)
    z = rt["z"][:, None].T
    s = rt["sin_theta"][:, None].T
    E = torch.zeros(sht.nalm(lmax), dtype=C128)
    B = torch.zeros(sht.nalm(lmax), dtype=C128)
    for m, lam, dl, _ in sht.dtheta_columns(lmax, rt["z"], rt["sin_theta"]):
        l = torch.arange(m, lmax + 1, dtype=F64)[:, None]
        cot = z / s
        A = -2.0 * cot * dl - (l * (l + 1.0) - 2.0 * m * m / (s * s)) * lam
        Bf = (2.0 * m / s) * (dl - cot * lam)
        lg = l[:, 0]
        norm = torch.where(lg >= 2, torch.sqrt(torch.clamp((lg + 2) * (lg + 1) * lg * (lg - 1), min=1.0)),
                           torch.ones_like(lg))
        e = (A.to(C128) @ F1[:, m] - 1j * (Bf.to(C128) @ F2[:, m])) * w / norm
        b = (A.to(C128) @ F2[:, m] + 1j * (Bf.to(C128) @ F1[:, m])) * w / norm
        keep = (lg >= 2).to(C128)
        i0 = sht.alm_index(lmax, m, m)
        E[i0:i0 + lmax - m + 1] = e * keep
        B[i0:i0 + lmax - m + 1] = b * keep
    return E, B


def cl(alm, lmax, alm2=None):
    """Angular (cross-)power spectrum C_l = (a_l0 b_l0* + 2 sum_{m>0} Re a_lm b_lm*) / (2l+1)."""
    if alm2 is None:
        alm2 = alm
    out = torch.zeros(lmax + 1, dtype=F64)
    for m in range(lmax + 1):
        i0 = sht.alm_index(lmax, m, m)
        prod = (alm[i0:i0 + lmax - m + 1] * alm2[i0:i0 + lmax - m + 1].conj()).real
        out[m:] += prod * (1.0 if m == 0 else 2.0)
    return out / (2.0 * torch.arange(lmax + 1, dtype=F64) + 1.0)


def spectra_from_A(A, nside, lmax):
    """kappa, E, B and omega spectra from inverse magnification matrices
    A[Npix, 2, 2] on the RING pixel grid of the ray start positions
    (Eq. invmagmat, Sec. 5), each given in the tangent basis at its pixel
    centre (rays.image_basis carries a traced A there)."""
    kappa = 1.0 - 0.5 * (A[:, 0, 0] + A[:, 1, 1])
    g1 = -0.5 * (A[:, 0, 0] - A[:, 1, 1])
    g2 = -0.5 * (A[:, 0, 1] + A[:, 1, 0])
    om = 0.5 * (A[:, 0, 1] - A[:, 1, 0])
    E, B = eb_analysis(g1, g2, nside, lmax)
    k = sht.analysis(kappa, nside, lmax)
    w = sht.analysis(om, nside, lmax)
    return {"kappa": cl(k, lmax), "E": cl(E, lmax), "B": cl(B, lmax), "omega": cl(w, lmax)}
