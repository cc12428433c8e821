"""Sphere differential geometry of Appendix A (oracle; test infrastructure).

Appendix A gives, for the metric ds^2 = dtheta^2 + sin^2 theta dphi^2, the
orthonormal-basis components of the gradient and of the covariant Hessian of
a scalar Psi:
    grad_theta = d_t Psi,              grad_phi = d_p Psi / sin t,
    U_tt = d_tt Psi,
    U_pp = d_pp Psi / sin^2 t + cot t d_t Psi,
    U_tp = d_tp Psi / sin t - cos t d_p Psi / sin^2 t,
and the lensing conventions alpha = -grad Psi,
gamma_1 = -(U_pp - U_tt) / 2, gamma_2 = U_tp, kappa = U_tt + U_pp.
"""
import torch

F64 = torch.float64


def lens_fields_from_partials(p_t, p_p, p_tt, p_pp, p_tp, s, c):
    """alpha (theta, phi) and U (tt, pp, tp) from coordinate partials of
    psi at points with sin theta = s, cos theta = c (Appendix A)."""
    return {
        "a_th": -p_t,
        "a_ph": -p_p / s,
        "u_tt": p_tt,
        "u_pp": p_pp / (s * s) + (c / s) * p_t,
        "u_tp": p_tp / s - c * p_p / (s * s),
    }


def kappa_gamma(u_tt, u_pp, u_tp):
    """kappa (trace of U; twice the standard convergence, Eq. lenspoisson),
    gamma_1, gamma_2 (Appendix A)."""
    return u_tt + u_pp, 0.5 * (u_tt - u_pp), u_tp


def basis(n):
    """Orthonormal tangent basis (theta-hat, phi-hat) at unit vectors n[..., 3];
    on a pole, where it is undefined, its limit along phi = 0."""
    x, y, z = n[..., 0], n[..., 1], n[..., 2]
    rho = torch.sqrt(x * x + y * y)
    pole = rho == 0
    r = torch.where(pole, torch.ones_like(rho), rho)
    th = torch.stack([z * x / r, z * y / r, -rho], -1)
    ph = torch.stack([-y / r, x / r, torch.zeros_like(x)], -1)
    zero = torch.zeros_like(x)
    th_pole = torch.stack([torch.where(z >= 0, torch.ones_like(z), -torch.ones_like(z)), zero, zero], -1)
    ph_pole = torch.stack([zero, torch.ones_like(x), zero], -1)
    th = torch.where(pole[..., None], th_pole, th)
    ph = torch.where(pole[..., None], ph_pole, ph)
    return th, ph


def zphi_of(n):
    """(z, phi) of unit vectors, phi in [0, 2 pi)."""
    phi = torch.atan2(n[..., 1], n[..., 0])
    phi = torch.where(phi < 0, phi + 2 * torch.pi, phi)
    return n[..., 2], phi


def rotate_rodrigues(v, k, cos_w, sin_w):
    """Rotate v counter-clockwise about the unit axis k by the angle whose
    cosine and sine are given (the rotation R(k, w) of Eq. betaprop)."""
    kxv = torch.cross(k, v, dim=-1)
    kdv = (k * v).sum(-1, keepdim=True)
    return v * cos_w[..., None] + kxv * sin_w[..., None] + k * kdv * (1.0 - cos_w[..., None])


def frame_rotation(e_to, e_from):
    """Q[a, b] = e_to[a] . e_from[b] for two orthonormal tangent bases at the
    same point; vector components map as v_to = Q v_from and rank-2 tensor
    components as T_to = Q T_from Q^T."""
    t_to, p_to = e_to
    t_fr, p_fr = e_from
    q00 = (t_to * t_fr).sum(-1)
    q01 = (t_to * p_fr).sum(-1)
    q10 = (p_to * t_fr).sum(-1)
    q11 = (p_to * p_fr).sum(-1)
    return torch.stack([torch.stack([q00, q01], -1), torch.stack([q10, q11], -1)], -2)
