"""Multiple-plane ray recursion on the sphere (oracle; test infrastructure).

Sec. 2.2 of the paper propagates each ray from lens plane n to n + 1 by
* rotating its propagation direction about n^(n) x alpha^(n) by |alpha^(n)|
  (Eq. betaprop, the method of Teyssier et al. 2009 App. A),
* advancing its Cartesian position along the new direction to the sphere of
  radius chi_{n+1}, with lambda > 0 solving
  lambda^2 + 2 lambda (x . beta) + chi_n^2 - chi_{n+1}^2 = 0 (Eq. posprop),
* updating the inverse magnification matrix with the two-plane recursion of
  Hilbert et al. 2009 (Eq. Atraj), A^(0) = A^(-1) = I,
* and parallel-transporting A^(n+1) and A^(n) along the geodesic from the
  old to the new angular position (Appendix B: rotate the old tangent basis
  with the 3D rotation that carries the old position onto the new one, then
  express the tensor in the new basis).
Appendix D: a galaxy between planes n and n + 1 takes
A_g = (1 - t) A_n + t A_{n+1}, t = (D_{n+1} / D_g)(D_{n,g} / D_{n,n+1}) (Eq. gatraj).

Readings: flat geometry, D_a = chi_a and D_ab = chi_b - chi_a; chi_{-1} = 0
(irrelevant because A^(-1) = A^(0)); alpha = -grad psi as in Appendix A, so
the rotation bends back-traced rays toward overdensities.  Everything is
written in differentiable torch FP64 ops.
"""
import torch

from . import geometry

F64 = torch.float64


def init_rays(n0, chi0):
    """Rays starting at unit vectors n0[M, 3] on the first plane (Eq. posprop,
    Eq. betaprop and Eq. Atraj initial conditions)."""
    M = n0.shape[0]
    eye = torch.eye(2, dtype=F64).expand(M, 2, 2).clone()
    return {"x": chi0 * n0, "beta": n0.clone(), "A": eye, "Ap": eye.clone()}


def recursion_coeffs(chi_prev, chi_n, chi_next):
    """(c, d): A^(n+1) = (1 - c) A^(n-1) + c A^(n) - d U^(n) A^(n) (Eq. Atraj)."""
    c = (chi_n / chi_next) * ((chi_next - chi_prev) / (chi_n - chi_prev))
    d = (chi_next - chi_n) / chi_next
    return c, d


def transport(A, n_old, n_new):
    """Parallel transport of tangent tensors A[M, 2, 2], given in the
    (theta-hat, phi-hat) basis at n_old, to the basis at n_new (Appendix B)."""
    cr = torch.cross(n_old, n_new, dim=-1)
    s = torch.linalg.vector_norm(cr, dim=-1)
    c = (n_old * n_new).sum(-1)
    moved = s > 0
    k = cr / torch.where(moved, s, 1.0)[..., None]
    t_old, p_old = geometry.basis(n_old)
    t_rot = geometry.rotate_rodrigues(t_old, k, c, s)
    p_rot = geometry.rotate_rodrigues(p_old, k, c, s)
    t_rot = torch.where(moved[..., None], t_rot, t_old)
    p_rot = torch.where(moved[..., None], p_rot, p_old)
    Q = geometry.frame_rotation(geometry.basis(n_new), (t_rot, p_rot))
    return Q @ A @ Q.transpose(-1, -2)


def step(state, lens, chi_prev, chi_n, chi_next):
    """One plane: lens(n[M, 3]) -> dict a_th, a_ph, u_tt, u_pp, u_tp in the
    global basis at n.  Returns the new state (Eq. betaprop, posprop, Atraj,
    Appendix B)."""
    x, beta, A, Ap = state["x"], state["beta"], state["A"], state["Ap"]
    n = x / torch.linalg.vector_norm(x, dim=-1, keepdim=True)
    L = lens(n)
    U = torch.stack([torch.stack([L["u_tt"], L["u_tp"]], -1),
                     torch.stack([L["u_tp"], L["u_pp"]], -1)], -2)
    c, d = recursion_coeffs(chi_prev, chi_n, chi_next)
    A_next = (1.0 - c) * Ap + c * A - d * (U @ A)
    th, ph = geometry.basis(n)
    avec = L["a_th"][..., None] * th + L["a_ph"][..., None] * ph
    amag = torch.linalg.vector_norm(avec, dim=-1)
    nz = amag > 0
    k = torch.cross(n, avec, dim=-1) / torch.where(nz, amag, 1.0)[..., None]
    beta_rot = geometry.rotate_rodrigues(beta, k, torch.cos(amag), torch.sin(amag))
    beta_new = torch.where(nz[..., None], beta_rot, beta)
    xb = (x * beta_new).sum(-1)
    dchi2 = chi_next * chi_next - chi_n * chi_n
    lam = dchi2 / (xb + torch.sqrt(xb * xb + dchi2))
    x_new = x + lam[..., None] * beta_new
    n_new = x_new / torch.linalg.vector_norm(x_new, dim=-1, keepdim=True)
    return {"x": x_new, "beta": beta_new,
            "A": transport(A_next, n, n_new), "Ap": transport(A, n, n_new)}


def image_basis(A, n_source, n_image):
    """A[M, 2, 2] carried from the tangent basis at the rays' positions on the
    source sphere to the basis at their image positions (the directions in
    which they were shot), by the transport of Appendix B along the geodesic
    between the two.  The recursion keeps A in the basis at the ray's current
    position; maps of the final shear over the image-plane grid (Sec. 5) are
    taken in the basis at each image position, the frame in which the
    relations C_l^E ~ C_l^kappa and C_l^B ~ C_l^omega hold."""
    return transport(A, n_source, n_image)


def trace(n0, chi, lenses, checkpoints=None):
    """Trace rays through planes 0 .. N-1 at distances chi[0 .. N-1] to the
    source sphere chi[N]; lenses[m](n) gives the plane-m lens fields.
    Returns the final state (and fills `checkpoints` with the state entering
    every plane, if a list is given)."""
    st = init_rays(n0, chi[0])
    N = len(lenses)
    for m in range(N):
        if checkpoints is not None:
            checkpoints.append(st)
        chi_prev = chi[m - 1] if m > 0 else 0.0
        st = step(st, lenses[m], chi_prev, chi[m], chi[m + 1])
    return st


def galaxy_interp(A_n, A_n1, chi_n, chi_n1, chi_g):
    """A_g = (1 - t) A_n + t A_{n+1}, t = (D_{n+1}/D_g)(D_{n,g}/D_{n,n+1})
    (Appendix D, Eq. gatraj); A_n and A_{n+1} in the same tangent basis."""
    t = (chi_n1 / chi_g) * ((chi_g - chi_n) / (chi_n1 - chi_n))
    return (1.0 - t)[..., None, None] * A_n + t[..., None, None] * A_n1


def decompose(A):
    """kappa, gamma_1, gamma_2, omega of A (Eq. invmagmat)."""
    kappa = 1.0 - 0.5 * (A[..., 0, 0] + A[..., 1, 1])
    g1 = -0.5 * (A[..., 0, 0] - A[..., 1, 1])
    g2 = -0.5 * (A[..., 0, 1] + A[..., 1, 0])
    om = 0.5 * (A[..., 0, 1] - A[..., 1, 0])
    return kappa, g1, g2, om


def map_lens(nside, fields):
    """Lens function for fields given at RING pixel centres (pure-SHT path):
    alpha is carried as a tangent 3-vector and U as a 3x3 tangent tensor,
    interpolated ring-bilinearly and projected on the basis at the ray."""
    from . import healpix as hp
    from . import interp
    pv = hp.pix2vec_ring(nside, torch.arange(hp.npix(nside)))
    tp, pp = geometry.basis(pv)
    a3 = fields["a_th"][:, None] * tp + fields["a_ph"][:, None] * pp
    U3 = (fields["u_tt"][:, None, None] * tp[:, :, None] * tp[:, None, :]
          + fields["u_pp"][:, None, None] * pp[:, :, None] * pp[:, None, :]
          + fields["u_tp"][:, None, None] * (tp[:, :, None] * pp[:, None, :] + pp[:, :, None] * tp[:, None, :]))

    def lens(n):
        rho = torch.sqrt(n[:, 0] ** 2 + n[:, 1] ** 2)
        th = torch.atan2(rho, n[:, 2])
        ph = torch.atan2(n[:, 1], n[:, 0])
        ph = torch.where(ph < 0, ph + 2 * torch.pi, ph)
        idx, w = interp.interp_weights(nside, th, ph)
        a = (a3[idx] * w[..., None]).sum(1)
        U = (U3[idx] * w[..., None, None]).sum(1)
        t, p = geometry.basis(n)
        return {"a_th": (a * t).sum(-1), "a_ph": (a * p).sum(-1),
                "u_tt": torch.einsum("mi,mij,mj->m", t, U, t),
                "u_pp": torch.einsum("mi,mij,mj->m", p, U, p),
                "u_tp": torch.einsum("mi,mij,mj->m", t, U, p)}
    return lens


def galaxy_bins(chi, gchi):
    """Plane n of each galaxy: chi[n] <= chi_g < chi[n + 1], n = 0 .. N - 1
    (a galaxy on the last sphere belongs to plane N - 1); -1 in front of the
    first plane (no lensing)."""
    chi_t = torch.as_tensor(chi, dtype=F64)
    N = chi_t.numel() - 1
    b = torch.searchsorted(chi_t, gchi, right=True) - 1
    return torch.where(gchi < chi_t[0], torch.full_like(b, -1), b.clamp(max=N - 1))


def galaxy_shear(kappas, nside, lmax, chi, gz, gphi, gchi):
    """Shear (gamma_1, gamma_2)[2, M] of M galaxies at (gz, gphi) and comoving
    distance gchi: rays start at the galaxy directions on plane 0, each plane's
    lens fields come from the pure-SHT solve of kappas[n] (Sec. 3.2), the rays
    follow the plane recursion (Sec. 2.2, Appendix B) and each galaxy takes
    A_g between the two planes that bracket it (Appendix D, Eq. gatraj), its
    shear from Eq. invmagmat.  Differentiable with respect to kappas."""
    from . import healpix as hp
    from . import sht
    chi = [float(c) for c in chi]
    N = len(kappas)
    s = torch.sqrt((1 - gz) * (1 + gz))
    n0 = torch.stack([s * torch.cos(gphi), s * torch.sin(gphi), gz], -1)
    bins = galaxy_bins(chi, gchi)
    st = init_rays(n0, chi[0])
    g1 = torch.zeros(gz.shape, dtype=F64)
    g2 = torch.zeros(gz.shape, dtype=F64)
    for m in range(N):
        fields = sht.poisson_sht(kappas[m], nside, lmax)
        chi_prev = chi[m - 1] if m > 0 else 0.0
        st = step(st, map_lens(nside, fields), chi_prev, chi[m], chi[m + 1])
        sel = bins == m
        Ag = galaxy_interp(st["Ap"], st["A"], torch.full_like(gchi, chi[m]), torch.full_like(gchi, chi[m + 1]),
                           torch.where(sel, gchi, torch.full_like(gchi, chi[m + 1])))
        _, a1, a2, _ = decompose(Ag)
        g1 = g1 + torch.where(sel, a1, torch.zeros_like(a1))
        g2 = g2 + torch.where(sel, a2, torch.zeros_like(a2))
    del hp
    return torch.stack([g1, g2])


def galaxy_shear_mg(kappas, nside_fine, nside_sht, lmax, nside_bundle, ncell, chi, gz, gphi, gchi, cycles=20,
                    nu1=2, nu2=2):
    """galaxy_shear with the SHT+MG solver of Sec. 3.2 on every plane: the
    plane's potential from solve_plane (`cycles` V-cycles, enough to converge
    to rounding), each galaxy's ray looked up in the patch of the bundle that
    contains its starting direction (rays keep their bundle, Sec. 3.1) with
    the fourth-order finite differences and rotation of Appendix A.
    Differentiable with respect to kappas (torch autograd through the SHT,
    the interpolations, the V-cycles and the lookup)."""
    from . import healpix as hp
    from . import mg
    chi = [float(c) for c in chi]
    N = len(kappas)
    s = torch.sqrt((1 - gz) * (1 + gz))
    n0 = torch.stack([s * torch.cos(gphi), s * torch.sin(gphi), gz], -1)
    home = hp.ang2pix_nest(nside_bundle, gz, gphi)
    bins = galaxy_bins(chi, gchi)
    st = init_rays(n0, chi[0])
    g1 = torch.zeros(gz.shape, dtype=F64)
    g2 = torch.zeros(gz.shape, dtype=F64)
    for m in range(N):
        sol = mg.solve_plane(kappas[m], nside_fine, nside_sht, lmax, nside_bundle, ncell=ncell, nu1=nu1, nu2=nu2,
                             fixed_cycles=cycles)
        chi_prev = chi[m - 1] if m > 0 else 0.0
        st = step(st, lambda n, sol=sol: mg.fields_at(sol, nside_bundle, n, home), chi_prev, chi[m], chi[m + 1])
        sel = bins == m
        Ag = galaxy_interp(st["Ap"], st["A"], torch.full_like(gchi, chi[m]), torch.full_like(gchi, chi[m + 1]),
                           torch.where(sel, gchi, torch.full_like(gchi, chi[m + 1])))
        _, a1, a2, _ = decompose(Ag)
        g1 = g1 + torch.where(sel, a1, torch.zeros_like(a1))
        g2 = g2 + torch.where(sel, a2, torch.zeros_like(a2))
    return torch.stack([g1, g2])

