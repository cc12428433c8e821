"""FAS multigrid patch solver of the SHT+MG method (oracle; test infrastructure).

Sec. 3.2: for every ray bundle (a low-resolution NEST HEALPix cell) a local
coordinate system puts the bundle centre at (theta', phi') = (pi/2, 0); a
patch four times the bundle's size is cut into cells of equal spacing
Delta theta' = Delta phi'; the SHT potential gives the Dirichlet boundary
values and the starting guess (both by HEALPix linear interpolation); the
plane Poisson equation is relaxed with red-black Gauss-Seidel accelerated by
FAS multigrid, with strictly conservative (area-weighted) restriction and
injection instead of interpolation for prolongation next to the boundary.
Fourth-order finite differences on the finest level, with one-sided stencils
at the patch edge, give the derivatives (Sec. 3.2).

Readings where the paper is silent (it defers to Barros 1992):
* patch side = 4 sqrt(pi / 3) / N_b radians (four times the square root of
  the bundle area), N x N cell-centred cells, h = side / N,
  theta'_i = pi/2 + (i + 1/2 - N/2) h, phi'_j = (j + 1/2 - N/2) h;
* rotation R_b = R_y(pi/2 - theta_c) R_z(-phi_c) (no roll);
* operator (Lu)_ij = [s_{i+1/2}(u_{i+1,j} - u_ij) - s_{i-1/2}(u_ij - u_{i-1,j})] / (h^2 s_i)
  + (u_{i,j+1} - 2 u_ij + u_{i,j-1}) / (h^2 s_i^2), s = sin theta';
* Dirichlet values g = psi_SHT at the centres of the patch-edge faces of
  every level, imposed through ghost cells holding 2 g - u_adjacent (the
  boundary value sits on the edge at all levels, so coarse corrections vanish
  where the fine error does);
* the source f is kappa (fine map) interpolated at the cell centres;
* red ((i + j) even) then black; nu1 = 2, nu2 = 1; coarsest level 8 x 8
  solved exactly (dense solve);
* restriction of u and of the residual weighted by cell area
  (cos theta'_{i-1/2} - cos theta'_{i+1/2}); FAS coarse source
  f_c = R(f - L u) + L_c(R u);
* prolongation of the coarse correction: cell-centred bilinear
  (9/16, 3/16, 3/16, 1/16), injection for cells next to the ghost ring;
* the V-cycles iterate on the correction e = u - u_SHT to the SHT solution:
  L e = f - L u_SHT with zero Dirichlet values at every level, starting from
  e = 0.  For the linear operator this gives the same iterates as cycling on
  u itself from the SHT starting guess, but the residual is no longer the
  difference of terms of size |u| / h^2, which put a 1e-10 relative
  tolerance below the FP64 round-off floor;
* convergence: every patch receives the same number of V-cycles, the
  smallest for which max over patches of ||f - L u||_2 / ||f||_2 < tol.
"""
import math

import torch

from . import healpix as hp
from . import interp
from . import geometry

F64 = torch.float64


def patch_side(nside_bundle, factor=4):
    return factor * math.sqrt(math.pi / 3.0) / nside_bundle


def level_sizes(ncell, coarsest=8):
    sizes = [ncell]
    while sizes[-1] > coarsest:
        sizes.append(sizes[-1] // 2)
    return sizes


def centres_1d(n, h):
    """theta' offsets from pi/2 (and phi' values) of the n cell centres, with
    the two patch edges (-n h / 2, +n h / 2) at positions -1 and n."""
    k = torch.arange(-1, n + 1, dtype=F64)
    c = (k + 0.5 - n / 2.0) * h
    c[0] = -(n / 2.0) * h
    c[-1] = (n / 2.0) * h
    return c


def rotation(nside_bundle, bundles):
    """R_b [B, 3, 3] mapping global unit vectors to patch-frame vectors."""
    z, phi = hp.pix2ang_nest(nside_bundle, torch.as_tensor(bundles))
    s = torch.sqrt((1.0 - z) * (1.0 + z))
    cp, sp = torch.cos(phi), torch.sin(phi)
    zero = torch.zeros_like(z)
    rows = [torch.stack([s * cp, s * sp, z], -1),
            torch.stack([-sp, cp, zero], -1),
            torch.stack([-z * cp, -z * sp, s], -1)]
    return torch.stack(rows, -2)


def patch_vectors(n, h):
    """Patch-frame unit vectors [n+2, n+2, 3]: cell centres inside, centres
    of the edge faces on the ghost ring (corners: the patch corners)."""
    d = centres_1d(n, h)
    th = math.pi / 2 + d
    ph = d
    st, ct = torch.sin(th), torch.cos(th)
    x = st[:, None] * torch.cos(ph)[None, :]
    y = st[:, None] * torch.sin(ph)[None, :]
    zz = ct[:, None].expand(n + 2, n + 2)
    return torch.stack([x, y, zz], -1)


def to_global(R, v):
    """Global vectors [B, ..., 3] of patch-frame vectors v[..., 3] (shared by
    all patches) for rotations R[B, 3, 3]: n = R^T n'."""
    return torch.einsum("bji,...j->b...i", R, v)


def theta_phi(n):
    """Colatitude and longitude (in [0, 2 pi)) of unit vectors."""
    rho = torch.sqrt(n[..., 0] ** 2 + n[..., 1] ** 2)
    th = torch.atan2(rho, n[..., 2])
    ph = torch.atan2(n[..., 1], n[..., 0])
    ph = torch.where(ph < 0, ph + 2 * math.pi, ph)
    return th, ph


class Operator:
    """Row coefficients of the discrete Laplace-Beltrami operator on one level."""

    def __init__(self, n, h):
        self.n, self.h = n, h
        i = torch.arange(n, dtype=F64)
        th = math.pi / 2 + (i + 0.5 - n / 2.0) * h
        s = torch.sin(th)
        sp = torch.sin(th + 0.5 * h)
        sm = torch.sin(th - 0.5 * h)
        self.aS = (sp / (h * h * s))[:, None]      # neighbour i + 1
        self.aN = (sm / (h * h * s))[:, None]      # neighbour i - 1
        self.b = (1.0 / (h * h * s * s))[:, None]  # neighbours j +- 1
        self.diag = self.aS + self.aN + 2.0 * self.b
        self.area = (torch.cos(th - 0.5 * h) - torch.cos(th + 0.5 * h))
        ii = torch.arange(n)
        self.red = ((ii[:, None] + ii[None, :]) % 2) == 0

        # Dirichlet value g on the patch edge: the ghost value 2 g - u_adjacent
        # (linear through the edge) moves the -u_adjacent part onto the diagonal
        diag = self.diag.expand(n, n).clone()
        diag[0, :] += self.aN[0, 0]
        diag[-1, :] += self.aS[-1, 0]
        diag[:, 0] += self.b[:, 0]
        diag[:, -1] += self.b[:, 0]
        self.diag_eff = diag

    def neighbours(self, u):
        return (self.aS * u[:, 2:, 1:-1] + self.aN * u[:, :-2, 1:-1]
                + self.b * (u[:, 1:-1, 2:] + u[:, 1:-1, :-2]))

    def apply(self, u):
        """(L u) on the interior of u[B, n+2, n+2] whose ghost ring holds 2 g."""
        return self.neighbours(u) - self.diag_eff * u[:, 1:-1, 1:-1]

    def smooth(self, u, f):
        """One red-black Gauss-Seidel sweep, red first, in place."""
        for colour in (self.red, ~self.red):
            new = (self.neighbours(u) - f) / self.diag_eff
            u[:, 1:-1, 1:-1] = torch.where(colour, new, u[:, 1:-1, 1:-1])

    def restrict(self, v):
        """Area-weighted 2x2 average of interior values v[B, n, n]."""
        a = self.area[None, :, None]
        num = (a * v).reshape(v.shape[0], self.n // 2, 2, self.n // 2, 2).sum((2, 4))
        den = 2.0 * (self.area[0::2] + self.area[1::2])[None, :, None]
        return num / den


def prolong(ec, n):
    """Fine-level correction [B, n, n] from a coarse correction ec[B, n/2, n/2]:
    cell-centred bilinear, injection next to the ghost ring."""
    B = ec.shape[0]
    i = torch.arange(n)
    I = i // 2
    di = torch.where(i % 2 == 0, -1, 1)
    Ii = (I + di).clamp(0, n // 2 - 1)
    c00 = ec[:, I][:, :, I]
    c10 = ec[:, Ii][:, :, I]
    c01 = ec[:, I][:, :, Ii]
    c11 = ec[:, Ii][:, :, Ii]
    bil = (9.0 * c00 + 3.0 * c10 + 3.0 * c01 + c11) / 16.0
    edge = (i == 0) | (i == n - 1)
    inj = edge[:, None] | edge[None, :]
    return torch.where(inj, c00, bil)


class PatchSolver:
    """FAS V-cycles on a batch of bundle patches with fixed Dirichlet ghosts."""

    def __init__(self, ncell, h, ghosts, nu1=2, nu2=1, coarsest=8):
        self.sizes = level_sizes(ncell, coarsest)
        self.ops = [Operator(n, h * (ncell // n)) for n in self.sizes]
        self.ghosts = ghosts          # per level: [B, n+2, n+2], ghost ring holds 2 g
        self.nu1, self.nu2 = nu1, nu2
        nc = self.sizes[-1]
        # dense operator of the coarsest level (interior unknowns, zero ghosts)
        op = self.ops[-1]
        eye = torch.eye(nc * nc, dtype=F64).reshape(nc * nc, nc, nc)
        pad = torch.zeros((nc * nc, nc + 2, nc + 2), dtype=F64)
        pad[:, 1:-1, 1:-1] = eye
        self.coarse_matrix = op.apply(pad).reshape(nc * nc, nc * nc).T

    def _coarse_solve(self, u, f):
        op = self.ops[-1]
        nc = op.n
        g = u.clone()
        g[:, 1:-1, 1:-1] = 0.0
        rhs = (f - op.apply(g)).reshape(u.shape[0], nc * nc)
        sol = torch.linalg.solve(self.coarse_matrix, rhs.T).T
        u[:, 1:-1, 1:-1] = sol.reshape(u.shape[0], nc, nc)

    def vcycle(self, lev, u, f):
        op = self.ops[lev]
        if lev == len(self.ops) - 1:
            self._coarse_solve(u, f)
            return
        for _ in range(self.nu1):
            op.smooth(u, f)
        r = f - op.apply(u)
        uc = self.ghosts[lev + 1].clone()
        uc[:, 1:-1, 1:-1] = op.restrict(u[:, 1:-1, 1:-1])
        fc = op.restrict(r) + self.ops[lev + 1].apply(uc)
        uc0 = uc[:, 1:-1, 1:-1].clone()
        self.vcycle(lev + 1, uc, fc)
        u[:, 1:-1, 1:-1] += prolong(uc[:, 1:-1, 1:-1] - uc0, op.n)
        for _ in range(self.nu2):
            op.smooth(u, f)

    def residual_ratio(self, u, f):
        r = f - self.ops[0].apply(u)
        rn = torch.sqrt((r * r).sum((1, 2)))
        fn = torch.sqrt((f * f).sum((1, 2)))
        return rn / torch.where(fn > 0, fn, 1.0)

    def solve(self, u, f, tol=1e-10, max_cycles=50, fixed_cycles=None):
        """Run V-cycles in place; returns (cycles run, max residual ratio)."""
        if fixed_cycles is not None:
            for _ in range(fixed_cycles):
                self.vcycle(0, u, f)
            return fixed_cycles, float(self.residual_ratio(u, f).max())
        k = 0
        rr = float(self.residual_ratio(u, f).max())
        while rr >= tol and k < max_cycles:
            self.vcycle(0, u, f)
            k += 1
            rr = float(self.residual_ratio(u, f).max())
        return k, rr


def setup_patches(kappa_fine, nside_fine, psi_sht, nside_sht, nside_bundle, bundles,
                  ncell=256, factor=4, coarsest=8):
    """Source, starting guess and per-level ghost rings (2 psi_SHT at the edge
    faces) for the given bundles.
    Returns (R, h, u0 [B, N+2, N+2], f [B, N, N], ghosts per level)."""
    bundles = torch.as_tensor(bundles)
    R = rotation(nside_bundle, bundles)
    side = patch_side(nside_bundle, factor)
    h = side / ncell
    ghosts = []
    u0 = f = None
    for n in level_sizes(ncell, coarsest):
        hl = h * (ncell // n)
        v = to_global(R, patch_vectors(n, hl))
        th, ph = theta_phi(v)
        psi = interp.interpolate(nside_sht, psi_sht, th, ph)
        ghosts.append(2.0 * psi)
        if n == ncell:
            u0 = 2.0 * psi
            u0[:, 1:-1, 1:-1] = psi[:, 1:-1, 1:-1]
            f = interp.interpolate(nside_fine, kappa_fine, th[:, 1:-1, 1:-1], ph[:, 1:-1, 1:-1])
    return R, h, u0, f, ghosts


# fourth-order first / second derivative stencils on 5 points (Fornberg
# weights x 12); rows: evaluation at offset 0, 1 (one-sided) and 2 (central)
D1 = torch.tensor([[-25., 48., -36., 16., -3.],
                   [-3., -10., 18., -6., 1.],
                   [1., -8., 0., 8., -1.]], dtype=F64) / 12.0
D2 = torch.tensor([[35., -104., 114., -56., 11.],
                   [11., -20., 6., 4., -1.],
                   [-1., 16., -30., 16., -1.]], dtype=F64) / 12.0


def _deriv_axis(u, h, W, axis, sign):
    """Apply 5-point stencils along `axis` of interior-only data u[B, n, n]."""
    n = u.shape[axis]
    u = u.movedim(axis, -1)
    out = torch.empty_like(u)
    # central cells
    c = W[2]
    out[..., 2:n - 2] = sum(c[k] * u[..., k:n - 4 + k] for k in range(5))
    for off in (0, 1):
        w = W[off]
        out[..., off] = sum(w[k] * u[..., k] for k in range(5))
        out[..., n - 1 - off] = sign * sum(w[k] * u[..., n - 1 - k] for k in range(5))
    return out.movedim(-1, axis) / h


def fd_partials(u, h):
    """psi_t', psi_p', psi_t't', psi_p'p', psi_t'p' at the cell centres of the
    finest level from interior values u[B, N, N] (rows theta', cols phi')."""
    pt = _deriv_axis(u, h, D1, 1, -1.0)
    pp = _deriv_axis(u, h, D1, 2, -1.0)
    ptt = _deriv_axis(u, h * h, D2, 1, 1.0)
    ppp = _deriv_axis(u, h * h, D2, 2, 1.0)
    ptp = _deriv_axis(pp, h, D1, 1, -1.0)
    return torch.stack([pt, pp, ptt, ppp, ptp], 1)   # [B, 5, N, N]


def derivs_at(partials, R, h, b_index, nvec):
    """alpha (theta, phi) and U (tt, pp, tp) in the global (theta-hat, phi-hat)
    basis at unit vectors nvec[M, 3], each looked up in the patch b_index[M]
    (an index into the batch): bilinear interpolation of the patch partials
    in cell coordinates, Appendix A formulas in the patch basis, then the
    rotation of alpha (vector) and U (rank-2 tensor) to the global basis."""
    n = partials.shape[-1]
    Rm = R[b_index]
    v = torch.einsum("mij,mj->mi", Rm, nvec)                 # patch-frame vector
    thp, php = theta_phi(v)
    php = torch.where(php > math.pi, php - 2 * math.pi, php)
    x = (thp - math.pi / 2) / h + n / 2.0 - 0.5
    y = php / h + n / 2.0 - 0.5
    i0 = torch.floor(x).clamp(0, n - 2)
    j0 = torch.floor(y).clamp(0, n - 2)
    fx = x - i0
    fy = y - j0
    i0 = i0.long()
    j0 = j0.long()
    def at(ii, jj):
        return partials[b_index, :, ii, jj]                  # [M, 5]

    val = ((1 - fx)[:, None] * (1 - fy)[:, None] * at(i0, j0) + fx[:, None] * (1 - fy)[:, None] * at(i0 + 1, j0)
           + (1 - fx)[:, None] * fy[:, None] * at(i0, j0 + 1) + fx[:, None] * fy[:, None] * at(i0 + 1, j0 + 1))
    s = torch.sin(thp)
    c = torch.cos(thp)
    lf = geometry.lens_fields_from_partials(val[:, 0], val[:, 1], val[:, 2], val[:, 3], val[:, 4], s, c)
    # patch basis at the point, in global coordinates
    tp_ = torch.stack([c * torch.cos(php), c * torch.sin(php), -s], -1)
    pp_ = torch.stack([-torch.sin(php), torch.cos(php), torch.zeros_like(s)], -1)
    ebp = (torch.einsum("mji,mj->mi", Rm, tp_), torch.einsum("mji,mj->mi", Rm, pp_))
    Q = geometry.frame_rotation(geometry.basis(nvec), ebp)
    a = torch.stack([lf["a_th"], lf["a_ph"]], -1)
    ag = torch.einsum("mab,mb->ma", Q, a)
    U = torch.stack([torch.stack([lf["u_tt"], lf["u_tp"]], -1), torch.stack([lf["u_tp"], lf["u_pp"]], -1)], -2)
    Ug = Q @ U @ Q.transpose(-1, -2)
    return {"a_th": ag[:, 0], "a_ph": ag[:, 1], "u_tt": Ug[:, 0, 0], "u_pp": Ug[:, 1, 1], "u_tp": Ug[:, 0, 1]}


def home_bundle(nside_fine, nside_bundle, nest_pix):
    """Bundle (NEST pixel at Nside_bundle) of a NEST pixel at Nside_fine: a
    right shift by 2 log2(Nf / N_b) bits (Sec. 3.1)."""
    shift = 2 * (hp.nside_order(nside_fine) - hp.nside_order(nside_bundle))
    return torch.as_tensor(nest_pix) >> shift


def tau_estimate(S, u, ghost_c):
    """The fine-grid truncation-error estimate of the full approximation
    scheme (Sec. 3.2, stopping rule): tau = L_c R u - R L_f u, u[B, N+2, N+2]
    with 2 g on its ghost ring, ghost_c[B, N/2+2, N/2+2] the coarse level's
    ghost ring (2 g at the coarse edge faces).  Returns tau [B, N/2, N/2]."""
    op, opc = S.ops[0], S.ops[1]
    uc = ghost_c.clone()
    uc[:, 1:-1, 1:-1] = op.restrict(u[:, 1:-1, 1:-1])
    return opc.apply(uc) - op.restrict(op.apply(u))


def solve_correction(base, f, h, ncell, nu1=2, nu2=2, tol=1e-10, max_cycles=60, fixed_cycles=None, coarsest=8,
                     stop="residual", eps=0.1, ghost_c=None):
    """V-cycles on the correction e = u - base: L e = f - L base with zero
    Dirichlet values on every level, from e = 0.  base[B, N+2, N+2] holds the
    starting guess inside and 2 g on its ghost ring.  Stopping rules (every
    patch receives the same number of V-cycles):
    * "residual": max over patches of ||f - L u||_2 / ||f||_2 < tol, with
      the original source f;
    * "tau" (the paper's rule, Sec. 3.2, after Press et al. Sec. 20.6):
      max over patches of rms(f - L u) / rms(tau) < eps, rms the root mean
      square over the patch's fine (residual) or coarse (tau) cells, tau the
      estimate of tau_estimate on u = base + e (ghost_c: the coarse level's
      ghost ring, 2 g).
    Returns (u interior, cycles, ratio of the chosen rule)."""
    B = f.shape[0]
    zeros = [torch.zeros((B, n + 2, n + 2), dtype=F64) for n in level_sizes(ncell, coarsest)]
    S = PatchSolver(ncell, h, zeros, nu1=nu1, nu2=nu2, coarsest=coarsest)
    fd = f - S.ops[0].apply(base)
    e = zeros[0].clone()
    fn = torch.sqrt((f * f).sum((1, 2)))
    fn = torch.where(fn > 0, fn, 1.0)

    def ratio():
        r = fd - S.ops[0].apply(e)
        if stop == "tau":
            u = base + e
            t = tau_estimate(S, u, ghost_c)
            rr = torch.sqrt((r * r).mean((1, 2)))
            tt = torch.sqrt((t * t).mean((1, 2)))
            return float((rr / torch.where(tt > 0, tt, 1e-300)).max().detach())
        return float((torch.sqrt((r * r).sum((1, 2))) / fn).max().detach())
    limit = eps if stop == "tau" else tol
    k = 0
    rr = ratio()
    if fixed_cycles is not None:
        for _ in range(fixed_cycles):
            S.vcycle(0, e, fd)
        k, rr = fixed_cycles, ratio()
    else:
        while rr >= limit and k < max_cycles:
            S.vcycle(0, e, fd)
            k += 1
            rr = ratio()
    return base[:, 1:-1, 1:-1] + e[:, 1:-1, 1:-1], k, rr


def solve_plane(kappa_fine, nside_fine, nside_sht, lmax, nside_bundle, ncell=256, nu1=2, nu2=2,
                tol=1e-10, max_cycles=60, fixed_cycles=None, bundles=None, coarsest=8, psi_sht=None,
                stop="residual", eps=0.1):
    """The whole SHT+MG plane solve of Sec. 3.2 for the given bundles (all by
    default): degrade kappa to the SHT grid, SHT Poisson solve, patch set-up,
    V-cycles on the correction to the SHT solution.  A caller that already
    holds the SHT potential of this kappa (psi_sht, RING map at nside_sht)
    may pass it to skip the SHT step.  Returns dict with R, h, u (interior
    [B, N, N]), partials, bundles, cycles, residual and psi_sht."""
    from . import binning, sht
    if bundles is None:
        bundles = torch.arange(12 * nside_bundle * nside_bundle)
    bundles = torch.as_tensor(bundles)
    if psi_sht is None:
        ks = binning.degrade_ring(kappa_fine, nside_fine, nside_sht)
        psi_sht = sht.poisson_sht(ks, nside_sht, lmax, derivatives=False)["psi"]
    R, h, u, f, ghosts = setup_patches(kappa_fine, nside_fine, psi_sht, nside_sht, nside_bundle, bundles,
                                       ncell=ncell, coarsest=coarsest)
    ui, cycles, rr = solve_correction(u, f, h, ncell, nu1=nu1, nu2=nu2, tol=tol, max_cycles=max_cycles,
                                      fixed_cycles=fixed_cycles, coarsest=coarsest, stop=stop, eps=eps,
                                      ghost_c=ghosts[1])
    return {"R": R, "h": h, "u": ui, "partials": fd_partials(ui, h), "bundles": bundles, "cycles": cycles,
            "residual": rr, "psi_sht": psi_sht}


def fields_at(sol, nside_bundle, nvec, home):
    """Lens fields at unit vectors nvec[M, 3] whose home bundles are home[M]
    (NEST indices at nside_bundle) from a solve_plane result."""
    lookup = {int(b): k for k, b in enumerate(sol["bundles"].tolist())}
    idx = torch.tensor([lookup[int(b)] for b in home.tolist()], dtype=torch.long)
    return derivs_at(sol["partials"], sol["R"], sol["h"], idx, nvec)


def partial_sky_kappa(density, covered, scale):
    """Plane source of a light cone that covers only part of the sphere
    (Sec. 3.4): outside the covered pixels (RING boolean mask) the matter is
    at the mean density of the universe, so kappa = 0 there; inside,
    kappa_p = scale * (density_p / nbar - 1) (Eq. lenspoisson) with density
    the particle number per pixel (binned counts or a smoothed map) and nbar
    the light cone's own mean over its covered pixels.  With that mean the
    source integrates to zero over the sphere, the condition for a solution
    of the Poisson equation on the closed sphere: the SHT step drops l = 0,
    and the MG patches, which see the source itself, then solve the same
    problem."""
    d = torch.as_tensor(density).to(F64)
    covered = torch.as_tensor(covered, dtype=torch.bool)
    nbar = d[covered].sum() / covered.sum()
    return torch.where(covered, scale * (d / nbar - 1.0), torch.zeros_like(d))


def domain_bundles(nside_bundle, centre, radius):
    """NEST bundles of a circular domain of interest: those whose centres lie
    within `radius` of the unit vector `centre`.  Partial-sky ray tracing
    (Sec. 3.4) runs the SHT over the full sky and MG only on these bundles:
    solve_plane(..., bundles=domain_bundles(...))."""
    z, phi = hp.pix2ang_nest(nside_bundle, torch.arange(12 * nside_bundle * nside_bundle))
    c = torch.as_tensor(centre, dtype=torch.float64)
    d = torch.arccos((hp.vec_from_zphi(z, phi) @ c).clamp(-1.0, 1.0))
    return torch.nonzero(d < radius).flatten()
