"""Pins of the oracle's SHT+MG patch solver and finite-difference
derivatives (paper Sec. 3.2, Appendix A)."""
import math

import numpy as np
import pytest
import scipy.special as sp
import torch

from oracle import mg, sht

F64 = torch.float64


def ylm_re(l, m, th, ph):
    return torch.from_numpy(np.ascontiguousarray(sp.sph_harm_y(l, m, th.numpy(), ph.numpy()).real))


def manufactured(n, l=7, m=3, nb=4, bundles=(5, 77), coarsest=8):
    """Patches whose exact solution is Re Y_lm in the global frame."""
    R = mg.rotation(nb, torch.tensor(bundles))
    h = mg.patch_side(nb) / n
    ghosts = []
    for nl in mg.level_sizes(n, coarsest):
        v = mg.to_global(R, mg.patch_vectors(nl, h * (n // nl)))
        th, ph = mg.theta_phi(v)
        ghosts.append(2.0 * ylm_re(l, m, th, ph))
    exact = ghosts[0][:, 1:-1, 1:-1] / 2.0
    f = -l * (l + 1) * exact
    u = ghosts[0].clone()
    u[:, 1:-1, 1:-1] = 0.0
    return R, h, ghosts, exact, f, u


def test_discretisation_error_is_second_order():
    errs = []
    for n in (32, 64):
        R, h, ghosts, exact, f, u = manufactured(n)
        S = mg.PatchSolver(n, h, ghosts, nu1=2, nu2=2)
        S.solve(u, f, tol=1e-13, max_cycles=60)
        errs.append(float((u[:, 1:-1, 1:-1] - exact).abs().max()))
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_converged_vcycles_equal_direct_solve():
    n = 16
    R, h, ghosts, exact, f, u = manufactured(n)
    S = mg.PatchSolver(n, h, ghosts, nu1=2, nu2=1)
    S.solve(u, f, fixed_cycles=40)
    op = mg.Operator(n, h)
    # dense matrix of the same operator, boundary terms moved to the right side
    eye = torch.eye(n * n, dtype=F64).reshape(n * n, n, n)
    pad = torch.zeros((n * n, n + 2, n + 2), dtype=F64)
    pad[:, 1:-1, 1:-1] = eye
    Amat = op.apply(pad).reshape(n * n, n * n).T
    g = ghosts[0].clone()
    g[:, 1:-1, 1:-1] = 0.0
    rhs = (f - op.apply(g)).reshape(2, n * n)
    direct = torch.linalg.solve(Amat, rhs.T).T.reshape(2, n, n)
    assert torch.allclose(u[:, 1:-1, 1:-1], direct, atol=1e-12 * float(direct.abs().max()), rtol=0)


@pytest.mark.parametrize("nu2,bound", [(1, 0.3), (2, 0.16)])
def test_vcycle_contraction(nu2, bound):
    n = 128
    R, h, ghosts, exact, f, u = manufactured(n)
    S = mg.PatchSolver(n, h, ghosts, nu1=2, nu2=nu2)
    rr = []
    for _ in range(8):
        S.vcycle(0, u, f)
        rr.append(float(S.residual_ratio(u, f).max()))
    rates = [rr[i + 1] / rr[i] for i in range(3, 7)]
    assert max(rates) < bound, rates


def test_fd_weights_from_polynomial_exactness():
    """Each 5-point stencil row is the unique one exact for polynomials of
    degree <= 4 (Fornberg 1988), derived here by a Vandermonde solve."""
    for deriv, W in ((1, mg.D1), (2, mg.D2)):
        for row, x0 in ((0, 0), (1, 1), (2, 2)):
            x = np.arange(5) - x0
            V = np.vander(x, 5, increasing=True).T          # V[k, j] = x_j^k
            rhs = np.zeros(5)
            rhs[deriv] = math.factorial(deriv)
            w = np.linalg.solve(V, rhs)
            assert np.allclose(W[row].numpy(), w, atol=1e-13)


def test_fd_partials_fourth_order():
    errs = []
    for n in (32, 64):
        h = 0.5 / n
        th = math.pi / 2 + (torch.arange(n, dtype=F64) + 0.5 - n / 2) * h
        ph = (torch.arange(n, dtype=F64) + 0.5 - n / 2) * h
        T, P = torch.meshgrid(th, ph, indexing="ij")
        u = (torch.sin(3 * T) * torch.cos(2 * P))[None]
        d = mg.fd_partials(u, h)[0]
        ex = torch.stack([3 * torch.cos(3 * T) * torch.cos(2 * P), -2 * torch.sin(3 * T) * torch.sin(2 * P),
                          -9 * torch.sin(3 * T) * torch.cos(2 * P), -4 * torch.sin(3 * T) * torch.cos(2 * P),
                          -6 * torch.cos(3 * T) * torch.sin(2 * P)])
        errs.append((float((d - ex)[:, 2:-2, 2:-2].abs().max()), float((d - ex).abs().max())))
    # central stencils: 4th order; one-sided edge rows: the second-derivative
    # stencil at the edge point is 3rd order
    assert 12 < errs[0][0] / errs[1][0] < 20, errs
    assert 7 < errs[0][1] / errs[1][1] < 20, errs


def test_patch_derivatives_in_global_basis_match_sht():
    """FD derivatives of Re Y_lm on a patch, interpolated to points near the
    patch centre and rotated to the global basis, match the pure-SHT
    derivative synthesis of the same harmonic (Appendix A conventions)."""
    l, m, nb, n = 6, 2, 8, 256
    R = mg.rotation(nb, torch.tensor([123]))
    h = mg.patch_side(nb) / n
    v = mg.to_global(R, mg.patch_vectors(n, h))
    th, ph = mg.theta_phi(v)
    u = ylm_re(l, m, th, ph)[:, 1:-1, 1:-1]
    part = mg.fd_partials(u, h)
    g = torch.Generator().manual_seed(9)
    # random points within a quarter patch of the centre
    off = (torch.rand(50, 2, generator=g, dtype=F64) - 0.5) * (n * h / 4)
    tpp = math.pi / 2 + off[:, 0]
    ppp = off[:, 1]
    vp = torch.stack([torch.sin(tpp) * torch.cos(ppp), torch.sin(tpp) * torch.sin(ppp), torch.cos(tpp)], -1)
    nvec = torch.einsum("ji,mj->mi", R[0], vp)
    out = mg.derivs_at(part, R, h, torch.zeros(50, dtype=torch.long), nvec)
    # reference: exact derivatives from the symbolic-free SHT synthesis at those points
    thg, phg = mg.theta_phi(nvec)
    L = 8
    import sympy
    t, p = sympy.symbols("t p", real=True)
    y = sympy.Ynm(l, m, t, p).expand(func=True)
    fns = {k: sympy.lambdify((t, p), sympy.re(e), "numpy") for k, e in {
        "p_t": sympy.diff(y, t), "p_p": sympy.diff(y, p), "p_tt": sympy.diff(y, t, 2),
        "p_pp": sympy.diff(y, p, 2), "p_tp": sympy.diff(y, t, p)}.items()}
    ev = {k: torch.from_numpy(np.broadcast_to(f(thg.numpy(), phg.numpy()), thg.shape).copy()) for k, f in fns.items()}
    from oracle import geometry
    ref = geometry.lens_fields_from_partials(ev["p_t"], ev["p_p"], ev["p_tt"], ev["p_pp"], ev["p_tp"],
                                             torch.sin(thg), torch.cos(thg))
    for k in ("a_th", "a_ph", "u_tt", "u_pp", "u_tp"):
        scale = float(ref[k].abs().max()) + 1e-3
        assert float((out[k] - ref[k]).abs().max()) < 2e-4 * scale, k


@pytest.mark.parametrize("cycles", [1, 3])
def test_correction_form_gives_the_fas_iterates(cycles):
    """V-cycles on the correction e = u - u_SHT with zero Dirichlet data
    (solve_correction) give the same iterates as FAS V-cycles on u itself
    from the SHT starting guess with the SHT ghosts (PatchSolver.solve): the
    operator is linear, so the two differ only by rounding."""
    from oracle import binning, healpix as hp
    from workloads import synthetic
    nf, ns, lmax, nb, n = 32, 8, 16, 2, 32
    z, phi = synthetic.lognormal_particles(200_000, 7)
    kappa = binning.kappa_from_counts(binning.bin_counts(nf, z, phi), z.numel() / hp.npix(nf), 1.0)
    psi = sht.poisson_sht(binning.degrade_ring(kappa, nf, ns), ns, lmax, derivatives=False)["psi"]
    R, h, u0, f, ghosts = mg.setup_patches(kappa, nf, psi, ns, nb, torch.arange(12 * nb * nb), ncell=n)
    S = mg.PatchSolver(n, h, ghosts, nu1=2, nu2=2)
    u = u0.clone()
    S.solve(u, f, fixed_cycles=cycles)
    ue, k, _ = mg.solve_correction(u0, f, h, n, nu1=2, nu2=2, fixed_cycles=cycles)
    assert k == cycles
    scale = float(u[:, 1:-1, 1:-1].abs().max())
    assert float((ue - u[:, 1:-1, 1:-1]).abs().max()) < 1e-12 * scale
    # and the correction made a difference (the comparison is not vacuous)
    assert float((ue - u0[:, 1:-1, 1:-1]).abs().max()) > 1e-4 * scale


def test_tau_estimate_is_second_order():
    """tau = L_c R u - R L_f u of the exact solution (a truncation-error
    estimate of the second-order discretisation) falls by four when the
    cells halve, away from the patch edge; in the two coarse rows and columns
    at the edge it stays of order one (the ghost-cell extrapolation of the
    Dirichlet data is a first-order boundary closure, whose truncation error
    still gives a second-order solution error)."""
    rms = []
    edge = []
    for n in (32, 64, 128):
        R, h, ghosts, exact, f, u = manufactured(n)
        S = mg.PatchSolver(n, h, ghosts)
        ue = ghosts[0].clone()
        ue[:, 1:-1, 1:-1] = exact
        t = mg.tau_estimate(S, ue, ghosts[1])
        ti = t[:, 2:-2, 2:-2]
        rms.append(float(torch.sqrt((ti * ti).mean())))
        edge.append(float(t.abs().max()))
    for a, b in zip(rms, rms[1:]):
        assert 3.8 < a / b < 4.2, rms
    assert min(edge) > 0.5 * max(edge), edge


def test_tau_rule_stops_at_the_discretisation_error():
    """The paper's rule ||r|| < eps ||tau|| (eps = 0.1) leaves the solution
    within a few per cent of the discretisation error of the converged one,
    after fewer V-cycles than a 1e-10 relative residual needs."""
    n = 64
    R, h, ghosts, exact, f, u0 = manufactured(n)
    conv, kc, _ = mg.solve_correction(u0, f, h, n, tol=1e-12)
    tau_u, kt, ratio = mg.solve_correction(u0, f, h, n, stop="tau", eps=0.1, ghost_c=ghosts[1])
    e_conv = float((conv - exact).abs().max())
    e_tau = float((tau_u - exact).abs().max())
    assert ratio < 0.1 and 1 <= kt < kc
    assert e_tau < 1.05 * e_conv, (e_tau, e_conv, kt, kc)
    # a looser eps stops earlier and further from the converged solution
    loose, kl, _ = mg.solve_correction(u0, f, h, n, stop="tau", eps=10.0, ghost_c=ghosts[1])
    assert kl <= kt and float((loose - conv).abs().max()) >= float((tau_u - conv).abs().max())
