"""Pins of the oracle's multiple-plane ray recursion (paper Sec. 2.2,
Appendix B, C, D)."""
import math

import torch

from oracle import geometry, rays

F64 = torch.float64


def _rand_unit(n, seed):
    g = torch.Generator().manual_seed(seed)
    v = torch.randn(n, 3, dtype=F64, generator=g)
    return v / torch.linalg.vector_norm(v, dim=-1, keepdim=True)


def _zero_lens(n):
    z = torch.zeros(n.shape[0], dtype=F64)
    return {"a_th": z, "a_ph": z, "u_tt": z, "u_pp": z, "u_tp": z}


def test_no_lensing_keeps_rays_straight():
    n0 = _rand_unit(100, 1)
    chi = [50.0 * (m + 0.5) for m in range(6)] + [300.0]
    st = rays.trace(n0, chi, [_zero_lens] * 6)
    assert torch.allclose(st["x"], 300.0 * n0, atol=1e-12)
    assert torch.allclose(st["A"], torch.eye(2, dtype=F64).expand(100, 2, 2), atol=1e-14)


def test_distance_identities():
    """D_ac = (D_a D_bc + D_ab D_c) / D_b and D_ad = (D_ac D_bd - D_ab D_cd) / D_bc
    (Appendix C and D) for flat r(chi) = chi."""
    g = torch.Generator().manual_seed(2)
    a, b, c, d = (100 + 3000 * torch.rand(4, 1000, dtype=F64, generator=g))
    D = lambda x, y: y - x
    assert torch.allclose(D(a, c), (a * D(b, c) + D(a, b) * c) / b, rtol=1e-12, atol=1e-9)
    assert torch.allclose(D(a, d), (D(a, c) * D(b, d) - D(a, b) * D(c, d)) / D(b, c), rtol=1e-9, atol=1e-7)


def test_recursion_equals_explicit_sum():
    """With rays held radial (no deflection), Eq. Atraj reproduces
    A_k = I - sum_{i<k} (D_ik / D_k) U_i A_i (Eq. Atrajold, Appendix C)."""
    M, N = 20, 8
    n0 = _rand_unit(M, 3)
    g = torch.Generator().manual_seed(4)
    Us = []
    for _ in range(N):
        u = 0.05 * torch.randn(M, 3, dtype=F64, generator=g)
        Us.append(u)
    chi = [70.0 * (m + 0.5) for m in range(N)] + [70.0 * N]

    def lens_of(u):
        def lens(n):
            z = torch.zeros(n.shape[0], dtype=F64)
            return {"a_th": z, "a_ph": z, "u_tt": u[:, 0], "u_pp": u[:, 1], "u_tp": u[:, 2]}
        return lens

    st = rays.trace(n0, chi, [lens_of(u) for u in Us])
    I = torch.eye(2, dtype=F64).expand(M, 2, 2)
    A = []
    for k in range(N + 1):
        acc = I.clone()
        for i in range(k):
            U = torch.stack([torch.stack([Us[i][:, 0], Us[i][:, 2]], -1),
                             torch.stack([Us[i][:, 2], Us[i][:, 1]], -1)], -2)
            acc = acc - ((chi[k] - chi[i]) / chi[k]) * (U @ A[i])
        A.append(acc)
    assert torch.allclose(st["A"], A[N], atol=1e-13)
    assert torch.allclose(st["Ap"], A[N - 1], atol=1e-13)


def test_single_plane():
    """One plane: A = I - (D_0s / D_s) U exactly and omega = 0."""
    M = 50
    n0 = _rand_unit(M, 5)
    g = torch.Generator().manual_seed(6)
    u = 0.01 * torch.randn(M, 3, dtype=F64, generator=g)
    lens = lambda n: {"a_th": torch.zeros(M, dtype=F64), "a_ph": torch.zeros(M, dtype=F64),
                      "u_tt": u[:, 0], "u_pp": u[:, 1], "u_tp": u[:, 2]}
    st = rays.trace(n0, [100.0, 250.0], [lens])
    U = torch.stack([torch.stack([u[:, 0], u[:, 2]], -1), torch.stack([u[:, 2], u[:, 1]], -1)], -2)
    assert torch.allclose(st["A"], torch.eye(2, dtype=F64) - (150.0 / 250.0) * U, atol=1e-15)
    assert torch.allclose(rays.decompose(st["A"])[3], torch.zeros(M, dtype=F64), atol=1e-16)


def test_transport_holonomy_is_spherical_excess():
    """Transporting a tangent vector around a geodesic triangle rotates it by
    the enclosed area (Gauss-Bonnet, unit sphere); there and back is the
    identity (Appendix B)."""
    a = torch.tensor([[0.0, 0.0, 1.0]], dtype=F64)
    b = torch.tensor([[1.0, 0.0, 0.0]], dtype=F64)
    c = torch.tensor([[0.0, 1.0, 0.0]], dtype=F64)
    # octant triangle: excess pi/2; go a -> b -> c -> a in small steps (the
    # pole a is avoided as a basis point by starting just off it)
    def arc(p, q, k):
        out = []
        w = math.acos(float((p * q).sum()))
        for i in range(1, k + 1):
            t = i / k
            v = (math.sin((1 - t) * w) * p + math.sin(t * w) * q) / math.sin(w)
            out.append(v)
        return out
    eps = 1e-3
    start = torch.tensor([[math.sin(eps), math.sin(eps), 1.0]], dtype=F64)
    start = start / torch.linalg.vector_norm(start)
    b2 = torch.tensor([[1.0, 1e-3, 1e-3]], dtype=F64); b2 = b2 / torch.linalg.vector_norm(b2)
    c2 = torch.tensor([[1e-3, 1.0, 1e-3]], dtype=F64); c2 = c2 / torch.linalg.vector_norm(c2)
    path = [start] + arc(start, b2, 50) + arc(b2, c2, 50) + arc(c2, start, 50)
    A = torch.tensor([[[1.0, 0.0], [0.0, 0.0]]], dtype=F64)   # v v^T with v = theta-hat
    for p, q in zip(path[:-1], path[1:]):
        A = rays.transport(A, p, q)
    # rank-2 tensor v v^T rotated by angle w: [[c^2, cs], [cs, s^2]]
    w = math.atan2(float(A[0, 0, 1]) * 2, float(A[0, 0, 0] - A[0, 1, 1]))
    # compare the enclosed solid angle (triangle slightly smaller than the octant)
    def solid_angle(p, q, r):
        num = float((p * torch.cross(q, r, dim=-1)).sum())
        den = 1 + float((p * q).sum() + (q * r).sum() + (r * p).sum())
        return 2 * math.atan2(num, den)
    omega = solid_angle(start, b2, c2)
    assert abs(abs(w) - 2 * omega) < 1e-9 or abs(abs(w) - (2 * math.pi - 2 * omega)) < 1e-9, (w, omega)
    # there and back
    B = torch.tensor([[[0.3, 0.1], [-0.2, 0.9]]], dtype=F64)
    p, q = path[10], path[120]
    assert torch.allclose(rays.transport(rays.transport(B, p, q), q, p), B, atol=1e-14)


def test_galaxy_interpolation_equivalence():
    """Eq. gatraj (interpolating A_n, A_{n+1}) equals Eq. truegatraj
    (one recursion step from planes n-1, n to the galaxy) when A_{n+1} comes
    from Eq. Atraj (Appendix D)."""
    g = torch.Generator().manual_seed(7)
    M = 30
    An1 = torch.eye(2, dtype=F64) + 0.1 * torch.randn(M, 2, 2, dtype=F64, generator=g)   # A_{n-1}
    An = torch.eye(2, dtype=F64) + 0.1 * torch.randn(M, 2, 2, dtype=F64, generator=g)    # A_n
    Un = 0.05 * torch.randn(M, 2, 2, dtype=F64, generator=g)
    Un = 0.5 * (Un + Un.transpose(-1, -2))
    cm1, cn, cn1 = 800.0, 900.0, 1000.0
    chig = 900.0 + 100.0 * torch.rand(M, dtype=F64, generator=g)
    c, d = rays.recursion_coeffs(cm1, cn, cn1)
    Anp1 = (1 - c) * An1 + c * An - d * (Un @ An)
    via_interp = rays.galaxy_interp(An, Anp1, cn, cn1, chig)
    cg, dg = rays.recursion_coeffs(cm1, cn, chig)
    direct = (1 - cg)[:, None, None] * An1 + cg[:, None, None] * An - dg[:, None, None] * (Un @ An)
    assert torch.allclose(via_interp, direct, atol=1e-13)


def test_rays_bend_toward_a_point_mass():
    """With the Appendix A point-mass deflection, a back-traced ray moves
    toward the mass (alpha = -grad psi, Eq. betaprop)."""
    mass = torch.tensor([0.0, 0.0, 1.0], dtype=F64)

    def lens(n):
        th = torch.atan2(torch.sqrt(n[:, 0] ** 2 + n[:, 1] ** 2), n[:, 2])
        a_th = -(1 / (4 * math.pi)) * torch.sin(th) / (1 - torch.cos(th)) * 1e-4
        z = torch.zeros_like(th)
        return {"a_th": a_th, "a_ph": z, "u_tt": z, "u_pp": z, "u_tp": z}

    n0 = torch.tensor([[math.sin(0.2), 0.0, math.cos(0.2)]], dtype=F64)
    st = rays.trace(n0, [500.0, 1000.0], [lens])
    nf = st["x"] / torch.linalg.vector_norm(st["x"])
    assert float((nf * mass).sum()) > float((n0 * mass).sum())
