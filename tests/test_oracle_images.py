"""Pins of the grid-search oracle for galaxy images (paper Sec. 2.3 and the
grid-search implementation, Sec. 3.3).

The triangulation is checked as a tiling of the sphere (count, orientation,
solid angles summing to 4 pi, every edge shared by exactly two triangles);
containment against spherical-excess areas; image positions against exact
results: an undeflected and a rigidly rotated sky (second-order bound of the
chord-plane interpolation), and the roots of the one-dimensional lens
equation of an axisymmetric lens, in its single-image and three-image
regimes (image counts exact away from the caustics, positions converging at
second order); the matrix interpolation against the ring-bilinear
interpolation of rotation-invariant matrices."""
import math

import torch

from oracle import healpix as hp, images as im, interp
from workloads import synthetic

F64 = torch.float64


def _solid_angle(a, b, c):
    """Signed solid angle of the spherical triangle (a, b, c) (Van Oosterom
    and Strackee 1983)."""
    det = (a * torch.linalg.cross(b, c, dim=-1)).sum(-1)
    den = 1.0 + (a * b).sum(-1) + (b * c).sum(-1) + (c * a).sum(-1)
    return 2.0 * torch.atan2(det, den)


def _angle(a, b):
    return torch.atan2(torch.linalg.vector_norm(torch.linalg.cross(a, b, dim=-1), dim=-1), (a * b).sum(-1))


def _rotation(axis, w):
    k = torch.tensor(axis, dtype=F64)
    k = k / k.norm()
    K = torch.tensor([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]], dtype=F64)
    return torch.eye(3, dtype=F64) + math.sin(w) * K + (1.0 - math.cos(w)) * (K @ K)


def _identity_A(npx):
    return torch.eye(2, dtype=F64).expand(npx, 2, 2).clone()


def test_triangles_tile_the_sphere():
    for nside in (1, 2, 4, 8):
        ids, tv = im.triangles(nside)
        npx = hp.npix(nside)
        assert ids.numel() == 2 * npx - 4
        assert torch.equal(ids, torch.sort(ids).values)
        c = hp.pix2vec_ring(nside, torch.arange(npx))
        a, b, d = c[tv[:, 0]], c[tv[:, 1]], c[tv[:, 2]]
        om = _solid_angle(a, b, d)
        assert float(om.min()) > 0.0                      # counter-clockwise from outside
        assert abs(float(om.sum()) - 4 * math.pi) < 1e-12
        # every directed edge once, and its reverse once: a closed oriented surface
        e = torch.cat([tv[:, [0, 1]], tv[:, [1, 2]], tv[:, [2, 0]]])
        key = e[:, 0] * npx + e[:, 1]
        rkey = e[:, 1] * npx + e[:, 0]
        assert torch.unique(key).numel() == key.numel()
        assert torch.equal(torch.sort(key).values, torch.sort(rkey).values)
        # every triangle holds its owner
        assert bool((tv == (ids // 2)[:, None]).any(-1).all())


def test_owner_subset_matches_full_list():
    nside = 8
    ids, tv = im.triangles(nside)
    owners = torch.tensor([0, 1, 3, 50, 377, hp.npix(nside) - 3, hp.npix(nside) - 1])
    sid, stv = im.triangles(nside, owners)
    sel = torch.isin(ids // 2, owners)
    assert torch.equal(sid, ids[sel]) and torch.equal(stv, tv[sel])


def test_undeflected_sky_one_image_within_second_order_bound():
    """x = c: one triangle holds each galaxy (its three sub-triangles' solid
    angles add up to its own), and the image deviates from the galaxy by at
    most (1 - cos d) tan d / cos d, d the largest vertex distance."""
    nside = 16
    npx = hp.npix(nside)
    c = hp.pix2vec_ring(nside, torch.arange(npx))
    z, phi = synthetic.uniform_sphere(200, 11)
    g = hp.vec_from_zphi(z, phi)
    nimg, tri, img, _ = im.find_images(nside, 2.5 * c, _identity_A(npx), 0.7 * g)
    assert torch.equal(nimg, torch.ones_like(nimg))
    ids, tv = im.triangles(nside)
    t = tv[torch.searchsorted(ids, tri[:, 0])]
    a, b, d = c[t[:, 0]], c[t[:, 1]], c[t[:, 2]]
    parts = _solid_angle(g, a, b) + _solid_angle(g, b, d) + _solid_angle(g, d, a)
    assert torch.allclose(parts, _solid_angle(a, b, d), rtol=0, atol=1e-13)
    dv = torch.stack([_angle(g, a), _angle(g, b), _angle(g, d)], -1).max(-1).values
    bound = (1 - torch.cos(dv)) * torch.tan(dv) / torch.cos(dv)
    err = _angle(img[:, 0], g)
    assert bool((err <= 1.001 * bound + 1e-15).all())
    assert float(err.max()) > 0.01 * float(bound.max())  # the bound is not vacuous


def test_rotated_sky_images_undo_the_rotation():
    nside = 16
    npx = hp.npix(nside)
    c = hp.pix2vec_ring(nside, torch.arange(npx))
    Q = _rotation([0.3, -0.5, 0.8], 0.2)
    z, phi = synthetic.uniform_sphere(150, 12)
    g = hp.vec_from_zphi(z, phi)
    nimg, tri, img, _ = im.find_images(nside, c @ Q.T, _identity_A(npx), g)
    assert torch.equal(nimg, torch.ones_like(nimg))
    want = g @ Q                                          # Q^T g
    pix = 2.0 * math.sqrt(math.pi / (3.0 * nside * nside))
    assert float(_angle(img[:, 0], want).max()) < 0.5 * pix ** 3
    # scale of the source positions is irrelevant, bit for bit
    n2, t2, i2, _ = im.find_images(nside, 3.75 * (c @ Q.T), _identity_A(npx), 5.0 * g)
    assert torch.equal(t2, tri) and torch.equal(n2, nimg)


def _lens_roots(alpha, beta, nsamp=400001):
    """Signed angles t (from the lens centre, along the direction of the
    source) with t - sign(t) alpha(|t|) = beta, by sign changes on a fine
    grid refined by bisection."""
    def f(t):
        return t - torch.sign(t) * alpha(torch.abs(t)) - beta

    t = torch.linspace(-math.pi + 1e-9, math.pi - 1e-9, nsamp, dtype=F64)
    ft = f(t)
    idx = torch.nonzero(torch.sign(ft[1:]) != torch.sign(ft[:-1])).flatten()
    lo, hi = t[idx], t[idx + 1]
    flo = ft[idx]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        same = torch.sign(fm) == torch.sign(flo)
        lo = torch.where(same, mid, lo)
        flo = torch.where(same, fm, flo)
        hi = torch.where(same, hi, mid)
    return 0.5 * (lo + hi)


def _lens_galaxies(L, betas, seed):
    gen = torch.Generator().manual_seed(seed)
    ang = 2 * math.pi * torch.rand(betas.numel(), generator=gen, dtype=F64)
    e1 = torch.linalg.cross(L, torch.tensor([0.0, 0.0, 1.0], dtype=F64))
    e1 = e1 / e1.norm()
    e2 = torch.linalg.cross(L, e1)
    dirs = torch.cos(ang)[:, None] * e1 + torch.sin(ang)[:, None] * e2
    g = torch.cos(betas)[:, None] * L + torch.sin(betas)[:, None] * dirs
    return g, dirs


def _lens_errors(nside, b, s, betas, seed, max_images=6):
    L = torch.tensor([0.2, 0.4, 0.7], dtype=F64)
    L = L / L.norm()
    c = hp.pix2vec_ring(nside, torch.arange(hp.npix(nside)))
    x, alpha = synthetic.cored_lens_map(c, L, b, s)
    g, dirs = _lens_galaxies(L, betas, seed)
    nimg, tri, img, _ = im.find_images(nside, x, _identity_A(hp.npix(nside)), g, max_images=max_images)
    counts, errs = [], []
    for m in range(betas.numel()):
        r = _lens_roots(alpha, float(betas[m]))
        counts.append((r.numel(), int(nimg[m])))
        want = torch.cos(r)[:, None] * L + torch.sin(r)[:, None] * dirs[m]
        for k in range(min(int(nimg[m]), max_images)):
            errs.append(float(_angle(img[m, k].expand_as(want), want).min()))
    return counts, errs


def test_weak_axisymmetric_lens_images_converge_at_second_order():
    """b / 2s < 1: one image per galaxy; the error against the root of the
    lens equation drops about fourfold per halving of the pixel size."""
    betas = 0.3 * torch.rand(40, generator=torch.Generator().manual_seed(21), dtype=F64)
    c16, e16 = _lens_errors(16, 0.02, 0.05, betas, 22)
    c32, e32 = _lens_errors(32, 0.02, 0.05, betas, 22)
    assert all(n == 1 and k == 1 for n, k in c16 + c32)
    assert max(e32) < 1e-3
    assert max(e16) / max(e32) > 3.0


def test_strong_axisymmetric_lens_image_counts():
    """b / 2s = 2.5: three images for sources inside the radial caustic
    (beta ~ 0.035 rad here), one outside; galaxies are kept clear of both
    caustics (beta = 0 and the radial one)."""
    gen = torch.Generator().manual_seed(23)
    inner = 0.008 + 0.014 * torch.rand(12, generator=gen, dtype=F64)
    outer = 0.06 + 0.24 * torch.rand(12, generator=gen, dtype=F64)
    counts, errs = _lens_errors(64, 0.15, 0.03, torch.cat([inner, outer]), 24)
    assert [n for n, _ in counts[:12]] == [3] * 12 and [n for n, _ in counts[12:]] == [1] * 12
    assert all(n == k for n, k in counts), counts
    assert max(errs) < 0.01


def test_matrix_interpolation_of_rotation_invariant_matrices():
    """A = a I + b J (J the quarter-turn) commutes with the transport's plane
    rotation, so the result is a_int I + b_int J with a_int, b_int the
    ring-bilinear interpolation of the scalar maps at the image."""
    nside = 16
    npx = hp.npix(nside)
    c = hp.pix2vec_ring(nside, torch.arange(npx))
    gen = torch.Generator().manual_seed(31)
    a = 1.0 + 0.1 * torch.randn(npx, generator=gen, dtype=F64)
    bb = 0.1 * torch.randn(npx, generator=gen, dtype=F64)
    J = torch.tensor([[0.0, 1.0], [-1.0, 0.0]], dtype=F64)
    A = a[:, None, None] * torch.eye(2, dtype=F64) + bb[:, None, None] * J
    Q = _rotation([1.0, 0.2, -0.4], 0.05)
    z, phi = synthetic.uniform_sphere(40, 32)
    g = hp.vec_from_zphi(z, phi)
    nimg, tri, img, Aimg = im.find_images(nside, c @ Q.T, A, g)
    v = img[:, 0]
    th = torch.atan2(torch.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2), v[:, 2])
    ph = torch.remainder(torch.atan2(v[:, 1], v[:, 0]), 2 * math.pi)
    ai = interp.interpolate(nside, a, th, ph)
    bi = interp.interpolate(nside, bb, th, ph)
    want = ai[:, None, None] * torch.eye(2, dtype=F64) + bi[:, None, None] * J
    assert torch.allclose(Aimg[:, 0], want, rtol=0, atol=1e-14)


def test_basis_at_a_pole_is_the_limit_along_phi_zero():
    from oracle import geometry
    eps = 1e-9
    for zs in (1.0, -1.0):
        t0, p0 = geometry.basis(torch.tensor([[0.0, 0.0, zs]], dtype=F64))
        t1, p1 = geometry.basis(torch.tensor([[math.sin(eps), 0.0, zs * math.cos(eps)]], dtype=F64))
        assert torch.allclose(t0, t1, atol=2 * eps) and torch.allclose(p0, p1, atol=2 * eps)
