"""GPU grid search for galaxy images (Sec. 2.3 and the grid-search
implementation, Sec. 3.3) against the oracle, which tests every triangle:
image counts and triangle ids bit for bit (both sides take the containment
decision with the same unfused FP64 triple products on identical inputs),
image positions and transported matrices to rounding.  Undeflected, rotated,
weakly and strongly lensed skies with random matrices; galaxies exactly on
rays and on edges (decisions at the rounding level), at the poles; fewer
slots than images; the call without matrices; bad arguments.  At Nside 2048
(the ray grid of the lens-plane workload) the single-image property of a
weak lens for every galaxy, and sampled galaxies against the oracle run on
the triangles around them."""
import math

import pytest
import torch

from oracle import healpix as hp, images as im
from tests.gpu_util import ctx
from workloads import synthetic

pytestmark = pytest.mark.gpu
F64 = torch.float64
LENS = torch.tensor([0.2, 0.4, 0.7], dtype=F64) / math.sqrt(0.69)


def _rotation(axis, w):
    k = torch.tensor(axis, dtype=F64)
    k = k / k.norm()
    K = torch.tensor([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]], dtype=F64)
    return torch.eye(3, dtype=F64) + math.sin(w) * K + (1.0 - math.cos(w)) * (K @ K)


def _sky(nside, kind):
    c = hp.pix2vec_ring(nside, torch.arange(hp.npix(nside)))
    if kind == "identity":
        return 2.5 * c
    if kind == "rotated":
        return c @ _rotation([0.3, -0.5, 0.8], 0.2).T
    b, s = {"weak": (0.02, 0.05), "strong": (0.15, 0.03)}[kind]
    return synthetic.cored_lens_map(c, LENS, b, s)[0]


def _galaxies(x, M, seed):
    z, phi = synthetic.uniform_sphere(M, seed)
    g = [hp.vec_from_zphi(z, phi)]
    # near the lens centre (several images for the strong lens)
    gen = torch.Generator().manual_seed(seed + 1)
    off = 0.05 * torch.randn(M // 4, 3, generator=gen, dtype=F64)
    g.append(LENS + off)
    # exactly on rays, on edge midpoints (unnormalised sums), at the poles
    p = torch.randint(0, x.shape[0], (8,), generator=gen)
    q = torch.remainder(p + 1, x.shape[0])
    g += [x[p], x[p] + x[q], torch.tensor([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], dtype=F64)]
    return torch.cat(g)


def _gpu(c, nside, x, A, g, max_images, matrices=True):
    npx = x.shape[0]
    out = c.find_images(nside, x.T.contiguous().cuda(), A.reshape(npx, 4).T.contiguous().cuda(),
                        g.T.contiguous().cuda(), max_images, matrices)
    c.sync()
    return [t.cpu() if t is not None else None for t in out]


def _maxabs(t):
    return float(t.abs().max()) if t.numel() else 0.0


def _check(nside, x, A, g, max_images, got, matrices=True):
    nimg, tri, img, Ai = got
    wn, wt, wi, wA = im.find_images(nside, x, A, g, max_images)
    assert torch.equal(nimg.long(), wn)
    assert torch.equal(tri.T, wt)
    used = wt >= 0
    v = img.permute(2, 1, 0)
    assert _maxabs(torch.linalg.vector_norm(v - wi, dim=-1)[used]) < 1e-13
    assert _maxabs(v[~used]) == 0.0
    if matrices:
        # at an image on a pole the (theta-hat, phi-hat) basis is undefined (each
        # side takes it from the rounding of x and y): there only the parts that
        # do not depend on the basis, trace and antisymmetric part, are compared
        ga = Ai.permute(2, 1, 0).reshape(g.shape[0], max_images, 2, 2)
        pole = torch.sqrt(wi[..., 0] ** 2 + wi[..., 1] ** 2) < 1e-8
        assert _maxabs((ga - wA)[~pole]) < 1e-12
        inv = lambda a: torch.stack([a[..., 0, 0] + a[..., 1, 1], a[..., 0, 1] - a[..., 1, 0]], -1)
        assert _maxabs((inv(ga) - inv(wA))[pole]) < 1e-12
    return wn


@pytest.mark.parametrize("nside,kind,M,max_images", [
    (1, "identity", 40, 4), (8, "rotated", 200, 4), (16, "weak", 300, 4), (32, "strong", 200, 6),
    (64, "strong", 80, 2), (16, "identity", 100, 1)])
def test_images_match_oracle(nside, kind, M, max_images):
    c = ctx()
    x = _sky(nside, kind)
    A = synthetic.random_jacobians(x.shape[0], 0.1, 500 + nside)
    g = _galaxies(x, M, 600 + nside)
    wn = _check(nside, x, A, g, max_images, _gpu(c, nside, x, A, g, max_images))
    if kind == "strong":
        assert int(wn.max()) >= 3          # the case reaches several images


def test_images_without_matrices_and_empty_call():
    c = ctx()
    nside = 16
    x = _sky(nside, "weak")
    A = synthetic.random_jacobians(x.shape[0], 0.1, 71)
    g = _galaxies(x, 100, 72)
    got = _gpu(c, nside, x, A, g, 3, matrices=False)
    assert got[3] is None
    _check(nside, x, A, g, 3, got, matrices=False)
    e = torch.empty(3, 0, dtype=F64, device="cuda")
    nimg, tri, img, Ai = c.find_images(nside, x.T.contiguous().cuda(), A.reshape(-1, 4).T.contiguous().cuda(),
                                       e, 2)
    c.sync()
    assert nimg.numel() == 0


def test_bad_arguments_are_rejected():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    nside = 4
    x = _sky(nside, "identity").T.contiguous().cuda()
    A = synthetic.random_jacobians(12 * nside * nside, 0.1, 73).reshape(-1, 4).T.contiguous().cuda()
    g = torch.ones(3, 5, dtype=F64, device="cuda")
    for bad in (dict(nside=3), dict(max_images=0), dict(max_images=9)):
        kw = dict(nside=nside, max_images=2)
        kw.update(bad)
        with pytest.raises(clc.CalclensError):
            c.find_images(kw["nside"], x, A, g, kw["max_images"])
    # rays scattered over the whole sphere: the search would cover most of
    # the 786 432 pixels for each of a million galaxies
    ns2 = 256
    far = torch.randn(3, 12 * ns2 * ns2, dtype=F64, device="cuda")
    A2 = torch.zeros(4, 12 * ns2 * ns2, dtype=F64, device="cuda")
    big = torch.ones(3, 1_000_000, dtype=F64, device="cuda")
    with pytest.raises(clc.CalclensError):
        c.find_images(ns2, far, A2, big, 2)
    c.sync()


def _local_owners(nside, g, radius):
    """RING pixels hit by a dense grid of points within `radius` of the unit
    vector g (spacing a quarter of the pixel size): a superset of the pixels
    whose centres lie within radius - one pixel size of g."""
    h = math.sqrt(4 * math.pi / hp.npix(nside))
    n = int(math.ceil(radius / (0.25 * h)))
    u = torch.linspace(-radius, radius, 2 * n + 1, dtype=F64)
    a = torch.linalg.cross(g, torch.tensor([0.0, 0.0, 1.0], dtype=F64))
    a = a / a.norm()
    b = torch.linalg.cross(g, a)
    U, V = torch.meshgrid(u, u, indexing="ij")
    r = torch.sqrt(U * U + V * V)
    keep = r <= radius
    U, V, r = U[keep], V[keep], r[keep]
    d = (U[:, None] * a + V[:, None] * b) / torch.where(r > 0, r, 1.0)[:, None]
    pts = torch.cos(r)[:, None] * g + torch.sin(r)[:, None] * d
    z = pts[:, 2].clamp(-1, 1)
    phi = torch.remainder(torch.atan2(pts[:, 1], pts[:, 0]), 2 * math.pi)
    return torch.unique(hp.ang2pix_ring(nside, z, phi))


def test_full_size_weak_lens_sampled():
    """Nside 2048 rays (50 331 648) through a weak cored lens with a
    deflection of up to 2e-3 rad: every galaxy has exactly one image, and
    sampled galaxies match the oracle run on the triangles owned by the
    pixels within (deflection + two triangle sizes) of them."""
    c = ctx()
    nside = 2048
    npx = hp.npix(nside)
    cen = hp.pix2vec_ring(nside, torch.arange(npx))
    x = synthetic.cored_lens_map(cen, LENS, 2e-3, 5e-3)[0]
    del cen
    A = synthetic.random_jacobians(npx, 0.05, 81)
    z, phi = synthetic.uniform_sphere(1_000_000, 82)
    g = torch.cat([hp.vec_from_zphi(z, phi), LENS + 0.01 * torch.randn(2000, 3, generator=torch.Generator().manual_seed(83), dtype=F64)])
    nimg, tri, img, Ai = _gpu(c, nside, x, A, g, 2)
    assert bool((nimg == 1).all())
    h = math.sqrt(4 * math.pi / npx)
    sample = torch.tensor([0, 1, 2, 3, 999_999, 1_000_000, 1_000_500, 1_001_999])
    for m in sample.tolist():
        gm = g[m] / g[m].norm()
        own = _local_owners(nside, gm, 2e-3 + 6 * h)
        wn, wt, wi, wA = im.find_images(nside, x, A, g[m:m + 1], 2, owners=own)
        assert int(wn[0]) == int(nimg[m]) and torch.equal(wt[0], tri[:, m])
        assert float(torch.linalg.vector_norm(img[:, 0, m] - wi[0, 0])) < 1e-13
        assert float((Ai[:, 0, m].reshape(2, 2) - wA[0, 0]).abs().max()) < 1e-12
