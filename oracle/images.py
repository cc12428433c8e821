"""Grid search for lensed galaxy images (oracle; test infrastructure).

Sec. 2.3 finds the image of a galaxy at a given source position with a grid
search: triangles built from the rays' starting points on the image sphere
map, vertex for vertex, to triangles of the same rays on the source sphere;
every source-sphere triangle that contains the galaxy gives one image, at the
position interpolated linearly over the triangle's image-sphere vertices.
Sec. 3.3 (the grid-search implementation) builds the triangles from the
HEALPix pixel centres, tests containment and interpolates with barycentric
coordinates in the plane tangent to the sphere at the galaxy's source
position, and obtains the inverse magnification matrix at the image from a
separate four-ray HEALPix interpolation on the image sphere after parallel
transport of the rays' matrices to the image position.

Readings taken here (the paper gives no formulas for them):

* Triangles.  Rays start at RING pixel centres.  Between rings r and r + 1
  (a strip) the centres of both rings are merged by longitude (no two are
  ever at equal longitude) and every centre closes one triangle with its
  predecessor on its own ring and the last centre of the other ring before
  it in longitude.  The four centres of ring 1 form two cap triangles, as do
  those of the last ring.  This tiles the sphere with 2 Npix - 4 triangles;
  all are listed counter-clockwise seen from outside.
* Triangle ids.  A centre p owns at most two triangles: id 2 p closes the
  strip below its ring (p on the upper ring), id 2 p + 1 the strip above it
  (p on the lower ring).  The cap triangles of ring 1 are ids 3 and 7, those
  of the last ring 2 (Npix - 3) and 2 (Npix - 1); every triangle contains its
  owner.
* Containment.  The projection is the gnomonic one (the tangent plane at the
  galaxy seen from the sphere's centre), which maps great circles to straight
  lines, so a galaxy g lies in a projected triangle (v0, v1, v2) exactly when
  the three triple products det(g, v0, v1), det(g, v1, v2), det(g, v2, v0)
  share a sign (all >= 0 for a triangle that kept its orientation, all <= 0
  for one that flipped, i.e. a negative-parity image), not all zero, and all
  three vertices lie in g's hemisphere.  The triple product of an edge is
  evaluated once per edge, on its endpoints in increasing pixel order, so
  the two triangles that share an edge see exactly opposite values.
* Interpolation.  The barycentric coordinates in that tangent plane are
  lambda_i proportional to det(g, v_j, v_k) (g . v_i) for the edge (j, k)
  opposite vertex i; the image is the unit vector along sum_i lambda_i c_i,
  c_i the vertices' image-sphere positions (pixel centres).
* Matrix.  The ring-bilinear interpolation of `interp.py` at the image
  position, each ray's A carried from the basis at its source-sphere
  position to the basis at the image by the parallel transport of
  Appendix B.
* Several images are reported in increasing triangle id.

Plain definition, no search structure: every triangle is tested.  The triple
products use separately rounded multiplies and adds in the order written, so
a decision taken on identical inputs can be reproduced bit for bit.
"""
import torch

from . import geometry
from . import healpix as hp
from . import interp
from . import rays

F64 = torch.float64
I64 = torch.int64


def _ring_offsets(nside):
    """Per ring (index r - 1): pixel count n, first pixel, and h = 1 when the
    ring's longitudes are (k + 1/2) 2 pi / n, h = 0 when they are k 2 pi / n."""
    rt = hp.ring_table(nside)
    return rt["npix"], rt["first"], (rt["phi0"] != 0).to(I64)


def _last_before(k, h, n, h2, n2):
    """Index on a ring (n2 points, offset h2) of the last point whose longitude
    lies below that of point k of a ring (n points, offset h), cyclically:
    the largest j with (2 j + h2) / n2 < (2 k + h) / n, -1 wrapping to n2 - 1."""
    num = (2 * k + h) * n2 - h2 * n - 1
    j = torch.div(num, 2 * n, rounding_mode="floor")
    return torch.where(j < 0, n2 - 1, j)


def triangles(nside, owners=None):
    """(ids [T], vertices [T, 3]) of the 2 Npix - 4 triangles, or of those
    owned by the given RING pixels: RING pixel ids, counter-clockwise seen
    from outside, ordered by triangle id."""
    npx = hp.npix(nside)
    nr, first, h = _ring_offsets(nside)
    if owners is None:
        p = torch.arange(npx, dtype=I64)
    else:
        p = torch.unique(torch.as_tensor(owners, dtype=I64))
    ring, k = hp.pix2ring(nside, p)
    r0 = ring - 1                                      # 0-based ring index
    nlast = 4 * nside - 1
    n, f0, hh = nr[r0], first[r0], h[r0]
    prev = f0 + torch.remainder(k - 1, n)
    # strip below (owner on the upper ring): (prev, last of ring below before p, p)
    rb = torch.clamp(r0 + 1, max=nlast - 1)
    jb = _last_before(k, hh, n, h[rb], nr[rb])
    below = torch.stack([prev, first[rb] + jb, p], -1)
    # strip above (owner on the lower ring): (prev, p, last of ring above before p)
    ra = torch.clamp(r0 - 1, min=0)
    ja = _last_before(k, hh, n, h[ra], nr[ra])
    above = torch.stack([prev, p, first[ra] + ja], -1)
    tri = torch.stack([below, above], 1).reshape(-1, 3)
    tid = torch.stack([2 * p, 2 * p + 1], 1).reshape(-1)
    valid = torch.stack([ring < nlast, ring > 1], 1).reshape(-1)
    # caps
    fs = npx - 4
    caps = {3: (0, 1, 2), 7: (2, 3, 0),
            2 * (fs + 1): (fs + 2, fs + 1, fs), 2 * (fs + 3): (fs, fs + 3, fs + 2)}
    for cid, v in caps.items():
        at = torch.nonzero(tid == cid).flatten()
        if at.numel():
            tri[at[0]] = torch.tensor(v, dtype=I64)
            valid[at[0]] = True
    return tid[valid], tri[valid]


def _edge_det(g, xa, xb):
    """det(g, x_a, x_b) = g . (x_a x x_b), each product and sum rounded
    separately in this order."""
    c0 = xa[..., 1] * xb[..., 2] - xa[..., 2] * xb[..., 1]
    c1 = xa[..., 2] * xb[..., 0] - xa[..., 0] * xb[..., 2]
    c2 = xa[..., 0] * xb[..., 1] - xa[..., 1] * xb[..., 0]
    return (g[..., 0] * c0 + g[..., 1] * c1) + g[..., 2] * c2


def _oriented(g, x, u, v):
    """det(g, x_u, x_v) from the edge's canonical evaluation (smaller id first)."""
    lo, hi = torch.minimum(u, v), torch.maximum(u, v)
    e = _edge_det(g, x[lo], x[hi])
    return torch.where(u < v, e, -e)


def find_images(nside, x, A, g, max_images=4, owners=None):
    """Images of galaxies at source positions g [M, 3] (any positive length).

    x [Npix, 3]: source-sphere positions of the rays started at the RING
    pixel centres (any common positive length); A [Npix, 2, 2]: their inverse
    magnification matrices in the (theta-hat, phi-hat) basis at x.
    owners: optional RING pixels whose triangles alone are tested (default:
    all triangles).
    Returns nimg [M] (images found), tri [M, max_images] (ids, -1 unused),
    img [M, max_images, 3] (unit vectors, 0 unused), Aimg [M, max_images, 2, 2].
    """
    x = torch.as_tensor(x, dtype=F64)
    A = torch.as_tensor(A, dtype=F64)
    g = torch.as_tensor(g, dtype=F64)
    ids, tv = triangles(nside, owners)
    M = g.shape[0]
    nimg = torch.zeros(M, dtype=I64)
    tri = torch.full((M, max_images), -1, dtype=I64)
    img = torch.zeros(M, max_images, 3, dtype=F64)
    Aimg = torch.zeros(M, max_images, 2, 2, dtype=F64)
    v0, v1, v2 = tv[:, 0], tv[:, 1], tv[:, 2]
    for m in range(M):
        gm = g[m].expand(ids.numel(), 3)
        d2 = _oriented(gm, x, v0, v1)
        d0 = _oriented(gm, x, v1, v2)
        d1 = _oriented(gm, x, v2, v0)
        pos = (d0 >= 0) & (d1 >= 0) & (d2 >= 0)
        neg = (d0 <= 0) & (d1 <= 0) & (d2 <= 0)
        nz = (d0 != 0) | (d1 != 0) | (d2 != 0)
        gx = torch.stack([(x[v] * gm).sum(-1) for v in (v0, v1, v2)], -1)
        front = (gx > 0).all(-1)
        hit = torch.nonzero((pos | neg) & nz & front).flatten()
        nimg[m] = hit.numel()
        for s, t in enumerate(hit[:max_images].tolist()):
            lam = torch.stack([d0[t], d1[t], d2[t]]) * gx[t]
            lam = lam / lam.sum()
            v = (lam[:, None] * hp.pix2vec_ring(nside, tv[t])).sum(0)
            v = v / torch.linalg.vector_norm(v)
            tri[m, s] = ids[t]
            img[m, s] = v
            Aimg[m, s] = interpolate_matrix(nside, x, A, v)
    return nimg, tri, img, Aimg


def interpolate_matrix(nside, x, A, v):
    """A at unit vector v on the image sphere: ring-bilinear weights of the
    pixels around v, each pixel's matrix transported from the basis at its
    ray's source-sphere direction x[p] / |x[p]| to the basis at v
    (Appendix B)."""
    z, phi = geometry.zphi_of(v)
    theta = torch.atan2(torch.sqrt(v[0] * v[0] + v[1] * v[1]), z)
    idx, w = interp.interp_weights(nside, theta.reshape(1), phi.reshape(1))
    idx, w = idx[0], w[0]
    xk = x[idx]
    xk = xk / torch.linalg.vector_norm(xk, dim=-1, keepdim=True)
    Ak = rays.transport(A[idx], xk, v.expand(idx.numel(), 3))
    return (w[:, None, None] * Ak).sum(0)
