// Grid search for lensed galaxy images (paper Sec. 2.3 and the grid-search
// implementation, Sec. 3.3).  Rays start at the RING pixel centres; the
// triangles joining centres of consecutive rings (every centre closes one
// triangle with its predecessor on its ring and the last centre of the
// neighbouring ring before it in longitude; two cap triangles at each pole)
// map, vertex for vertex, onto the rays' source-sphere positions.  A galaxy
// has one image per source-sphere triangle that contains it (gnomonic
// projection at the galaxy: the three triple products det(g, v_i, v_j) share
// a sign), at the image-sphere point given by the barycentric coordinates of
// that projection; the inverse magnification matrix there comes from the
// ring-bilinear interpolation of the rays' matrices, each parallel
// transported to the image (Appendix B).
//
// Search: a triangle that contains g has its owner (the centre it is listed
// under) within T of g, T the largest distance on the source sphere from an
// owner to the other vertices of its triangles, and that owner's pixel centre
// within D + T, D the largest distance between a ray's source position and
// its pixel centre.  One pass reduces D and T; then one thread per galaxy
// visits the pixel centres within D + T, keeps the owners whose rays lie
// within T and tests their triangles.  The candidate set contains every
// triangle that can contain g, so the result is that of testing all
// triangles.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "sphere.cuh"

namespace clc {

constexpr int kMaxImages = 8;
constexpr double kSearchMargin = 1e-9;   // radians added to D and T

// Integer geometry of ring r: first pixel, pixel count n, and h (longitudes
// (2 k + h) pi / n, h = 1 on rings offset by half a pixel).
struct RingI {
  int64_t first;
  int n;
  int h;
};

__device__ __forceinline__ RingI ring_int(int nside, int r) {
  const int64_t ns = nside;
  RingI o;
  if (r < nside) {
    o.n = 4 * r;
    o.first = 2 * (int64_t)r * (r - 1);
    o.h = 1;
  } else if (r > 3 * nside) {
    const int64_t ip = 4 * ns - r;
    o.n = (int)(4 * ip);
    o.first = 12 * ns * ns - 2 * ip * (ip + 1);
    o.h = 1;
  } else {
    o.n = 4 * nside;
    o.first = 2 * ns * (ns - 1) + (int64_t)(r - nside) * 4 * ns;
    o.h = ((r - nside) & 1) == 0 ? 1 : 0;
  }
  return o;
}

// Index on ring b of its last point before point k of ring a in longitude,
// cyclically: the largest j with (2 j + h_b) / n_b < (2 k + h_a) / n_a (two
// rings never share a longitude).
__device__ __forceinline__ int last_before(int k, const RingI& a, const RingI& b) {
  const int64_t num = (int64_t)(2 * k + a.h) * b.n - (int64_t)b.h * a.n - 1;
  return num < 0 ? b.n - 1 : (int)(num / (2 * (int64_t)a.n));
}

// Vertices, counter-clockwise seen from outside, of triangle 2 p + s (s = 0:
// the strip below p's ring, s = 1: the strip above) for p at position k of
// ring r; false for unused ids.
__device__ __forceinline__ bool tri_vertices_rk(int nside, int64_t p, int r, int k, int s, int64_t v[3]) {
  if (s == 1 && r == 1) {
    if (p == 1) { v[0] = 0; v[1] = 1; v[2] = 2; return true; }
    if (p == 3) { v[0] = 2; v[1] = 3; v[2] = 0; return true; }
    return false;
  }
  if (s == 0 && r == 4 * nside - 1) {
    const int64_t f = 12 * (int64_t)nside * nside - 4;
    if (p == f + 1) { v[0] = f + 2; v[1] = f + 1; v[2] = f; return true; }
    if (p == f + 3) { v[0] = f; v[1] = f + 3; v[2] = f + 2; return true; }
    return false;
  }
  const RingI a = ring_int(nside, r), b = ring_int(nside, s == 0 ? r + 1 : r - 1);
  const int64_t prev = a.first + (k == 0 ? a.n - 1 : k - 1);
  const int64_t q = b.first + last_before(k, a, b);
  v[0] = prev;
  v[1] = s == 0 ? q : p;
  v[2] = s == 0 ? p : q;
  return true;
}

__device__ __forceinline__ bool tri_vertices(int nside, int64_t p, int s, int64_t v[3]) {
  int64_t k;
  const int r = pix2ring(nside, p, &k);
  return tri_vertices_rk(nside, p, r, (int)k, s, v);
}

__device__ __forceinline__ void load3(const double* __restrict__ x, int64_t n, int64_t p, double o[3]) {
  o[0] = x[p];
  o[1] = x[n + p];
  o[2] = x[2 * n + p];
}

// det(g, a, b) = g . (a x b), every product and sum rounded separately in
// this order (the decision must not depend on FMA contraction)
__device__ __forceinline__ double edge_det(const double g[3], const double a[3], const double b[3]) {
  const double c0 = __dsub_rn(__dmul_rn(a[1], b[2]), __dmul_rn(a[2], b[1]));
  const double c1 = __dsub_rn(__dmul_rn(a[2], b[0]), __dmul_rn(a[0], b[2]));
  const double c2 = __dsub_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0]));
  return __dadd_rn(__dadd_rn(__dmul_rn(g[0], c0), __dmul_rn(g[1], c1)), __dmul_rn(g[2], c2));
}

// det(g, x_u, x_v), evaluated on the edge's endpoints in increasing pixel
// order so that the two triangles sharing the edge see opposite values
__device__ __forceinline__ double oriented(const double g[3], int64_t u, const double xu[3], int64_t v,
                                           const double xv[3]) {
  return u < v ? edge_det(g, xu, xv) : -edge_det(g, xv, xu);
}

// Containment of g in the source-sphere triangle v; d[i] = det(g, v_j, v_k)
// for the edge opposite vertex i, gx[i] = g . x_{v_i}.
__device__ __forceinline__ bool contains(const double* __restrict__ x, int64_t n, const double g[3],
                                         const int64_t v[3], double d[3], double gx[3]) {
  double a[3], b[3], c[3];
  load3(x, n, v[0], a);
  load3(x, n, v[1], b);
  load3(x, n, v[2], c);
  d[2] = oriented(g, v[0], a, v[1], b);
  d[0] = oriented(g, v[1], b, v[2], c);
  d[1] = oriented(g, v[2], c, v[0], a);
  gx[0] = dot3(a, g);
  gx[1] = dot3(b, g);
  gx[2] = dot3(c, g);
  const bool pos = d[0] >= 0.0 && d[1] >= 0.0 && d[2] >= 0.0;
  const bool neg = d[0] <= 0.0 && d[1] <= 0.0 && d[2] <= 0.0;
  const bool nz = d[0] != 0.0 || d[1] != 0.0 || d[2] != 0.0;
  return (pos || neg) && nz && gx[0] > 0.0 && gx[1] > 0.0 && gx[2] > 0.0;
}

__device__ __forceinline__ void normalize3(const double a[3], double o[3]) {
  const double is = rsqrt(dot3(a, a));
  o[0] = a[0] * is;
  o[1] = a[1] * is;
  o[2] = a[2] * is;
}

// squared chord between unit vectors, and the angle it spans
__device__ __forceinline__ double chord2(const double a[3], const double b[3]) {
  const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ double chord2_angle(double c2) { return 2.0 * asin(fmin(1.0, 0.5 * sqrt(c2))); }

// unit vector of the centre of the pixel at position k of ring r
__device__ __forceinline__ void centre_vec(int nside, int r, int64_t k, double c[3]) {
  const Ring g = ring_geom(nside, r);
  const int h = g.phi0 != 0.0 ? 1 : 0;
  double sn, cs;
  sincospi((double)(2 * k + h) / (double)g.npix, &sn, &cs);
  c[0] = g.s * cs;
  c[1] = g.s * sn;
  c[2] = g.z;
}

__device__ __forceinline__ void centre_vec(int nside, int64_t p, double c[3]) {
  int64_t k;
  const int r = pix2ring(nside, p, &k);
  centre_vec(nside, r, k, c);
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));   // v >= 0: bit order = value order
}

// bounds[0], bounds[1]: the squared chords of D and T (as the bits of
// non-negative doubles, whose integer order is their value order)
__global__ void k_image_bounds(const double* __restrict__ x, int nside, int64_t npx,
                               unsigned long long* __restrict__ bounds) {
  double dmax = 0.0, tmax = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += stride) {
    int64_t k;
    const int r = pix2ring(nside, p, &k);
    double xr[3], xn[3], c[3];
    load3(x, npx, p, xr);
    normalize3(xr, xn);
    centre_vec(nside, r, k, c);
    dmax = fmax(dmax, chord2(xn, c));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      int64_t v[3];
      if (!tri_vertices_rk(nside, p, r, (int)k, s, v)) continue;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (v[i] == p) continue;
        double yr[3], yn[3];
        load3(x, npx, v[i], yr);
        normalize3(yr, yn);
        tmax = fmax(tmax, chord2(xn, yn));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_pos(bounds, dmax);
    atomic_max_pos(bounds + 1, tmax);
  }
}

struct ImageOut {
  int32_t* nimg;
  int64_t* tri;
  double* img;   // [3][max_images][ngal]
  double* A;     // [4][max_images][ngal] or null
};

__global__ void __launch_bounds__(128, 4) k_find_images(const double* __restrict__ x, const double* __restrict__ Ar,
                                                     int nside, int64_t npx, const double* __restrict__ gal,
                                                     int64_t ngal, const unsigned long long* __restrict__ bounds,
                                                     int max_images, ImageOut out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ngal) return;
  double g[3], gn[3];
  load3(gal, ngal, m, g);
  const double gg = dot3(g, g);
  if (!(gg > 0.0) || !isfinite(gg)) {   // no direction: no image
    out.nimg[m] = 0;
    for (int q = 0; q < max_images; ++q) {
      const size_t o = (size_t)q * ngal + m;
      out.tri[o] = -1;
      for (int c = 0; c < 3; ++c) out.img[((size_t)c * max_images + q) * ngal + m] = 0.0;
      if (out.A)
        for (int c = 0; c < 4; ++c) out.A[((size_t)c * max_images + q) * ngal + m] = 0.0;
    }
    return;
  }
  normalize3(g, gn);
  const double dmax = chord2_angle(__longlong_as_double((long long)bounds[0]));
  const double tmax = chord2_angle(__longlong_as_double((long long)bounds[1]));
  const double tm = tmax + kSearchMargin;
  const double R = dmax + tm + kSearchMargin;
  // chord^2 limits (a 4 admits every point of the sphere)
  const bool filter = tm < 0.5 * kPi;
  const double hs = sin(0.5 * tm), c2t = filter ? 4.0 * hs * hs * (1.0 + 1e-12) : 4.0;
  const double hr = sin(0.5 * fmin(R, kPi)), c2r = R < kPi ? 4.0 * hr * hr * (1.0 + 1e-12) : 4.0;
  const double sp = sqrt(gn[0] * gn[0] + gn[1] * gn[1]);
  const double thp = atan2(sp, gn[2]);
  double pp = atan2(gn[1], gn[0]);
  if (pp < 0.0) pp += 2.0 * kPi;
  const double zhi = cos(fmax(0.0, thp - R)), zlo = cos(fmin(kPi, thp + R));
  const int i0 = max(1, (int)floor(ring_coord(nside, zhi)) - 1);
  const int i1 = min(4 * nside - 1, (int)ceil(ring_coord(nside, zlo)) + 1);
  int64_t found[kMaxImages];
  int nfound = 0, count = 0;
  for (int i = i0; i <= i1; ++i) {
    const Ring r = ring_geom(nside, i);
    const int np = r.npix;
    int jl = 0, jh = np - 1;
    const double den = 2.0 * sp * r.s;
    if (den > 1e-300) {
      const double C = (2.0 - c2r - 2.0 * gn[2] * r.z) / den;
      if (C >= 1.0) continue;
      if (C > -1.0) {
        const double span = acos(C), dphi = 2.0 * kPi / (double)np;
        const double base = (pp - r.phi0) / dphi;
        jl = (int)floor(base - span / dphi) - 1;
        jh = (int)ceil(base + span / dphi) + 1;
        if (jh - jl + 1 >= np) {
          jl = 0;
          jh = np - 1;
        }
      }
    }
    for (int j = jl; j <= jh; ++j) {
      const int64_t p = r.first + (int64_t)(((j % np) + np) % np);
      double xr[3], xn[3];
      load3(x, npx, p, xr);
      normalize3(xr, xn);
      if (chord2(xn, gn) > c2t) continue;
      const int jw = (int)(p - r.first);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int64_t v[3];
        double d[3], gx[3];
        if (!tri_vertices_rk(nside, p, i, jw, s, v) || !contains(x, npx, g, v, d, gx)) continue;
        ++count;
        // keep the max_images smallest triangle ids, ascending
        const int64_t id = 2 * p + s;
        int pos = nfound;
        while (pos > 0 && found[pos - 1] > id) --pos;
        if (pos < max_images) {
          const int last = nfound < max_images ? nfound : max_images - 1;
          for (int q = last; q > pos; --q) found[q] = found[q - 1];
          found[pos] = id;
          if (nfound < max_images) ++nfound;
        }
      }
    }
  }
  out.nimg[m] = count;
  for (int q = 0; q < max_images; ++q) {
    const size_t o = (size_t)q * ngal + m;
    if (q >= nfound) {
      out.tri[o] = -1;
      for (int c = 0; c < 3; ++c) out.img[((size_t)c * max_images + q) * ngal + m] = 0.0;
      if (out.A)
        for (int c = 0; c < 4; ++c) out.A[((size_t)c * max_images + q) * ngal + m] = 0.0;
      continue;
    }
    const int64_t id = found[q];
    int64_t v[3];
    double d[3], gx[3];
    tri_vertices(nside, id >> 1, (int)(id & 1), v);
    contains(x, npx, g, v, d, gx);
    // barycentric coordinates in the gnomonic plane at g; image on the image sphere
    double lam[3], tot = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lam[i] = d[i] * gx[i];
      tot += lam[i];
    }
    double w3[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double c[3];
      centre_vec(nside, v[i], c);
      const double li = lam[i] / tot;
      w3[0] += li * c[0];
      w3[1] += li * c[1];
      w3[2] += li * c[2];
    }
    double ni[3];
    normalize3(w3, ni);
    out.tri[o] = id;
    for (int c = 0; c < 3; ++c) out.img[((size_t)c * max_images + q) * ngal + m] = ni[c];
    if (!out.A) continue;
    // inverse magnification matrix at the image
    const double rho = sqrt(ni[0] * ni[0] + ni[1] * ni[1]);
    double ph = atan2(ni[1], ni[0]);
    if (ph < 0.0) ph += 2.0 * kPi;
    const Interp8 w = interp_weights(nside, atan2(rho, ni[2]), ph);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < 8; ++k) {
      if (w.w[k] == 0.0) continue;
      const int64_t pk = w.p[k];
      double xr[3], xn[3], t0[3], p0[3], Q[4], Ak[4], At[4];
      load3(x, npx, pk, xr);
      normalize3(xr, xn);
      tangent_basis(xn, t0, p0);
      transport_q(xn, t0, ni, Q);
#pragma unroll
      for (int c = 0; c < 4; ++c) Ak[c] = Ar[(size_t)c * npx + pk];
      qaqt(Q, Ak, At);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += w.w[k] * At[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) out.A[((size_t)c * max_images + q) * ngal + m] = acc[c];
  }
}

}  // namespace clc

using namespace clc;

extern "C" int clc_find_images(clc_ctx* ctx, int nside, const double* x, const double* A, int64_t ngal,
                               const double* g, int max_images, int32_t* nimg, int64_t* tri, double* img,
                               double* A_img) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside) || ngal < 0 || max_images < 1 || max_images > kMaxImages)
    return set_err(ctx, CLC_EINVAL, "clc_find_images: bad nside, ngal or max_images (1..8)");
  if (ngal == 0) return CLC_OK;
  if ((A == nullptr) != (A_img == nullptr))
    return set_err(ctx, CLC_EINVAL, "clc_find_images: A and A_img must both be given or both be NULL");
  if (!x || !g || !nimg || !tri || !img)
    return set_err(ctx, CLC_EINVAL, "clc_find_images: null pointer");
  cudaSetDevice(ctx->device);
  const int64_t npx = 12 * (int64_t)nside * nside;
  auto* bounds = (unsigned long long*)scratch(ctx, 6, 2 * sizeof(unsigned long long));
  if (!bounds) return CLC_ENOMEM;
  if (cuda_check(ctx, cudaMemsetAsync(bounds, 0, 2 * sizeof(unsigned long long), ctx->stream), "memset"))
    return CLC_ECUDA;
  int64_t nb = (npx + 255) / 256;
  const int64_t cap = (int64_t)num_sms(ctx) * 8;
  if (nb > cap) nb = cap;
  CLC_LAUNCH(ctx, "k_image_bounds", k_image_bounds, (int)nb, 256, 0, x, nside, npx, bounds);
  if (int rc = launch_check(ctx, "k_image_bounds")) return rc;
  // the search radius sets the work per galaxy: refuse inputs whose rays
  // moved so far from their pixels that the search would cover a large part
  // of the sphere for many galaxies
  unsigned long long hb[2];
  if (cuda_check(ctx, cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, ctx->stream), "bounds copy") ||
      cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "bounds sync"))
    return CLC_ECUDA;
  double c2d, c2t;
  memcpy(&c2d, &hb[0], sizeof(double));
  memcpy(&c2t, &hb[1], sizeof(double));
  if (!(c2d >= 0.0) || !(c2t >= 0.0) || !std::isfinite(c2d) || !std::isfinite(c2t))
    return set_err(ctx, CLC_EINVAL, "clc_find_images: non-finite ray positions");
  const double dm = 2.0 * std::asin(std::fmin(1.0, 0.5 * std::sqrt(c2d)));
  const double tm = 2.0 * std::asin(std::fmin(1.0, 0.5 * std::sqrt(c2t)));
  const double R = std::fmin(dm + tm + 2 * kSearchMargin, kPi);
  // pixels within R, plus the margin of a few pixels on each ring in range
  const double cand = 0.5 * (1.0 - std::cos(R)) * (double)npx + 3.0 * (8.0 * R * nside / kPi + 3.0);
  if (cand * (double)ngal > 5e10)
    return set_err(ctx, CLC_EINVAL, "clc_find_images: rays too far from their pixels for the search (radius " +
                                        std::to_string(R) + " rad)");
  ImageOut out{nimg, tri, img, A_img};
  const int threads = 128;
  const int64_t blocks = (ngal + threads - 1) / threads;
  if (blocks > 0x7fffffff) return set_err(ctx, CLC_EINVAL, "clc_find_images: too many galaxies");
  CLC_LAUNCH(ctx, "k_find_images", k_find_images, (int)blocks, threads, 0, x, A, nside, npx, g, ngal, bounds,
             max_images, out);
  return launch_check(ctx, "k_find_images");
}
