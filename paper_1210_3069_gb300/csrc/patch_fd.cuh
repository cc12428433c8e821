// Lens fields from the finest multigrid patch level (paper Sec. 3.2: fourth-
// order finite differences, one-sided Fornberg stencils at the patch edge,
// bilinear interpolation to the point, Christoffel terms of Appendix A and
// rotation back to the global basis).
#pragma once

#include "mg.cuh"
#include "sphere.cuh"

namespace clc {

// 5-point stencils x 12 (first / second derivative), rows: evaluation at
// offset 0, 1 (one-sided) and 2 (central) of the five points.
__device__ __constant__ static const double kD1[3][5] = {
    {-25., 48., -36., 16., -3.}, {-3., -10., 18., -6., 1.}, {1., -8., 0., 8., -1.}};
__device__ __constant__ static const double kD2[3][5] = {
    {35., -104., 114., -56., 11.}, {11., -20., 6., 4., -1.}, {-1., 16., -30., 16., -1.}};

// weights w[5] and first index of the stencil of derivative `order` at cell k
// of n cells (interior cells only)
__device__ __forceinline__ int fd_stencil(int k, int n, int order, double w[5]) {
  const double(*D)[5] = order == 1 ? kD1 : kD2;
  if (k >= 2 && k <= n - 3) {
#pragma unroll
    for (int t = 0; t < 5; ++t) w[t] = D[2][t];
    return k - 2;
  }
  if (k < 2) {
#pragma unroll
    for (int t = 0; t < 5; ++t) w[t] = D[k][t];
    return 0;
  }
  const int off = n - 1 - k;
  const double sg = order == 1 ? -1.0 : 1.0;
#pragma unroll
  for (int t = 0; t < 5; ++t) w[t] = sg * D[off][4 - t];
  return n - 5;
}

// Bilinear blend of the stencils of cells k and k + 1 (weights 1 - f, f) as
// one stencil on the six points first .. first + 5: w1 (first derivative),
// w2 (second derivative), both x 12.  The second cell's stencil starts at
// the same point as the first one's or one later (offset known only at run
// time, so both placements are formed and selected).
__device__ __forceinline__ int fd_blend(int k, int n, double f, double w1[6], double w2[6]) {
  const double g = 1.0 - f;
  if (k >= 2 && k + 1 <= n - 3) {   // both central: the second is shifted by one point
    w1[0] = g * 1.0;
    w1[1] = g * -8.0 + f * 1.0;
    w1[2] = g * 0.0 + f * -8.0;
    w1[3] = g * 8.0 + f * 0.0;
    w1[4] = g * -1.0 + f * 8.0;
    w1[5] = f * -1.0;
    w2[0] = g * -1.0;
    w2[1] = g * 16.0 + f * -1.0;
    w2[2] = g * -30.0 + f * 16.0;
    w2[3] = g * 16.0 + f * -30.0;
    w2[4] = g * -1.0 + f * 16.0;
    w2[5] = f * -1.0;
    return k - 2;
  }
  double a1[5], a2[5], b1[5], b2[5];
  const int ba = fd_stencil(k, n, 1, a1), bb = fd_stencil(k + 1, n, 1, b1);
  fd_stencil(k, n, 2, a2);
  fd_stencil(k + 1, n, 2, b2);
  const int first = min(ba, bb);
  const bool sa = ba > first, sb = bb > first;   // stencil starts one point later
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const double a1t = t < 5 ? a1[t] : 0.0, a1s = t >= 1 ? a1[t - 1] : 0.0;
    const double a2t = t < 5 ? a2[t] : 0.0, a2s = t >= 1 ? a2[t - 1] : 0.0;
    const double b1t = t < 5 ? b1[t] : 0.0, b1s = t >= 1 ? b1[t - 1] : 0.0;
    const double b2t = t < 5 ? b2[t] : 0.0, b2s = t >= 1 ? b2[t - 1] : 0.0;
    w1[t] = g * (sa ? a1s : a1t) + f * (sb ? b1s : b1t);
    w2[t] = g * (sa ? a2s : a2t) + f * (sb ? b2s : b2t);
  }
  return first;
}

// asin(s) by its Maclaurin series through s^13 for |s| < 0.04 (first omitted
// term below 1e-21 relative); coefficients (2k)! / (4^k (k!)^2 (2k + 1)).
__device__ __forceinline__ double asin_small(double s) {
  const double s2 = s * s;
  return s * (1.0 + s2 * ((1.0 / 6.0) + s2 * ((3.0 / 40.0) + s2 * ((5.0 / 112.0) + s2 * ((35.0 / 1152.0) +
              s2 * ((63.0 / 2816.0) + s2 * (231.0 / 13312.0)))))));
}

// Fourth-order central stencils x 12 (first, second derivative) at point
// s + 2 of the 6-vector y: y_s - y_{s+4} + 8 (y_{s+3} - y_{s+1}) and
// 16 (y_{s+1} + y_{s+3}) - 30 y_{s+2} - (y_s + y_{s+4}).
__device__ __forceinline__ double c_d1(const double* y, int s) { return fma(8.0, y[s + 3] - y[s + 1], y[s] - y[s + 4]); }
__device__ __forceinline__ double c_d2(const double* y, int s) {
  return fma(-30.0, y[s + 2], fma(16.0, y[s + 1] + y[s + 3], -(y[s] + y[s + 4])));
}
// the blend (1 - f) D(k) + f D(k + 1) of two neighbouring cells' stencils
__device__ __forceinline__ double blend_d1(const double* y, double f) { return fma(f, c_d1(y, 1) - c_d1(y, 0), c_d1(y, 0)); }
// The six weights of blend_d1 over y[0 .. 5] (g = 1 - f): g D + f D shifted
// by one point, D = (1, -8, 0, 8, -1), for sums taken several times with one f
__device__ __forceinline__ void d1_weights(double f, double g, double w[6]) {
  w[0] = g;
  w[1] = fma(-8.0, g, f);
  w[2] = -8.0 * f;
  w[3] = 8.0 * g;
  w[4] = fma(8.0, f, -g);
  w[5] = -f;
}
__device__ __forceinline__ double dot6(const double w[6], const double* y) {
  double s = w[0] * y[0];
#pragma unroll
  for (int b = 1; b < 6; ++b) s = fma(w[b], y[b], s);
  return s;
}
__device__ __forceinline__ double blend_d2(const double* y, double f) { return fma(f, c_d2(y, 1) - c_d2(y, 0), c_d2(y, 0)); }

// Lens fields at unit vector nv (tangent basis et, ep there) from patch
// potential u (n x n cells of size h, ghost-ring layout), R the patch
// rotation.  The five partials of the four cells around the point are blended
// bilinearly; each partial is a tensor-product stencil, so the blend is one
// tensor-product stencil on the 6 x 6 block of cells ii - 2 .. ii + 3,
// jj - 2 .. jj + 3.  Away from the patch edge (every ray in its home bundle's
// patch) all stencils are central and the blend is applied as (1 - f) D_k +
// f D_{k+1} with the integer stencils, on row and column blends read straight
// from the block; within two cells of the edge the one-sided stencils are
// blended into six-point weights (fd_blend).  The patch angles come from the
// rotated unit vector: theta' - pi/2 = -asin(v_z), phi' = asin(v_y / rho).
template <typename T>
__device__ __forceinline__ void patch_lens_fields_t(const T* u, int n, double h, double inv_h, const double* R,
                                                    const double nv[3], const double et[3], const double ep[3],
                                                    double out[5]) {
  // patch-frame vector and angles
  const double vx = R[0] * nv[0] + R[1] * nv[1] + R[2] * nv[2];
  const double vy = R[3] * nv[0] + R[4] * nv[1] + R[5] * nv[2];
  const double vz = R[6] * nv[0] + R[7] * nv[1] + R[8] * nv[2];
  const double r2 = vx * vx + vy * vy, is = rsqrt(r2), rho = r2 * is;
  const double sp = vy * is, cp = vx * is;   // sin, cos of phi'
  double dth, php;
  if (fabs(vz) < 0.04 && fabs(sp) < 0.04 && vx > 0.0) {
    dth = -asin_small(vz);
    php = asin_small(sp);
  } else {
    dth = atan2(rho, vz) - 0.5 * kPi;
    php = atan2(vy, vx);
  }
  const double x = dth * inv_h + 0.5 * n - 0.5;
  const double y = php * inv_h + 0.5 * n - 0.5;
  int ii = __double2int_rd(x), jj = __double2int_rd(y);
  ii = min(max(ii, 0), n - 2);
  jj = min(max(jj, 0), n - 2);
  const double fx = x - (double)ii, fy = y - (double)jj;
  const size_t pitch = (size_t)n + 2;
  double pt, ptt, ptp, pp, ppp;
  if (ii >= 2 && ii + 4 <= n && jj >= 2 && jj + 4 <= n) {
    // central stencils: block rows / columns ii - 2 .. ii + 3, jj - 2 .. jj + 3
    const T* ub = u + (size_t)(ii - 1) * pitch + (jj - 1);
    double c[6], mix[6], r[6], wx[6], wy[6];
    const double gy = 1.0 - fy, gx = 1.0 - fx;
    d1_weights(fx, gx, wx);
    d1_weights(fy, gy, wy);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const T* row = ub + (size_t)a * pitch;
      double v[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) v[b] = (double)row[b];
      c[a] = fma(fy, v[3], gy * v[2]);    // columns jj, jj + 1
      mix[a] = dot6(wy, v);
    }
    const T* ra = ub + 2 * pitch;         // rows ii, ii + 1
#pragma unroll
    for (int b = 0; b < 6; ++b) r[b] = fma(fx, (double)ra[pitch + b], gx * (double)ra[b]);
    pt = dot6(wx, c);
    ptt = blend_d2(c, fx);
    ptp = dot6(wx, mix);
    pp = dot6(wy, r);
    ppp = blend_d2(r, fy);
  } else {
    double A1[6], A2[6], B1[6], B2[6];
    const int r0 = fd_blend(ii, n, fx, A1, A2);
    const int c0 = fd_blend(jj, n, fy, B1, B2);
    const T* ub = u + (size_t)(r0 + 1) * pitch + (c0 + 1);
    const int ci = jj - c0, ri = ii - r0;   // the bilinear cells inside the 6 x 6 block
    pt = ptt = ptp = pp = ppp = 0.0;
    double rl[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const T* row = ub + (size_t)a * pitch;
      const double cl = (1.0 - fy) * (double)row[ci] + fy * (double)row[ci + 1];
      double mix = 0.0;
#pragma unroll
      for (int b = 0; b < 6; ++b) mix += B1[b] * (double)row[b];
      pt += A1[a] * cl;
      ptt += A2[a] * cl;
      ptp += A1[a] * mix;
    }
#pragma unroll
    for (int b = 0; b < 6; ++b)
      rl[b] = (1.0 - fx) * (double)ub[(size_t)ri * pitch + b] + fx * (double)ub[(size_t)(ri + 1) * pitch + b];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      pp += B1[b] * rl[b];
      ppp += B2[b] * rl[b];
    }
  }
  const double c1 = inv_h * (1.0 / 12.0), c2 = c1 * inv_h;
  const double v0 = pt * c1, v1 = pp * c1, v2 = ptt * c2, v3 = ppp * c2, v4 = ptp * (c1 * c1);
  // Appendix A in the patch basis at the point: sin(theta') = rho, cos(theta') = vz
  const double co = vz;
  const double a_t = -v0, a_p = -v1 * is;
  const double u_tt = v2;
  const double u_pp = (v3 * is + co * v0) * is;
  const double u_tp = (v4 - co * v1 * is) * is;
  // theta-hat' of the patch basis at the point, in global coordinates (R^T);
  // both bases are right-handed at the same point, so the change of basis is
  // the plane rotation [[q00, -q10], [q10, q00]]
  const double tl[3] = {co * cp, co * sp, -rho};
  double tg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) tg[k] = R[k] * tl[0] + R[3 + k] * tl[1] + R[6 + k] * tl[2];
  const double q00 = et[0] * tg[0] + et[1] * tg[1] + et[2] * tg[2];
  const double q10 = ep[0] * tg[0] + ep[1] * tg[1];
  out[0] = q00 * a_t - q10 * a_p;
  out[1] = q10 * a_t + q00 * a_p;
  // U_g = Q U Q^T: the trace is kept and the traceless part
  // ((u_tt - u_pp) / 2, u_tp) turns by twice the angle of Q
  const double cq = fma(q00, q00, -q10 * q10), sq = 2.0 * q00 * q10;
  const double hs = 0.5 * (u_tt + u_pp), hd = 0.5 * (u_tt - u_pp);
  const double e2 = fma(cq, hd, -sq * u_tp);
  out[2] = hs + e2;                          // U_tt
  out[3] = hs - e2;                          // U_pp
  out[4] = fma(sq, hd, cq * u_tp);           // U_tp
}

// Patch slot of bundle b: the bundle itself on the full sky, the domain's
// slot map on a partial sky (-1: the bundle has no patch; the lookup is
// counted and gives zero fields, the lens action of matter at the mean
// density, Sec. 3.4).
__device__ __forceinline__ int mg_slot(const MGView& V, int b) {
  if (!V.slot) return b;
  const int s = V.slot[b];
  if (s < 0 && V.outside) atomicAdd(V.outside, 1ull);
  return s;
}

__device__ __forceinline__ void patch_lens_fields(const MGView& V, int b, const double nv[3], const double et[3],
                                                  const double ep[3], double out[5]) {
  const int s = mg_slot(V, b);
  if (s < 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k] = 0.0;
    return;
  }
  const size_t stride = (size_t)(V.n + 2) * (V.n + 2);
  patch_lens_fields_t(V.u + stride * s, V.n, V.h, V.inv_h, V.rot + 9 * (size_t)s, nv, et, ep, out);
}

}  // namespace clc
