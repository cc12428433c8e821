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

// atan(t) by the Gregory series through t^13 for |t| < 0.04 (first omitted
// term below 1e-20 relative).
__device__ __forceinline__ double atan_small(double t) {
  const double t2 = t * t;
  return t * (1.0 - t2 * ((1.0 / 3.0) - t2 * ((1.0 / 5.0) - t2 * ((1.0 / 7.0) - t2 * ((1.0 / 9.0) -
                                                                                    t2 * ((1.0 / 11.0) - t2 * (1.0 / 13.0)))))));
}

template <typename T>
__device__ __forceinline__ double uat(const T* u, int n, int i, int j) {
  return (double)u[(size_t)(i + 1) * (n + 2) + (j + 1)];
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

// Lens fields at unit vector nv (tangent basis et, ep there) from patch
// potential u (n x n cells of size h, ghost-ring layout), R the patch rotation.  The five partials of the four
// cells around the point are blended bilinearly; since each partial is a
// tensor-product stencil, the blend is one tensor-product stencil on a 6 x 6
// block of cells.  The patch angles' sines and cosines come from the
// components of the rotated unit vector.
template <typename T>
__device__ __forceinline__ void patch_lens_fields_t(const T* u, int n, double h, double inv_h, const double* R,
                                                    const double nv[3], const double et[3], const double ep[3],
                                                    double out[5]) {
  // patch-frame vector and angles
  const double vx = R[0] * nv[0] + R[1] * nv[1] + R[2] * nv[2];
  const double vy = R[3] * nv[0] + R[4] * nv[1] + R[5] * nv[2];
  const double vz = R[6] * nv[0] + R[7] * nv[1] + R[8] * nv[2];
  const double r2 = vx * vx + vy * vy, is = rsqrt(r2), rho = r2 * is;
  // theta' - pi/2 = -atan(vz / rho) and phi' = atan(vy / vx): near the patch
  // centre (theta', phi') = (pi/2, 0) both ratios are small
  const double tz = vz * is, ty = vx > 0.0 ? vy / vx : 1.0;
  const double dth = fabs(tz) < 0.04 ? -atan_small(tz) : atan2(rho, vz) - 0.5 * kPi;
  const double php = fabs(ty) < 0.04 ? atan_small(ty) : atan2(vy, vx);
  const double x = dth * inv_h + 0.5 * n - 0.5;
  const double y = php * inv_h + 0.5 * n - 0.5;
  double i0 = floor(x), j0 = floor(y);
  i0 = fmin(fmax(i0, 0.0), (double)(n - 2));
  j0 = fmin(fmax(j0, 0.0), (double)(n - 2));
  const double fx = x - i0, fy = y - j0;
  const int ii = (int)i0, jj = (int)j0;
  // blended stencils (rows: theta', columns: phi')
  double A1[6], A2[6], B1[6], B2[6];
  const int r0 = fd_blend(ii, n, fx, A1, A2);
  const int c0 = fd_blend(jj, n, fy, B1, B2);
  const size_t pitch = (size_t)n + 2;
  const T* ub = u + (size_t)(r0 + 1) * pitch + (c0 + 1);
  const int ci = jj - c0, ri = ii - r0;   // the bilinear cells inside the 6 x 6 block
  double pt = 0, ptt = 0, ptp = 0, pp = 0, ppp = 0;
  double rl[6] = {0, 0, 0, 0, 0, 0};      // rows ii, ii + 1 blended, per column
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const T* row = ub + (size_t)a * pitch;
    double v[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) v[b] = (double)row[b];
    // columns jj, jj + 1 blended in this row
    double cl = 0.0, mix = 0.0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      if (b == ci) cl += (1.0 - fy) * v[b];
      if (b == ci + 1) cl += fy * v[b];
      mix += B1[b] * v[b];
    }
    pt += A1[a] * cl;
    ptt += A2[a] * cl;
    ptp += A1[a] * mix;
    const double wr = (a == ri) ? 1.0 - fx : (a == ri + 1 ? fx : 0.0);
#pragma unroll
    for (int b = 0; b < 6; ++b) rl[b] += wr * v[b];
  }
#pragma unroll
  for (int b = 0; b < 6; ++b) {
    pp += B1[b] * rl[b];
    ppp += B2[b] * rl[b];
  }
  const double c1 = inv_h / 12.0, c2 = inv_h * inv_h / 12.0;
  const double v0 = pt * c1, v1 = pp * c1, v2 = ptt * c2, v3 = ppp * c2, v4 = ptp * c1 * inv_h / 12.0;
  // Appendix A in the patch basis at the point: sin(theta') = rho, cos(theta') = vz
  // (the rotated vector is a unit vector), sin(phi') = vy / rho, cos(phi') = vx / rho
  const double s = rho, co = vz;
  const double a_t = -v0, a_p = -v1 * is;
  const double u_tt = v2;
  const double u_pp = v3 * is * is + co * is * v0;
  const double u_tp = v4 * is - co * v1 * is * is;
  // patch basis vectors at the point, mapped to global coordinates (R^T)
  const double sp = vy * is, cp = vx * is;
  const double tl[3] = {co * cp, co * sp, -s};
  const double pl[3] = {-sp, cp, 0.0};
  double tg[3], pg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tg[k] = R[k] * tl[0] + R[3 + k] * tl[1] + R[6 + k] * tl[2];
    pg[k] = R[k] * pl[0] + R[3 + k] * pl[1] + R[6 + k] * pl[2];
  }
  const double q00 = et[0] * tg[0] + et[1] * tg[1] + et[2] * tg[2];
  const double q01 = et[0] * pg[0] + et[1] * pg[1] + et[2] * pg[2];
  const double q10 = ep[0] * tg[0] + ep[1] * tg[1] + ep[2] * tg[2];
  const double q11 = ep[0] * pg[0] + ep[1] * pg[1] + ep[2] * pg[2];
  out[0] = q00 * a_t + q01 * a_p;
  out[1] = q10 * a_t + q11 * a_p;
  // U_g = Q U Q^T
  const double m00 = q00 * u_tt + q01 * u_tp, m01 = q00 * u_tp + q01 * u_pp;
  const double m10 = q10 * u_tt + q11 * u_tp, m11 = q10 * u_tp + q11 * u_pp;
  out[2] = m00 * q00 + m01 * q01;            // U_tt
  out[3] = m10 * q10 + m11 * q11;            // U_pp
  out[4] = m00 * q10 + m01 * q11;            // U_tp
}

__device__ __forceinline__ void patch_lens_fields(const MGView& V, int b, const double nv[3], const double et[3],
                                                  const double ep[3], double out[5]) {
  const size_t stride = (size_t)(V.n + 2) * (V.n + 2);
  patch_lens_fields_t(V.u + stride * b, V.n, V.h, V.inv_h, V.rot + 9 * (size_t)b, nv, et, ep, out);
}

}  // namespace clc
