// Lens fields from the finest multigrid patch level (paper Sec. 3.2: fourth-
// order finite differences, one-sided Fornberg stencils at the patch edge,
// bilinear interpolation to the point, Christoffel terms of Appendix A and
// rotation back to the global basis).
#pragma once

#include "mg.cuh"

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

template <typename T>
__device__ __forceinline__ double uat(const T* u, int n, int i, int j) {
  return (double)u[(size_t)(i + 1) * (n + 2) + (j + 1)];
}

// psi_t', psi_p', psi_t't', psi_p'p', psi_t'p' at cell (i, j)
template <typename T>
__device__ __forceinline__ void cell_partials(const T* u, int n, int i, int j, double inv_h, double p[5]) {
  double wi1[5], wj1[5], wi2[5], wj2[5];
  const int bi1 = fd_stencil(i, n, 1, wi1), bj1 = fd_stencil(j, n, 1, wj1);
  const int bi2 = fd_stencil(i, n, 2, wi2), bj2 = fd_stencil(j, n, 2, wj2);
  double pt = 0, pp = 0, ptt = 0, ppp = 0, ptp = 0;
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    pt += wi1[t] * uat(u, n, bi1 + t, j);
    ptt += wi2[t] * uat(u, n, bi2 + t, j);
    pp += wj1[t] * uat(u, n, i, bj1 + t);
    ppp += wj2[t] * uat(u, n, i, bj2 + t);
    double row = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) row += wj1[s] * uat(u, n, bi1 + t, bj1 + s);
    ptp += wi1[t] * row;
  }
  const double c1 = inv_h / 12.0, c2 = inv_h * inv_h / 12.0;
  p[0] = pt * c1;
  p[1] = pp * c1;
  p[2] = ptt * c2;
  p[3] = ppp * c2;
  p[4] = ptp * c1 * inv_h / 12.0;
}

template <typename T>
__device__ __forceinline__ void patch_lens_fields_t(const T* u, int n, double h, const double* R, const double nv[3],
                                                    double out[5]) {
  // patch-frame vector and angles
  const double vx = R[0] * nv[0] + R[1] * nv[1] + R[2] * nv[2];
  const double vy = R[3] * nv[0] + R[4] * nv[1] + R[5] * nv[2];
  const double vz = R[6] * nv[0] + R[7] * nv[1] + R[8] * nv[2];
  const double rho = sqrt(vx * vx + vy * vy);
  const double thp = atan2(rho, vz);
  const double php = atan2(vy, vx);
  const double x = (thp - 0.5 * kPi) / h + 0.5 * n - 0.5;
  const double y = php / h + 0.5 * n - 0.5;
  double i0 = floor(x), j0 = floor(y);
  i0 = fmin(fmax(i0, 0.0), (double)(n - 2));
  j0 = fmin(fmax(j0, 0.0), (double)(n - 2));
  const double fx = x - i0, fy = y - j0;
  const int ii = (int)i0, jj = (int)j0;
  double v[5] = {0, 0, 0, 0, 0};
  const double inv_h = 1.0 / h;
  double p[5];
  const double wts[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    cell_partials(u, n, ii + (c & 1), jj + (c >> 1), inv_h, p);
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += wts[c] * p[k];
  }
  // Appendix A in the patch basis at the point
  const double s = sin(thp), co = cos(thp);
  const double is = 1.0 / s;
  const double a_t = -v[0], a_p = -v[1] * is;
  const double u_tt = v[2];
  const double u_pp = v[3] * is * is + co * is * v[0];
  const double u_tp = v[4] * is - co * v[1] * is * is;
  // patch basis vectors at the point, mapped to global coordinates (R^T)
  const double sp = sin(php), cp = cos(php);
  const double tl[3] = {co * cp, co * sp, -s};
  const double pl[3] = {-sp, cp, 0.0};
  double tg[3], pg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tg[k] = R[k] * tl[0] + R[3 + k] * tl[1] + R[6 + k] * tl[2];
    pg[k] = R[k] * pl[0] + R[3 + k] * pl[1] + R[6 + k] * pl[2];
  }
  const double gr = sqrt(nv[0] * nv[0] + nv[1] * nv[1]);
  const double et[3] = {nv[2] * nv[0] / gr, nv[2] * nv[1] / gr, -gr};
  const double ep[3] = {-nv[1] / gr, nv[0] / gr, 0.0};
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

__device__ __forceinline__ void patch_lens_fields(const MGView& V, int b, const double nv[3], double out[5]) {
  const size_t stride = (size_t)(V.n + 2) * (V.n + 2);
  patch_lens_fields_t(V.u + stride * b, V.n, V.h, V.rot + 9 * (size_t)b, nv, out);
}

}  // namespace clc
