// Vectors and tangent frames on the unit sphere shared by the ray recursion
// and the image search: the (theta-hat, phi-hat) basis, Rodrigues rotation
// and the parallel transport of Appendix B.
#pragma once

#include <cuda_runtime.h>

namespace clc {

// Tangent basis (theta-hat, phi-hat) at the unit vector n; on a pole (where
// it is undefined) its limit along phi = 0.
__device__ __forceinline__ void tangent_basis(const double n[3], double t[3], double p[3]) {
  const double r2 = n[0] * n[0] + n[1] * n[1];
  if (r2 == 0.0) {
    t[0] = n[2] >= 0.0 ? 1.0 : -1.0; t[1] = 0.0; t[2] = 0.0;
    p[0] = 0.0; p[1] = 1.0; p[2] = 0.0;
    return;
  }
  const double ir = rsqrt(r2), rho = r2 * ir;
  t[0] = n[2] * n[0] * ir; t[1] = n[2] * n[1] * ir; t[2] = -rho;
  p[0] = -n[1] * ir; p[1] = n[0] * ir; p[2] = 0.0;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// rotate v about unit axis k by the angle with cosine c, sine s
__device__ __forceinline__ void rodrigues(const double v[3], const double k[3], double c, double s, double o[3]) {
  double kv[3];
  cross3(k, v, kv);
  const double kd = dot3(k, v) * (1.0 - c);
#pragma unroll
  for (int i = 0; i < 3; ++i) o[i] = v[i] * c + kv[i] * s + k[i] * kd;
}

// Transport matrix Q (2x2) from the basis (t0, p0) at n0 to the basis at n1
// along the great circle: the rotation R taking n0 to n1 maps (t0, p0, n0)
// to the right-handed frame (R t0, n1 x R t0, n1) of the tangent plane at n1,
// so Q is the plane rotation [[c, -s], [s, c]] with c = t1 . R t0,
// s = p1 . R t0.
__device__ __forceinline__ void transport_q(const double n0[3], const double t0[3], const double n1[3],
                                            double Q[4]) {
  double cr[3];
  cross3(n0, n1, cr);
  const double s2 = dot3(cr, cr);
  const double c = dot3(n0, n1);
  double t1[3], p1[3];
  tangent_basis(n1, t1, p1);
  double tr[3];
  if (s2 > 0.0) {
    const double is = rsqrt(s2), s = s2 * is;
    const double k[3] = {cr[0] * is, cr[1] * is, cr[2] * is};
    rodrigues(t0, k, c, s, tr);
  } else {
    for (int i = 0; i < 3; ++i) tr[i] = t0[i];
  }
  Q[0] = dot3(t1, tr);
  Q[2] = dot3(p1, tr);
  Q[1] = -Q[2];
  Q[3] = Q[0];
}

// o = Q A Q^T (row-major 2x2)
__device__ __forceinline__ void qaqt(const double Q[4], const double A[4], double o[4]) {
  const double m0 = Q[0] * A[0] + Q[1] * A[2], m1 = Q[0] * A[1] + Q[1] * A[3];
  const double m2 = Q[2] * A[0] + Q[3] * A[2], m3 = Q[2] * A[1] + Q[3] * A[3];
  o[0] = m0 * Q[0] + m1 * Q[1];
  o[1] = m0 * Q[2] + m1 * Q[3];
  o[2] = m2 * Q[0] + m3 * Q[1];
  o[3] = m2 * Q[2] + m3 * Q[3];
}

}  // namespace clc
