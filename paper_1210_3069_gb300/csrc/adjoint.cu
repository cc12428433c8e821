// Galaxy shears through the pure-SHT multiple-plane ray tracer and their
// adjoint with respect to the lens-plane convergence maps (paper Sec. 2.2,
// Sec. 3.2, Appendix B, Appendix D).
//
// Forward: one ray per galaxy starts at the galaxy's direction on plane 0;
// each plane's lens fields come from the SHT Poisson solve of its
// convergence map; after plane n every galaxy with chi_n <= chi_g < chi_{n+1}
// takes A_g = (1 - t) A^(n) + t A^(n+1), t = (chi_{n+1} / chi_g)
// ((chi_g - chi_n) / (chi_{n+1} - chi_n)) (Eq. gatraj) and its shear
// gamma_1 = -(A_11 - A_22) / 2, gamma_2 = -(A_12 + A_21) / 2 (Eq. invmagmat).
// The ray state entering every plane is checkpointed.
//
// Reverse: planes from last to first.  Each plane's lens maps are recomputed
// from its convergence map; each ray's step is re-run from its checkpoint
// with forward-mode dual numbers, which give the vector-Jacobian product of
// the step with respect to the entering state (including the dependence of
// the lens lookup on the ray position) and to the five lens values at the
// ray; the latter are scattered through the interpolation weights into
// adjoint lens maps, and the adjoint SHT Poisson solve (transposed ring
// FFTs, transposed derivative combinations, transposed Legendre synthesis,
// transposed Poisson and analysis) turns them into the gradient map.
#include "fft.cuh"
#include "legendre.cuh"
#include "patch_fd.cuh"

int clc_poisson_sht(clc_ctx*, const double*, int, int, int, double*, const clc_derivs*);
int clc_sht_synthesis(clc_ctx*, const double*, int, int, double*);
int clc_poisson_shtmg(clc_ctx*, const double*, int, const clc_mg_params*, clc_plane_solution*, const clc_derivs*);
int clc_solution_create(clc_ctx*, int, const clc_mg_params*, clc_plane_solution**);
int clc_solution_destroy(clc_plane_solution*);

namespace clc {

// the dual-number overloads below must not hide the FP64 math functions
using ::atan2;
using ::sincos;
using ::sqrt;

// ---------------------------------------------------------------------------
// forward-mode dual numbers with K tangent directions

template <int K>
struct Dual {
  double v;
  double d[K];
};

template <int K>
__device__ __forceinline__ Dual<K> dual_const(double a) {
  Dual<K> r;
  r.v = a;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = 0.0;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, double b) {
  Dual<K> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(double b, const Dual<K>& a) { return a * b; }
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, double b) {
  Dual<K> r = a;
  r.v += b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator+(double b, const Dual<K>& a) { return a + b; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, double b) {
  Dual<K> r = a;
  r.v -= b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator-(double b, const Dual<K>& a) {
  Dual<K> r = -a;
  r.v += b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, double b) { return a * (1.0 / b); }
template <int K>
__device__ __forceinline__ Dual<K> operator/(double a, const Dual<K>& b) { return dual_const<K>(a) / b; }
template <int K>
__device__ __forceinline__ Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = ::sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int K>
__device__ __forceinline__ void sincos(const Dual<K>& a, Dual<K>* s, Dual<K>* c) {
  double sv, cv;
  ::sincos(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s->d[k] = cv * a.d[k];
    c->d[k] = -sv * a.d[k];
  }
}
template <int K>
__device__ __forceinline__ Dual<K> atan2(const Dual<K>& y, const Dual<K>& x) {
  Dual<K> r;
  r.v = ::atan2(y.v, x.v);
  const double q = 1.0 / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * q;
  return r;
}

__device__ __forceinline__ double val(double a) { return a; }
template <int K>
__device__ __forceinline__ double val(const Dual<K>& a) { return a.v; }

template <typename S>
struct Lift {
  __device__ __forceinline__ static S of(double a) { return S(a); }
};
template <int K>
struct Lift<Dual<K>> {
  __device__ __forceinline__ static Dual<K> of(double a) { return dual_const<K>(a); }
};

// ---------------------------------------------------------------------------
// geometry of one ray step, templated on the scalar (double or dual)

template <typename S>
__device__ __forceinline__ S dot3s(const S a[3], const S b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
template <typename S>
__device__ __forceinline__ void cross3s(const S a[3], const S b[3], S c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
// (theta-hat, phi-hat) at unit vector n
template <typename S>
__device__ __forceinline__ void basis_s(const S n[3], S t[3], S p[3]) {
  const S rho = sqrt(n[0] * n[0] + n[1] * n[1]);
  t[0] = n[2] * n[0] / rho;
  t[1] = n[2] * n[1] / rho;
  t[2] = -rho;
  p[0] = -n[1] / rho;
  p[1] = n[0] / rho;
  p[2] = Lift<S>::of(0.0);
}
// rotate v about unit axis k by the angle with cosine c, sine s
template <typename S>
__device__ __forceinline__ void rodrigues_s(const S v[3], const S k[3], const S& c, const S& s, S o[3]) {
  S kv[3];
  cross3s(k, v, kv);
  const S kd = dot3s(k, v) * (1.0 - c);
#pragma unroll
  for (int i = 0; i < 3; ++i) o[i] = v[i] * c + kv[i] * s + k[i] * kd;
}
// transport matrix Q (2x2) from the tangent basis at n0 to the one at n1 (Appendix B)
template <typename S>
__device__ void transport_q_s(const S n0[3], const S n1[3], S Q[4]) {
  S cr[3];
  cross3s(n0, n1, cr);
  const S s = sqrt(dot3s(cr, cr));
  const S c = dot3s(n0, n1);
  S t0[3], p0[3], t1[3], p1[3], tr[3], pr[3];
  basis_s(n0, t0, p0);
  basis_s(n1, t1, p1);
  if (val(s) > 0.0) {
    const S k[3] = {cr[0] / s, cr[1] / s, cr[2] / s};
    rodrigues_s(t0, k, c, s, tr);
    rodrigues_s(p0, k, c, s, pr);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      tr[i] = t0[i];
      pr[i] = p0[i];
    }
  }
  Q[0] = dot3s(t1, tr);
  Q[1] = dot3s(t1, pr);
  Q[2] = dot3s(p1, tr);
  Q[3] = dot3s(p1, pr);
}
template <typename S>
__device__ __forceinline__ void qaqt_s(const S Q[4], const S A[4], S o[4]) {
  const S m0 = Q[0] * A[0] + Q[1] * A[2], m1 = Q[0] * A[1] + Q[1] * A[3];
  const S m2 = Q[2] * A[0] + Q[3] * A[2], m3 = Q[2] * A[1] + Q[3] * A[3];
  o[0] = m0 * Q[0] + m1 * Q[1];
  o[1] = m0 * Q[2] + m1 * Q[3];
  o[2] = m2 * Q[0] + m3 * Q[1];
  o[3] = m2 * Q[2] + m3 * Q[3];
}

struct StepC {
  double c, d, dchi2;
};

// One plane (Eq. Atraj, Eq. betaprop, Eq. posprop, Appendix B) given the
// lens values L = (alpha_t, alpha_p, U_tt, U_pp, U_tp) at the ray:
// out = x1[3], beta1[3], A^(n+1)[4], A^(n)[4] (both in the basis at x1).
template <typename S>
__device__ void step_eval(const S x[3], const S be[3], const S A[4], const S Ap[4], const S L[5], const StepC& sc,
                          S out[14]) {
  const S xn = sqrt(dot3s(x, x));
  const S nv[3] = {x[0] / xn, x[1] / xn, x[2] / xn};
  S An[4];
  An[0] = (1.0 - sc.c) * Ap[0] + sc.c * A[0] - sc.d * (L[2] * A[0] + L[4] * A[2]);
  An[1] = (1.0 - sc.c) * Ap[1] + sc.c * A[1] - sc.d * (L[2] * A[1] + L[4] * A[3]);
  An[2] = (1.0 - sc.c) * Ap[2] + sc.c * A[2] - sc.d * (L[4] * A[0] + L[3] * A[2]);
  An[3] = (1.0 - sc.c) * Ap[3] + sc.c * A[3] - sc.d * (L[4] * A[1] + L[3] * A[3]);
  S t[3], q[3];
  basis_s(nv, t, q);
  const S av[3] = {L[0] * t[0] + L[1] * q[0], L[0] * t[1] + L[1] * q[1], L[0] * t[2] + L[1] * q[2]};
  const S am = sqrt(dot3s(av, av));
  S bn[3] = {be[0], be[1], be[2]};
  if (val(am) > 0.0) {
    S kx[3];
    cross3s(nv, av, kx);
    const S kk[3] = {kx[0] / am, kx[1] / am, kx[2] / am};
    S sn, cs;
    sincos(am, &sn, &cs);
    rodrigues_s(be, kk, cs, sn, bn);
  }
  const S xb = dot3s(x, bn);
  const S lam = sc.dchi2 / (xb + sqrt(xb * xb + sc.dchi2));
  S x1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) x1[c] = x[c] + lam * bn[c];
  const S x1n = sqrt(dot3s(x1, x1));
  const S n1[3] = {x1[0] / x1n, x1[1] / x1n, x1[2] / x1n};
  S Q[4];
  transport_q_s(nv, n1, Q);
  qaqt_s(Q, An, out + 6);
  qaqt_s(Q, A, out + 10);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[c] = x1[c];
    out[3 + c] = bn[c];
  }
}

// ring pair bracketing phi on ring i with the fraction f (templated in phi)
template <typename S>
__device__ __forceinline__ void ring_pair_s(int nside, int i, const S& phi, int64_t* p0, int64_t* p1, S* f) {
  const Ring r = ring_geom(nside, i);
  const S t = (phi - r.phi0) * ((double)r.npix / (2.0 * kPi));
  const double j0 = floor(val(t));
  *f = t - j0;
  int64_t j = imod((int64_t)j0, r.npix);
  *p0 = r.first + j;
  *p1 = r.first + (j + 1 == r.npix ? 0 : j + 1);
}

// Ring-bilinear interpolation weights (with the polar blend) at (theta, phi),
// templated in the position: the pixels follow the values, the weights carry
// the tangents.
template <typename S>
struct InterpS {
  int64_t p[8];
  S w[8];
  int n;
};

template <typename S>
__device__ void interp_weights_s(int nside, const S& theta, const S& phi, InterpS<S>& o) {
  const double th = val(theta);
  int i1 = ring_above(nside, cos(th), 0.0);
  const int nr = 4 * nside - 1;
  while (i1 >= 1 && ring_theta(nside, i1) > th) --i1;
  while (i1 + 1 <= nr && ring_theta(nside, i1 + 1) <= th) ++i1;
  if (i1 == 0 || i1 == nr) {
    const int ir = (i1 == 0) ? 1 : nr;
    const double tr = ring_theta(nside, ir);
    const S w = (i1 == 0) ? theta / tr : (kPi - theta) / (kPi - tr);
    S fa;
    ring_pair_s(nside, ir, phi, &o.p[0], &o.p[1], &fa);
    o.w[0] = w * (1.0 - fa);
    o.w[1] = w * fa;
    const Ring r = ring_geom(nside, ir);
    for (int k = 0; k < 4; ++k) {
      o.p[2 + k] = r.first + k;
      o.w[2 + k] = (1.0 - w) * 0.25;
    }
    o.n = 6;
    return;
  }
  const double ta = ring_theta(nside, i1), tb = ring_theta(nside, i1 + 1);
  const S w = (theta - ta) / (tb - ta);
  S fa, fb;
  ring_pair_s(nside, i1, phi, &o.p[0], &o.p[1], &fa);
  ring_pair_s(nside, i1 + 1, phi, &o.p[2], &o.p[3], &fb);
  o.w[0] = (1.0 - w) * (1.0 - fa);
  o.w[1] = (1.0 - w) * fa;
  o.w[2] = w * (1.0 - fb);
  o.w[3] = w * fb;
  o.n = 4;
}

// tangent basis at a RING pixel centre
__device__ __forceinline__ void pixel_basis(int nside, int64_t p, double t[3], double q[3]) {
  int64_t j;
  const int i = pix2ring(nside, p, &j);
  const Ring r = ring_geom(nside, i);
  const double phi = r.phi0 + (2.0 * kPi) * (double)j / (double)r.npix;
  const double cp = cos(phi), sp = sin(phi);
  t[0] = r.z * cp;
  t[1] = r.z * sp;
  t[2] = -r.s;
  q[0] = -sp;
  q[1] = cp;
  q[2] = 0.0;
}

// Lens values at unit vector nv from the five RING maps: alpha as a tangent
// 3-vector and U as a tangent 3x3 tensor, interpolated and projected on the
// basis at nv (the ray step's lookup).
template <typename S>
__device__ void lens_eval(const clc_derivs& M, int nside, const S nv[3], S out[5]) {
  const S rho = sqrt(nv[0] * nv[0] + nv[1] * nv[1]);
  const S th = atan2(rho, nv[2]);
  S ph = atan2(nv[1], nv[0]);
  if (val(ph) < 0) ph = ph + 2.0 * kPi;
  InterpS<S> w;
  interp_weights_s(nside, th, ph, w);
  S a3[3], U3[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    a3[a] = Lift<S>::of(0.0);
#pragma unroll
    for (int b = 0; b < 3; ++b) U3[a][b] = Lift<S>::of(0.0);
  }
  for (int k = 0; k < w.n; ++k) {
    const int64_t p = w.p[k];
    double t[3], q[3];
    pixel_basis(nside, p, t, q);
    const double at = M.a_th[p], ap = M.a_ph[p], utt = M.u_tt[p], upp = M.u_pp[p], utp = M.u_tp[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      a3[a] = a3[a] + w.w[k] * (at * t[a] + ap * q[a]);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        U3[a][b] = U3[a][b] + w.w[k] * (utt * t[a] * t[b] + upp * q[a] * q[b] + utp * (t[a] * q[b] + q[a] * t[b]));
    }
  }
  S t[3], q[3];
  basis_s(nv, t, q);
  out[0] = dot3s(a3, t);
  out[1] = dot3s(a3, q);
  S Ut[3], Uq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Ut[a] = U3[a][0] * t[0] + U3[a][1] * t[1] + U3[a][2] * t[2];
    Uq[a] = U3[a][0] * q[0] + U3[a][1] * q[1] + U3[a][2] * q[2];
  }
  out[2] = dot3s(t, Ut);
  out[3] = dot3s(q, Uq);
  out[4] = dot3s(t, Uq);
}

// Adjoint of the lookup's linear dependence on the maps: the five adjoint
// maps receive, at each interpolation pixel, w_k P_k^T Lbar.
__device__ void lens_scatter(const clc_derivs& Mbar, int nside, const double nv[3], const double Lb[5]) {
  const double rho = ::sqrt(nv[0] * nv[0] + nv[1] * nv[1]);
  const double th = ::atan2(rho, nv[2]);
  double ph = ::atan2(nv[1], nv[0]);
  if (ph < 0) ph += 2.0 * kPi;
  InterpS<double> w;
  interp_weights_s(nside, th, ph, w);
  double t[3], q[3];
  basis_s(nv, t, q);
  for (int k = 0; k < w.n; ++k) {
    const int64_t p = w.p[k];
    double tk[3], qk[3];
    pixel_basis(nside, p, tk, qk);
    const double a = tk[0] * t[0] + tk[1] * t[1] + tk[2] * t[2];
    const double b = qk[0] * t[0] + qk[1] * t[1] + qk[2] * t[2];
    const double c = tk[0] * q[0] + tk[1] * q[1] + tk[2] * q[2];
    const double e = qk[0] * q[0] + qk[1] * q[1] + qk[2] * q[2];
    const double ww = w.w[k];
    atomicAdd(&Mbar.a_th[p], ww * (a * Lb[0] + c * Lb[1]));
    atomicAdd(&Mbar.a_ph[p], ww * (b * Lb[0] + e * Lb[1]));
    atomicAdd(&Mbar.u_tt[p], ww * (a * a * Lb[2] + c * c * Lb[3] + a * c * Lb[4]));
    atomicAdd(&Mbar.u_pp[p], ww * (b * b * Lb[2] + e * e * Lb[3] + b * e * Lb[4]));
    atomicAdd(&Mbar.u_tp[p], ww * (2.0 * a * b * Lb[2] + 2.0 * c * e * Lb[3] + (a * e + b * c) * Lb[4]));
  }
}

// ---------------------------------------------------------------------------
// SHT+MG lens lookup templated in the scalar (the galaxy rays' lookup in
// their home bundle's patch, Sec. 3.2): fourth-order finite differences on
// the finest patch level (one-sided stencils at the edge), the bilinear blend
// of the four cells around the point as one tensor-product stencil on a 6 x 6
// block, Appendix A in the patch basis and the rotation to the global basis
// at the point.  The position enters through the patch angles and the blend
// fractions, so dual numbers carry the lookup's dependence on the ray.

template <typename S>
__device__ __forceinline__ S asin_s(const S& x) {
  const S x2 = x * x;
  return x * (1.0 + x2 * ((1.0 / 6.0) + x2 * ((3.0 / 40.0) + x2 * ((5.0 / 112.0) + x2 * ((35.0 / 1152.0) +
              x2 * ((63.0 / 2816.0) + x2 * (231.0 / 13312.0)))))));
}

// six-point weights of the blend (1 - f) D_k + f D_{k+1} (x 12), first point returned
template <typename S>
__device__ __forceinline__ int fd_blend_s(int k, int n, const S& f, S w1[6], S w2[6]) {
  double a1[5], a2[5], b1[5], b2[5];
  const int ba = fd_stencil(k, n, 1, a1), bb = fd_stencil(k + 1, n, 1, b1);
  fd_stencil(k, n, 2, a2);
  fd_stencil(k + 1, n, 2, b2);
  const int first = min(ba, bb);
  const bool sa = ba > first, sb = bb > first;
  const S g = 1.0 - f;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const double A1 = sa ? (t >= 1 ? a1[t - 1] : 0.0) : (t < 5 ? a1[t] : 0.0);
    const double B1 = sb ? (t >= 1 ? b1[t - 1] : 0.0) : (t < 5 ? b1[t] : 0.0);
    const double A2 = sa ? (t >= 1 ? a2[t - 1] : 0.0) : (t < 5 ? a2[t] : 0.0);
    const double B2 = sb ? (t >= 1 ? b2[t - 1] : 0.0) : (t < 5 ? b2[t] : 0.0);
    w1[t] = g * A1 + f * B1;
    w2[t] = g * A2 + f * B2;
  }
  return first;
}

// position-dependent part of the lookup: patch angles, blend weights
template <typename S>
struct PatchGeo {
  S v[3];            // patch-frame unit vector
  S rho, is, sp, cp; // sin theta', 1 / sin theta', sin phi', cos phi'
  S A1[6], A2[6], B1[6], B2[6], Rx[6], Cy[6];
  int r0, c0;        // first row / column of the 6 x 6 block (interior cell indices)
};

template <typename S>
__device__ void patch_geo(const MGView& V, int b, const S nv[3], PatchGeo<S>& G) {
  const int n = V.n;
  const double* R = V.rot + 9 * (size_t)b;
#pragma unroll
  for (int r = 0; r < 3; ++r) G.v[r] = R[3 * r] * nv[0] + R[3 * r + 1] * nv[1] + R[3 * r + 2] * nv[2];
  G.rho = sqrt(G.v[0] * G.v[0] + G.v[1] * G.v[1]);
  G.is = 1.0 / G.rho;
  G.sp = G.v[1] * G.is;
  G.cp = G.v[0] * G.is;
  S dth, php;
  if (fabs(val(G.v[2])) < 0.04 && fabs(val(G.sp)) < 0.04 && val(G.v[0]) > 0.0) {
    dth = -asin_s(G.v[2]);
    php = asin_s(G.sp);
  } else {
    dth = atan2(G.rho, G.v[2]) - 0.5 * kPi;
    php = atan2(G.v[1], G.v[0]);
  }
  const S x = dth * V.inv_h + (0.5 * n - 0.5);
  const S y = php * V.inv_h + (0.5 * n - 0.5);
  int ii = (int)floor(val(x)), jj = (int)floor(val(y));
  ii = min(max(ii, 0), n - 2);
  jj = min(max(jj, 0), n - 2);
  const S fx = x - (double)ii, fy = y - (double)jj;
  G.r0 = fd_blend_s(ii, n, fx, G.A1, G.A2);
  G.c0 = fd_blend_s(jj, n, fy, G.B1, G.B2);
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    G.Rx[t] = Lift<S>::of(0.0);
    G.Cy[t] = Lift<S>::of(0.0);
  }
  // bilinear weights of cells ii, ii + 1 (rows) and jj, jj + 1 (columns) in the block
  for (int t = 0; t < 6; ++t) {
    if (t == ii - G.r0) G.Rx[t] = 1.0 - fx;
    if (t == ii - G.r0 + 1) G.Rx[t] = fx;
    if (t == jj - G.c0) G.Cy[t] = 1.0 - fy;
    if (t == jj - G.c0 + 1) G.Cy[t] = fy;
  }
}

// lens fields at the point from the five patch partials (x 12 stencil sums)
// P = (pt, pp, ptt, ppp, ptp): Appendix A in the patch basis, then alpha and
// U rotated to the basis (et, ep) at nv
template <typename S, typename P>
__device__ void fields_from_partials(const MGView& V, int b, const PatchGeo<S>& G, const P pr[5], const S et[3],
                                     const S ep[3], P out[5]) {
  const double* R = V.rot + 9 * (size_t)b;
  const double c1 = V.inv_h / 12.0, c2 = c1 * V.inv_h;
  const P v0 = pr[0] * c1, v1 = pr[1] * c1, v2 = pr[2] * c2, v3 = pr[3] * c2, v4 = pr[4] * (c1 * c1);
  const S co = G.v[2];
  const P a_t = -v0, a_p = -(v1 * G.is);
  const P u_tt = v2;
  const P u_pp = (v3 * G.is + co * v0) * G.is;
  const P u_tp = (v4 - co * v1 * G.is) * G.is;
  const S tl[3] = {co * G.cp, co * G.sp, -G.rho};
  S tg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) tg[k] = R[k] * tl[0] + R[3 + k] * tl[1] + R[6 + k] * tl[2];
  const S q00 = et[0] * tg[0] + et[1] * tg[1] + et[2] * tg[2];
  const S q10 = ep[0] * tg[0] + ep[1] * tg[1] + ep[2] * tg[2];
  out[0] = q00 * a_t - q10 * a_p;
  out[1] = q10 * a_t + q00 * a_p;
  const P m00 = q00 * u_tt - q10 * u_tp, m01 = q00 * u_tp - q10 * u_pp;
  const P m10 = q10 * u_tt + q00 * u_tp, m11 = q10 * u_tp + q00 * u_pp;
  out[2] = m00 * q00 - m01 * q10;
  out[3] = m10 * q10 + m11 * q00;
  out[4] = m00 * q10 + m01 * q00;
}

// Lens values at nv in patch slot b (double or dual scalar)
template <typename S>
__device__ void patch_eval(const MGView& V, int b, const S nv[3], S out[5]) {
  PatchGeo<S> G;
  patch_geo(V, b, nv, G);
  const int n = V.n;
  const double* ub = V.u + (size_t)(n + 2) * (n + 2) * b + (size_t)(G.r0 + 1) * (n + 2) + (G.c0 + 1);
  S c[6], mix[6], rr[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) rr[t] = Lift<S>::of(0.0);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const double* row = ub + (size_t)a * (n + 2);
    S ca = Lift<S>::of(0.0), ma = Lift<S>::of(0.0);
#pragma unroll
    for (int bb = 0; bb < 6; ++bb) {
      ca = ca + G.Cy[bb] * row[bb];
      ma = ma + G.B1[bb] * row[bb];
      rr[bb] = rr[bb] + G.Rx[a] * row[bb];
    }
    c[a] = ca;
    mix[a] = ma;
  }
  S pr[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) pr[q] = Lift<S>::of(0.0);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    pr[0] = pr[0] + G.A1[a] * c[a];      // pt
    pr[2] = pr[2] + G.A2[a] * c[a];      // ptt
    pr[4] = pr[4] + G.A1[a] * mix[a];    // ptp
    pr[1] = pr[1] + G.B1[a] * rr[a];     // pp
    pr[3] = pr[3] + G.B2[a] * rr[a];     // ppp
  }
  S et[3], ep[3];
  basis_s(nv, et, ep);
  fields_from_partials<S, S>(V, b, G, pr, et, ep, out);
}

// Adjoint of the lookup's linear dependence on the patch potential: the five
// lens adjoints Lb at nv become adjoints of the five partials (dual numbers
// seeded on the partials give the Jacobian of fields_from_partials), which
// the tensor-product stencils spread over the 6 x 6 block of ubar.
__device__ void patch_scatter(const MGView& V, int b, const double nv[3], const double Lb[5], double* ubar) {
  typedef Dual<5> D5;
  PatchGeo<double> G;
  patch_geo(V, b, nv, G);
  double et[3], ep[3];
  basis_s(nv, et, ep);
  D5 pr[5], out[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    pr[q] = dual_const<5>(0.0);
    pr[q].d[q] = 1.0;
  }
  fields_from_partials<double, D5>(V, b, G, pr, et, ep, out);
  double pb[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 5; ++c) acc += Lb[c] * out[c].d[q];
    pb[q] = acc;
  }
  const int n = V.n;
  double* ub = ubar + (size_t)n * n * b + (size_t)G.r0 * n + G.c0;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int bb = 0; bb < 6; ++bb) {
      const double g = pb[0] * G.A1[a] * G.Cy[bb] + pb[2] * G.A2[a] * G.Cy[bb] + pb[4] * G.A1[a] * G.B1[bb] +
                       pb[1] * G.Rx[a] * G.B1[bb] + pb[3] * G.Rx[a] * G.B2[bb];
      if (g != 0.0) atomicAdd(ub + (size_t)a * n + bb, g);
    }
}

// ---------------------------------------------------------------------------
// kernels

struct RaySoA {
  double* s;      // [14][n]: x, beta, A, Ap
  int64_t n;
};

__global__ void k_gal_init(const double* __restrict__ z, const double* __restrict__ phi,
                           const double* __restrict__ gchi, const double* __restrict__ chi, int N, double* st, int64_t n,
                           int* __restrict__ bin, double* __restrict__ tw, int nb, int32_t* __restrict__ bundle) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double zz = z[k], pp = phi[k];
    if (nb > 0) bundle[k] = (int32_t)ang2pix_nest(nb, zz, pp);   // the ray keeps its start bundle (Sec. 3.1)
    const double s = sqrt((1.0 - zz) * (1.0 + zz));
    const double v[3] = {s * cos(pp), s * sin(pp), zz};
    for (int c = 0; c < 3; ++c) {
      st[c * n + k] = chi[0] * v[c];
      st[(3 + c) * n + k] = v[c];
    }
    const double I[4] = {1.0, 0.0, 0.0, 1.0};
    for (int c = 0; c < 4; ++c) {
      st[(6 + c) * n + k] = I[c];
      st[(10 + c) * n + k] = I[c];
    }
    const double g = gchi[k];
    int b = -1;
    if (g >= chi[0]) {
      b = 0;
      while (b + 1 < N && g >= chi[b + 1]) ++b;
    }
    bin[k] = b;
    tw[k] = b >= 0 ? (chi[b + 1] / g) * ((g - chi[b]) / (chi[b + 1] - chi[b])) : 0.0;
  }
}

// lens source of a plane: RING maps of nside (pure SHT) or the SHT+MG patches
struct LensSrc {
  clc_derivs M;
  int nside;
  MGView V;
  const int32_t* bundle;
};

template <bool kMG, typename S>
__device__ __forceinline__ void lens_at(const LensSrc& src, int64_t k, const S nv[3], S L[5]) {
  if (kMG) {
    const int slot = mg_slot(src.V, src.bundle[k]);
    if (slot >= 0) {
      patch_eval<S>(src.V, slot, nv, L);
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c) L[c] = Lift<S>::of(0.0);   // outside a partial sky's domain
    }
  } else {
    lens_eval<S>(src.M, src.nside, nv, L);
  }
}

template <bool kMG>
__global__ void k_gal_step(double* st, int64_t n, LensSrc src, StepC sc, const int* __restrict__ bin,
                           const double* __restrict__ tw, int plane, double* __restrict__ gamma) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double in[14], o[14];
#pragma unroll
    for (int c = 0; c < 14; ++c) in[c] = st[c * n + k];
    const double xn = ::sqrt(in[0] * in[0] + in[1] * in[1] + in[2] * in[2]);
    const double nv[3] = {in[0] / xn, in[1] / xn, in[2] / xn};
    double L[5];
    lens_at<kMG, double>(src, k, nv, L);
    step_eval<double>(in, in + 3, in + 6, in + 10, L, sc, o);
#pragma unroll
    for (int c = 0; c < 14; ++c) st[c * n + k] = o[c];
    if (bin[k] == plane) {
      const double t = tw[k];
      double Ag[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) Ag[c] = (1.0 - t) * o[10 + c] + t * o[6 + c];
      gamma[k] = -0.5 * (Ag[0] - Ag[3]);
      gamma[n + k] = -0.5 * (Ag[1] + Ag[2]);
    }
  }
}

// Reverse of one plane.  adj[14][n] holds the adjoint of the state leaving
// the plane on entry and of the state entering it on return.
constexpr int kDualK = 5;

template <bool kMG>
__global__ void __launch_bounds__(128) k_gal_step_adjoint(const double* __restrict__ ck, double* adj, int64_t n,
                                                          LensSrc src, clc_derivs Mbar, double* ubar, StepC sc,
                                                          const int* __restrict__ bin, const double* __restrict__ tw,
                                                          int plane, const double* __restrict__ gbar) {
  typedef Dual<kDualK> D;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double v[14];
#pragma unroll
    for (int c = 0; c < 14; ++c) v[c] = adj[c * n + k];
    if (bin[k] == plane) {
      // gamma_1 = -(A_g00 - A_g11) / 2, gamma_2 = -(A_g01 + A_g10) / 2, A_g = (1 - t) A^(n) + t A^(n+1)
      const double g1 = gbar[k], g2 = gbar[n + k], t = tw[k];
      const double Ab[4] = {-0.5 * g1, -0.5 * g2, -0.5 * g2, 0.5 * g1};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        v[6 + c] += t * Ab[c];
        v[10 + c] += (1.0 - t) * Ab[c];
      }
    }
    double in0[14];
#pragma unroll
    for (int c = 0; c < 14; ++c) in0[c] = ck[c * n + k];
    double ib[14], Lb[5];
    // directions 0..13: entering state; 14..18: the five lens values
    for (int d0 = 0; d0 < 19; d0 += kDualK) {
      D in[14];
#pragma unroll
      for (int c = 0; c < 14; ++c) {
        in[c] = dual_const<kDualK>(in0[c]);
#pragma unroll
        for (int j = 0; j < kDualK; ++j) in[c].d[j] = (d0 + j == c) ? 1.0 : 0.0;
      }
      const D xn = sqrt(in[0] * in[0] + in[1] * in[1] + in[2] * in[2]);
      const D nv[3] = {in[0] / xn, in[1] / xn, in[2] / xn};
      D L[5];
      lens_at<kMG, D>(src, k, nv, L);
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int j = 0; j < kDualK; ++j)
          if (d0 + j == 14 + c) L[c].d[j] += 1.0;
      D o[14];
      step_eval<D>(in, in + 3, in + 6, in + 10, L, sc, o);
#pragma unroll
      for (int j = 0; j < kDualK; ++j) {
        const int dir = d0 + j;
        if (dir >= 19) break;
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 14; ++c) acc += v[c] * o[c].d[j];
        if (dir < 14) ib[dir] = acc;
        else Lb[dir - 14] = acc;
      }
    }
#pragma unroll
    for (int c = 0; c < 14; ++c) adj[c * n + k] = ib[c];
    const double xn = ::sqrt(in0[0] * in0[0] + in0[1] * in0[1] + in0[2] * in0[2]);
    const double nv[3] = {in0[0] / xn, in0[1] / xn, in0[2] / xn};
    if (kMG) {
      const int slot = src.V.slot ? src.V.slot[src.bundle[k]] : src.bundle[k];
      if (slot >= 0) patch_scatter(src.V, slot, nv, Lb, ubar);
    } else {
      lens_scatter(Mbar, src.nside, nv, Lb);
    }
  }
}

// adjoint of the degrade to the SHT grid (mean of k children): every fine
// RING pixel receives its coarse parent's adjoint / k
__global__ void k_degrade_adjoint(const double* __restrict__ coarse_bar, int ns, int nf, double* __restrict__ fine_bar) {
  const int64_t np = 12ll * nf * nf;
  const int shift = 2 * (ilog2(nf) - ilog2(ns));
  const double inv = 1.0 / (double)(1ll << shift);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t j;
    const int i = pix2ring(nf, p, &j);
    const int64_t parent = nest2ring(ns, ring_pos2nest(nf, i, j) >> shift);
    fine_bar[p] += coarse_bar[parent] * inv;
  }
}

// ---- adjoint of the SHT Poisson solve with derivative outputs

// Adjoint of the per-ring combinations of the synthesis: from the adjoint
// ring spectra of alpha_t, alpha_p, u_tt, u_pp, u_tp (already scaled by
// 2 - delta_m0) to the adjoint Legendre sums of psi, b and kappa_bl.
__global__ void k_spec_adjoint(int nside, int lmax, const double2* __restrict__ Fb, size_t fq, int ldf,
                               double2* __restrict__ Gb, size_t gq) {
  const int m = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < 4 * nside - 1; r += gridDim.x * blockDim.x) {
    const Ring g = ring_geom(nside, r + 1);
    const double is = 1.0 / g.s, is2 = is * is, c = g.z, dm = (double)m;
    const double f = m == 0 ? 1.0 : 2.0;
    double2 s[5];
    for (int q = 0; q < 5; ++q) {
      const double2 v = Fb[q * fq + (size_t)m * ldf + r];
      s[q] = make_double2(f * v.x, m == 0 ? 0.0 : f * v.y);
    }
    // conj(C) for alpha_p = -i m is g0, u_tt = g2 - (-m^2 g0 + c g1) is2,
    // u_pp = (-m^2 g0 + c g1) is2, u_tp = i m is2 (g1 - c g0), alpha_t = -is g1
    const double2 sa = s[0], sp = s[1], stt = s[2], spp = s[3], stp = s[4];
    double2 G0, G1, G2;
    // i m is sp + m^2 is2 (stt - spp) + i m c is2 stp
    G0.x = -dm * is * sp.y + dm * dm * is2 * (stt.x - spp.x) - dm * c * is2 * stp.y;
    G0.y = dm * is * sp.x + dm * dm * is2 * (stt.y - spp.y) + dm * c * is2 * stp.x;
    // -is sa - c is2 stt + c is2 spp - i m is2 stp
    G1.x = -is * sa.x - c * is2 * stt.x + c * is2 * spp.x + dm * is2 * stp.y;
    G1.y = -is * sa.y - c * is2 * stt.y + c * is2 * spp.y - dm * is2 * stp.x;
    G2 = stt;
    Gb[(size_t)m * ldf + r] = G0;
    Gb[gq + (size_t)m * ldf + r] = G1;
    Gb[2 * gq + (size_t)m * ldf + r] = G2;
  }
}

// Adjoint of the Poisson solve and of the rhs construction: from the adjoint
// right-hand sides (psi, b, kappa_bl; band limit lmax + 1 packing) to the
// coefficients whose (weighted) synthesis is the gradient map.
__global__ void k_poisson_adjoint(const double2* __restrict__ rb, long long Q, int lmax, double weight,
                                  double2* __restrict__ out) {
  const int m = blockIdx.y;
  const int lt = lmax + 1;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  auto eps = [&](int ll) -> double {
    if (ll <= m) return 0.0;
    return sqrt(((double)ll * ll - (double)m * m) / (4.0 * ll * ll - 1.0));
  };
  double2 r = make_double2(0.0, 0.0);
  if (l >= 1) {
    const double2 r0 = rb[alm_idx(lt, l, m)];
    const double2 r2 = rb[2 * Q + alm_idx(lt, l, m)];
    const double ll1 = (double)l * (l + 1.0);
    // psi_l enters rhs_1 at l + 1 with c1(l + 1) = l eps_{l+1} and at l - 1 with -c2(l - 1) = -(l + 1) eps_l
    const double2 up = rb[Q + alm_idx(lt, l + 1, m)];
    double2 dn = make_double2(0.0, 0.0);
    if (l - 1 >= m) dn = rb[Q + alm_idx(lt, l - 1, m)];
    const double c1 = (double)l * eps(l + 1), c2 = (l + 1.0) * eps(l);
    const double px = r0.x + c1 * up.x - c2 * dn.x - ll1 * r2.x;
    const double py = r0.y + c1 * up.y - c2 * dn.y - ll1 * r2.y;
    // kappa_lm -> psi_lm = -kappa_lm / (l (l + 1)); analysis adjoint: weight w, m > 0 halved for the synthesis
    const double s = -weight / ll1 / (m == 0 ? 1.0 : 2.0);
    r = make_double2(s * px, m == 0 ? 0.0 : s * py);
  }
  out[alm_idx(lmax, l, m)] = r;
}

// ---------------------------------------------------------------------------
// host

static int launch_blocks(clc_ctx* ctx, int64_t n, int threads, int per_sm) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms(ctx) * per_sm;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace clc

using namespace clc;

struct clc_gal_tape {
  clc_ctx* ctx = nullptr;
  int N = 0, nside = 0, lmax = 0, precision = CLC_FP64;
  int solver = CLC_SOLVER_SHT;
  clc_mg_params mg{};                 // CLC_SOLVER_SHTMG: the plane solver's parameters
  clc_plane_solution* sol = nullptr;  // CLC_SOLVER_SHTMG: one plane's multigrid state, reused
  int64_t n = 0;
  std::vector<double> chi;
  std::vector<const double*> kappa;
  Buffer d_chi, state, ckpt, adj, bin, tw, maps, fbar, work, bundle, ubar, psibar, kbar_s;
  ~clc_gal_tape() {
    if (sol) clc_solution_destroy(sol);
  }
};

static int sht_poisson_adjoint(clc_gal_tape* T, const clc_derivs& Fb, double* kbar) {
  clc_ctx* ctx = T->ctx;
  const int ns = T->nside, L = T->lmax;
  int rc;
  auto plan = get_fft_plan(ctx, ns, &rc);
  if (rc) return rc;
  auto tab = get_legendre_table(ctx, ns, L, &rc);
  if (rc) return rc;
  const int ldf = 4 * ns - 1;
  const size_t fq = (size_t)ldf * (L + 1);
  const long long Q = alm_idx(L + 1, L + 1, L + 1) + 1;
  const size_t nalm = (size_t)(L + 1) * (L + 2) / 2;
  const size_t bytes = sizeof(double2) * (5 * fq + 3 * fq + 3 * (size_t)Q + nalm);
  if (T->work.bytes < bytes) {
    if (T->work.p) cudaFree(T->work.p);
    T->work.p = nullptr;
    T->work.bytes = 0;
    if (cudaMalloc(&T->work.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, CLC_ENOMEM, "adjoint SHT work space");
    }
    T->work.bytes = bytes;
  }
  double2* Fh = (double2*)T->work.p;
  double2* Gb = Fh + 5 * fq;
  double2* rb = Gb + 3 * fq;
  double2* kt = rb + 3 * Q;
  const double* maps[5] = {Fb.a_th, Fb.a_ph, Fb.u_tt, Fb.u_pp, Fb.u_tp};
  // transposed ring synthesis: ring analysis without quadrature weight
  for (int f = 0; f < 5; ++f)
    if ((rc = ring_analysis(ctx, *plan, maps[f], L, 1.0, Fh + f * fq, ldf))) return rc;
  dim3 g1((4 * ns - 1 + 127) / 128, L + 1);
  CLC_LAUNCH(ctx, "k_spec_adjoint", k_spec_adjoint, g1, 128, 0, ns, L, Fh, fq, ldf, Gb, fq);
  if ((rc = launch_check(ctx, "k_spec_adjoint"))) return rc;
  // transposed Legendre synthesis: Legendre analysis up to l = lmax + 1
  for (int q = 0; q < 3; ++q)
    if ((rc = legendre_analysis(ctx, *tab, Gb + q * fq, ldf, rb + q * Q, L + 1))) return rc;
  dim3 g2((L + 1 + 127) / 128, L + 1);
  const double w = 4.0 * kPi / (12.0 * (double)ns * ns);
  CLC_LAUNCH(ctx, "k_poisson_adjoint", k_poisson_adjoint, g2, 128, 0, rb, Q, L, w, kt);
  if ((rc = launch_check(ctx, "k_poisson_adjoint"))) return rc;
  // transposed analysis: weighted synthesis
  return clc_sht_synthesis(ctx, (const double*)kt, ns, L, kbar);
}

static bool tape_alloc(Buffer& b, size_t bytes) {
  b.bytes = bytes;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    b.bytes = 0;
    return false;
  }
  return true;
}

static StepC step_coef(const std::vector<double>& chi, int m) {
  StepC sc;
  const double cp = m > 0 ? chi[m - 1] : 0.0, cn = chi[m], cx = chi[m + 1];
  sc.c = (cn / cx) * ((cx - cp) / (cn - cp));
  sc.d = (cx - cn) / cx;
  sc.dchi2 = cx * cx - cn * cn;
  return sc;
}

// the lens source of plane m: its maps (pure SHT) or its patch solution
static int plane_lens(clc_gal_tape* T, int m, LensSrc* src) {
  clc_ctx* ctx = T->ctx;
  if (T->solver == CLC_SOLVER_SHT) {
    const size_t np = 12ull * T->nside * T->nside;
    double* mp = (double*)T->maps.p;
    src->M = clc_derivs{mp, mp + np, mp + 2 * np, mp + 3 * np, mp + 4 * np};
    src->nside = T->nside;
    src->bundle = nullptr;
    return clc_poisson_sht(ctx, T->kappa[m], T->nside, T->lmax, T->precision, nullptr, &src->M);
  }
  int rc = clc_poisson_shtmg(ctx, T->kappa[m], T->nside, &T->mg, T->sol, nullptr);
  if (rc != CLC_OK && rc != CLC_ENOTCONVERGED) return rc;
  src->M = clc_derivs{};
  src->nside = 0;
  src->V = mg_view(T->sol);
  src->bundle = (const int32_t*)T->bundle.p;
  return CLC_OK;
}

static int gal_trace(std::unique_ptr<clc_gal_tape> T, const double* gz, const double* gphi, const double* gchi,
                     double* gamma, clc_gal_tape** tape_out) {
  clc_ctx* ctx = T->ctx;
  const int N = T->N;
  const int64_t ngal = T->n;
  const size_t nn = (size_t)std::max<int64_t>(ngal, 1);
  const bool keep = tape_out != nullptr;
  const bool mg = T->solver == CLC_SOLVER_SHTMG;
  if (!tape_alloc(T->d_chi, sizeof(double) * (N + 1)) || !tape_alloc(T->state, sizeof(double) * 14 * nn) ||
      !tape_alloc(T->bin, sizeof(int) * nn) || !tape_alloc(T->tw, sizeof(double) * nn) ||
      (!mg && !tape_alloc(T->maps, sizeof(double) * 5 * 12ull * T->nside * T->nside)) ||
      (mg && !tape_alloc(T->bundle, sizeof(int32_t) * nn)) ||
      (keep && !tape_alloc(T->ckpt, sizeof(double) * 14 * nn * N)))
    return set_err(ctx, CLC_ENOMEM, "clc_gal_trace: allocation failed");
  int rc;
  if (mg && (rc = clc_solution_create(ctx, T->nside, &T->mg, &T->sol))) return rc;
  if ((rc = cuda_check(ctx, cudaMemcpyAsync(T->d_chi.p, T->chi.data(), sizeof(double) * (N + 1),
                                            cudaMemcpyHostToDevice, ctx->stream), "chi upload")))
    return rc;
  if (ngal > 0) {
    cudaMemsetAsync(gamma, 0, sizeof(double) * 2 * ngal, ctx->stream);
    CLC_LAUNCH(ctx, "k_gal_init", k_gal_init, launch_blocks(ctx, ngal, 256, 16), 256, 0, gz, gphi, gchi,
               (const double*)T->d_chi.p, N, (double*)T->state.p, ngal, (int*)T->bin.p, (double*)T->tw.p,
               mg ? T->mg.nside_bundle : 0, (int32_t*)T->bundle.p);
    if ((rc = launch_check(ctx, "k_gal_init"))) return rc;
  }
  int status = CLC_OK;
  for (int m = 0; m < N; ++m) {
    LensSrc src;
    if ((rc = plane_lens(T.get(), m, &src))) return rc;
    if (mg && T->sol->residual >= T->mg.tol && T->mg.fixed_cycles == 0) status = CLC_ENOTCONVERGED;
    if (ngal == 0) continue;
    if (keep)
      cudaMemcpyAsync((double*)T->ckpt.p + (size_t)m * 14 * ngal, T->state.p, sizeof(double) * 14 * ngal,
                      cudaMemcpyDeviceToDevice, ctx->stream);
    const StepC sc = step_coef(T->chi, m);
    if (mg)
      CLC_LAUNCH(ctx, "k_gal_step", k_gal_step<true>, launch_blocks(ctx, ngal, 128, 16), 128, 0,
                 (double*)T->state.p, ngal, src, sc, (const int*)T->bin.p, (const double*)T->tw.p, m, gamma);
    else
      CLC_LAUNCH(ctx, "k_gal_step", k_gal_step<false>, launch_blocks(ctx, ngal, 128, 16), 128, 0,
                 (double*)T->state.p, ngal, src, sc, (const int*)T->bin.p, (const double*)T->tw.p, m, gamma);
    if ((rc = launch_check(ctx, "k_gal_step"))) return rc;
  }
  if (keep) *tape_out = T.release();
  else if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "gal trace"))) return rc;
  return status == CLC_OK ? CLC_OK : set_err(ctx, status, "clc_gal_trace: an SHT+MG plane stopped above tol");
}

static std::unique_ptr<clc_gal_tape> new_tape(clc_ctx* ctx, int nplanes, const double* const* kappa, int nside,
                                              const double* chi, int64_t ngal) {
  auto T = std::make_unique<clc_gal_tape>();
  T->ctx = ctx;
  T->N = nplanes;
  T->nside = nside;
  T->n = ngal;
  T->chi.assign(chi, chi + nplanes + 1);
  T->kappa.assign(kappa, kappa + nplanes);
  return T;
}

static int check_gal_args(clc_ctx* ctx, int nplanes, const double* const* kappa, const double* chi, int64_t ngal,
                          const double* gz, const double* gphi, const double* gchi, double* gamma) {
  if (nplanes < 1 || !kappa || !chi || ngal < 0 || (ngal > 0 && (!gz || !gphi || !gchi || !gamma)))
    return set_err(ctx, CLC_EINVAL, "clc_gal_trace: bad arguments");
  for (int m = 0; m < nplanes; ++m)
    if (!kappa[m] || !(chi[m] > 0) || !(chi[m + 1] > chi[m]))
      return set_err(ctx, CLC_EINVAL, "clc_gal_trace: null plane or non-increasing chi");
  return CLC_OK;
}

extern "C" int clc_gal_trace(clc_ctx* ctx, int nplanes, const double* const* kappa, int nside, int lmax,
                             int precision, const double* chi, int64_t ngal, const double* gz, const double* gphi,
                             const double* gchi, double* gamma, clc_gal_tape** tape_out) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_gal_args(ctx, nplanes, kappa, chi, ngal, gz, gphi, gchi, gamma);
  if (rc) return rc;
  if (!valid_nside(nside) || nside > 4096 || lmax < 1 || lmax > 4 * nside ||
      (precision != CLC_FP64 && precision != CLC_MIXED))
    return set_err(ctx, CLC_EINVAL, "clc_gal_trace: bad arguments");
  cudaSetDevice(ctx->device);
  auto T = new_tape(ctx, nplanes, kappa, nside, chi, ngal);
  T->lmax = lmax;
  T->precision = precision;
  return gal_trace(std::move(T), gz, gphi, gchi, gamma, tape_out);
}

extern "C" int clc_gal_trace_mg(clc_ctx* ctx, int nplanes, const double* const* kappa, int nside,
                                const clc_mg_params* params, const double* chi, int64_t ngal, const double* gz,
                                const double* gphi, const double* gchi, double* gamma, clc_gal_tape** tape_out) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_gal_args(ctx, nplanes, kappa, chi, ngal, gz, gphi, gchi, gamma);
  if (rc) return rc;
  if (!params || params->precision != CLC_FP64 || !valid_nside(nside))
    return set_err(ctx, CLC_EINVAL, "clc_gal_trace_mg: needs CLC_FP64 MG parameters");
  cudaSetDevice(ctx->device);
  auto T = new_tape(ctx, nplanes, kappa, nside, chi, ngal);
  T->solver = CLC_SOLVER_SHTMG;
  T->mg = *params;
  T->lmax = params->lmax;
  T->precision = CLC_FP64;
  return gal_trace(std::move(T), gz, gphi, gchi, gamma, tape_out);
}

// adjoint of one SHT+MG plane's solve: ubar (patch interiors) -> kappa_bar
static int shtmg_adjoint(clc_gal_tape* T, double* kbar) {
  clc_ctx* ctx = T->ctx;
  clc_plane_solution* S = T->sol;
  const int nf = T->nside, ns = T->mg.nside_sht;
  const int64_t nf2 = 12ll * nf * nf, ns2 = 12ll * ns * ns;
  cudaMemsetAsync(kbar, 0, sizeof(double) * nf2, ctx->stream);
  cudaMemsetAsync(T->psibar.p, 0, sizeof(double) * ns2, ctx->stream);
  // the adjoint solve stops two orders below the forward tolerance (or at
  // 1e-12), so that it is no less converged than the forward solve
  const double tol = std::min(T->mg.tol * 1e-2, 1e-12);
  int rc = mg_adjoint_solve(ctx, S, (const double*)T->ubar.p, tol, std::max(T->mg.max_cycles, 40), kbar,
                            (double*)T->psibar.p, nullptr, nullptr);
  if (rc != CLC_OK && rc != CLC_ENOTCONVERGED) return rc;
  const int st = rc;
  // the SHT potential's dependence on kappa_sht: the psi-only SHT Poisson
  // solve (analysis, -1 / l(l+1), synthesis) is symmetric, so its adjoint is
  // the same solve; then the transposed degrade
  if ((rc = clc_poisson_sht(ctx, (const double*)T->psibar.p, ns, T->mg.lmax, CLC_FP64, (double*)T->kbar_s.p,
                            nullptr)))
    return rc;
  CLC_LAUNCH(ctx, "k_degrade_adjoint", k_degrade_adjoint, launch_blocks(ctx, nf2, 256, 16), 256, 0,
             (const double*)T->kbar_s.p, ns, nf, kbar);
  if ((rc = launch_check(ctx, "k_degrade_adjoint"))) return rc;
  return st;
}

extern "C" int clc_gal_trace_adjoint(clc_gal_tape* T, const double* gamma_bar, double* const* kappa_bar) {
  if (!T || !T->ctx) return CLC_EINVAL;
  clc_ctx* ctx = T->ctx;
  if (!gamma_bar || !kappa_bar || !T->ckpt.p) return set_err(ctx, CLC_EINVAL, "clc_gal_trace_adjoint: bad arguments");
  for (int m = 0; m < T->N; ++m)
    if (!kappa_bar[m]) return set_err(ctx, CLC_EINVAL, "clc_gal_trace_adjoint: null gradient map");
  cudaSetDevice(ctx->device);
  const bool mg = T->solver == CLC_SOLVER_SHTMG;
  const int ns = T->nside;
  const size_t np = 12ull * ns * ns;
  const int64_t n = T->n;
  int rc;
  if (!T->adj.p && !tape_alloc(T->adj, sizeof(double) * 14 * (size_t)std::max<int64_t>(n, 1)))
    return set_err(ctx, CLC_ENOMEM, "adjoint state");
  if (!mg && !T->fbar.p && !tape_alloc(T->fbar, sizeof(double) * 5 * np))
    return set_err(ctx, CLC_ENOMEM, "adjoint maps");
  if (mg && !T->ubar.p) {
    const size_t nc = (size_t)T->mg.ncell;
    const size_t ns2 = 12ull * T->mg.nside_sht * T->mg.nside_sht;
    if (!tape_alloc(T->ubar, sizeof(double) * nc * nc * T->sol->npatch) || !tape_alloc(T->psibar, sizeof(double) * ns2) ||
        !tape_alloc(T->kbar_s, sizeof(double) * ns2))
      return set_err(ctx, CLC_ENOMEM, "SHT+MG adjoint buffers");
  }
  cudaMemsetAsync(T->adj.p, 0, T->adj.bytes, ctx->stream);
  double* fp = (double*)T->fbar.p;
  clc_derivs db{};
  if (!mg) db = clc_derivs{fp, fp + np, fp + 2 * np, fp + 3 * np, fp + 4 * np};
  int status = CLC_OK;
  for (int m = T->N - 1; m >= 0; --m) {
    // recompute the plane's lens fields from its convergence map
    LensSrc src;
    if ((rc = plane_lens(T, m, &src))) return rc;
    if (mg) cudaMemsetAsync(T->ubar.p, 0, T->ubar.bytes, ctx->stream);
    else cudaMemsetAsync(fp, 0, T->fbar.bytes, ctx->stream);
    if (n > 0) {
      const StepC sc = step_coef(T->chi, m);
      const double* ck = (const double*)T->ckpt.p + (size_t)m * 14 * n;
      if (mg)
        CLC_LAUNCH(ctx, "k_gal_step_adjoint", k_gal_step_adjoint<true>, launch_blocks(ctx, n, 128, 16), 128, 0, ck,
                   (double*)T->adj.p, n, src, db, (double*)T->ubar.p, sc, (const int*)T->bin.p,
                   (const double*)T->tw.p, m, gamma_bar);
      else
        CLC_LAUNCH(ctx, "k_gal_step_adjoint", k_gal_step_adjoint<false>, launch_blocks(ctx, n, 128, 16), 128, 0, ck,
                   (double*)T->adj.p, n, src, db, (double*)nullptr, sc, (const int*)T->bin.p,
                   (const double*)T->tw.p, m, gamma_bar);
      if ((rc = launch_check(ctx, "k_gal_step_adjoint"))) return rc;
    }
    if (mg) {
      rc = shtmg_adjoint(T, kappa_bar[m]);
      if (rc == CLC_ENOTCONVERGED) status = rc;
      else if (rc) return rc;
    } else if ((rc = sht_poisson_adjoint(T, db, kappa_bar[m]))) {
      return rc;
    }
  }
  return status;
}

extern "C" int clc_gal_tape_destroy(clc_gal_tape* T) {
  if (!T) return CLC_EINVAL;
  if (T->ctx) cudaStreamSynchronize(T->ctx->stream);
  delete T;
  return CLC_OK;
}
