// Multiple-plane ray recursion on the sphere (paper Sec. 2.2, Appendix B):
// per ray and plane, the lens fields at the ray, the Jacobian recursion
// A^(n+1) = (1 - c) A^(n-1) + c A^(n) - d U^(n) A^(n) (Eq. Atraj), the rotation
// of the propagation direction about n x alpha by |alpha| (Eq. betaprop), the
// advance to the next sphere (Eq. posprop, positive root) and the parallel
// transport of A^(n+1) and A^(n) to the tangent basis at the new position
// (Appendix B).  One thread per ray; the state is FP64 structure-of-arrays so
// that each component is a coalesced stream.
#include "mg.cuh"
#include "patch_fd.cuh"

int clc_poisson_sht(clc_ctx*, const double*, int, int, int, double*, const clc_derivs*);

namespace clc {

struct RayPtrs {
  double* x;
  double* beta;
  double* A;
  double* Ap;
  const int32_t* bundle;
  int64_t n;
};

__global__ void k_rays_init(const double* __restrict__ z, const double* __restrict__ phi, double chi0, int nb,
                            RayPtrs R) {
  const int64_t n = R.n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double zz = z[k], pp = phi[k];
    const double s = sqrt((1.0 - zz) * (1.0 + zz));
    const double v[3] = {s * cos(pp), s * sin(pp), zz};
    for (int c = 0; c < 3; ++c) {
      R.x[c * n + k] = chi0 * v[c];
      R.beta[c * n + k] = v[c];
    }
    R.A[k] = 1.0; R.A[n + k] = 0.0; R.A[2 * n + k] = 0.0; R.A[3 * n + k] = 1.0;
    R.Ap[k] = 1.0; R.Ap[n + k] = 0.0; R.Ap[2 * n + k] = 0.0; R.Ap[3 * n + k] = 1.0;
    if (nb > 0 && R.bundle) ((int32_t*)R.bundle)[k] = (int32_t)ang2pix_nest(nb, zz, pp);
  }
}

// rays at every RING pixel centre of nside: one CTA per ring, so the ring
// geometry is computed once; longitudes by sincospi of (2 j + shift) / npix
// for the first quarter of the ring (the other three are the same angles
// plus pi / 2, pi, 3 pi / 2: their cosines and sines are the first quarter's
// swapped and negated, exactly) and bundles by the integer RING -> NEST
// conversion
__global__ void k_rays_init_pixels(int nside, double chi0, int nb, RayPtrs R) {
  const int64_t n = R.n;
  const int i = blockIdx.x + 1;
  const Ring r = ring_geom(nside, i);
  const double inv = 1.0 / (double)r.npix;
  const int shift = r.phi0 != 0.0 ? 1 : 0;
  const int bshift = nb > 0 ? 2 * (ilog2(nside) - ilog2(nb)) : 0;
  const int quarter = r.npix / 4;
  for (int j = threadIdx.x; j < quarter; j += blockDim.x) {
    double sp, cp;
    sincospi((double)(2 * j + shift) * inv, &sp, &cp);
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) {
      // (cos, sin) of the angle plus qd pi / 2
      const double c = qd == 0 ? cp : qd == 1 ? -sp : qd == 2 ? -cp : sp;
      const double sn = qd == 0 ? sp : qd == 1 ? cp : qd == 2 ? -sp : -cp;
      const int jj = j + qd * quarter;
      const int64_t k = r.first + jj;
      const double v[3] = {r.s * c, r.s * sn, r.z};
      for (int d = 0; d < 3; ++d) {
        R.x[d * n + k] = chi0 * v[d];
        R.beta[d * n + k] = v[d];
      }
      R.A[k] = 1.0; R.A[n + k] = 0.0; R.A[2 * n + k] = 0.0; R.A[3 * n + k] = 1.0;
      R.Ap[k] = 1.0; R.Ap[n + k] = 0.0; R.Ap[2 * n + k] = 0.0; R.Ap[3 * n + k] = 1.0;
      if (nb > 0 && R.bundle) ((int32_t*)R.bundle)[k] = (int32_t)(ring_pos2nest(nside, i, jj) >> bshift);
    }
  }
}

// Lens fields at the ray from RING maps: alpha as a tangent 3-vector and U as
// a tangent 3x3 tensor, ring-bilinear interpolation, projection on the basis
// at the ray.
__device__ void map_lens_fields(const clc_derivs& M, int nside, const double nv[3], double out[5]) {
  const double th = atan2(sqrt(nv[0] * nv[0] + nv[1] * nv[1]), nv[2]);
  double ph = atan2(nv[1], nv[0]);
  if (ph < 0) ph += 2.0 * kPi;
  const Interp8 w = interp_weights(nside, th, ph);
  double a3[3] = {0, 0, 0}, U3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int k = 0; k < 8; ++k) {
    if (w.w[k] == 0.0) continue;
    const int64_t p = w.p[k];
    int64_t j;
    const int i = pix2ring(nside, p, &j);
    const Ring r = ring_geom(nside, i);
    const double phi = r.phi0 + (2.0 * kPi) * (double)j / (double)r.npix;
    const double cp = cos(phi), sp = sin(phi);
    const double t[3] = {r.z * cp, r.z * sp, -r.s};
    const double q[3] = {-sp, cp, 0.0};
    const double at = M.a_th[p], ap = M.a_ph[p], utt = M.u_tt[p], upp = M.u_pp[p], utp = M.u_tp[p];
    const double ww = w.w[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      a3[a] += ww * (at * t[a] + ap * q[a]);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        U3[a][b] += ww * (utt * t[a] * t[b] + upp * q[a] * q[b] + utp * (t[a] * q[b] + q[a] * t[b]));
    }
  }
  double t[3], q[3];
  tangent_basis(nv, t, q);
  out[0] = dot3(a3, t);
  out[1] = dot3(a3, q);
  double Ut[3], Uq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Ut[a] = U3[a][0] * t[0] + U3[a][1] * t[1] + U3[a][2] * t[2];
    Uq[a] = U3[a][0] * q[0] + U3[a][1] * q[1] + U3[a][2] * q[2];
  }
  out[2] = dot3(t, Ut);
  out[3] = dot3(q, Uq);
  out[4] = dot3(t, Uq);
}

struct StepCoef {
  double c, d, dchi2;
  double ichi_n, ichi_next;   // 1 / chi_n, 1 / chi_next
};

// Rotation of beta about the unit axis k = n x alpha / |alpha| by the angle
// a = |alpha| (Eq. betaprop), written with the unnormalised axis kk = n x alpha
// (|kk| = a, alpha being tangent at n):
//   R beta = beta cos a + (kk x beta) sin(a) / a + kk (kk . beta)(1 - cos a) / a^2,
// whose three coefficients are even functions of a: for a < 2^-5 their
// Maclaurin series in a^2 (through a^8; first omitted terms below 1e-21),
// so no square root or trigonometric call is needed; sincos beyond.
__device__ __forceinline__ void rotate_by_deflection(const double be[3], const double kk[3], double a2, double bn[3]) {
  double cs, sc, vc;
  if (a2 < 0.0009765625) {
    cs = 1.0 - a2 * (0.5 - a2 * ((1.0 / 24.0) - a2 * ((1.0 / 720.0) - a2 * (1.0 / 40320.0))));
    sc = 1.0 - a2 * ((1.0 / 6.0) - a2 * ((1.0 / 120.0) - a2 * ((1.0 / 5040.0) - a2 * (1.0 / 362880.0))));
    vc = 0.5 - a2 * ((1.0 / 24.0) - a2 * ((1.0 / 720.0) - a2 * ((1.0 / 40320.0) - a2 * (1.0 / 3628800.0))));
  } else {
    const double a = sqrt(a2);
    double sn;
    sincos(a, &sn, &cs);
    sc = sn / a;
    vc = (1.0 - cs) / a2;
  }
  double kb[3];
  cross3(kk, be, kb);
  const double kd = dot3(kk, be) * vc;
#pragma unroll
  for (int i = 0; i < 3; ++i) bn[i] = fma(be[i], cs, fma(kb[i], sc, kk[i] * kd));
}

// Transport matrix Q from the basis (t0, .) at n0 to the basis (t1, p1) at n1
// (Appendix B).  The rotation taking n0 to n1 about n0 x n1 maps a vector v
// orthogonal to n0 to v - ((n1 . v) / (1 + n0 . n1)) (n0 + n1); with
// t1 . n1 = p1 . n1 = 0 the change of basis is the plane rotation
// [[q0, -q1], [q1, q0]], q0 = t1 . t0 - (n1 . t0)(t1 . n0) / (1 + c),
// q1 = p1 . t0 - (n1 . t0)(p1 . n0) / (1 + c).  (The same Q as transport_q,
// without the normalised axis.)
__device__ __forceinline__ void transport_q_closed(const double n0[3], const double t0[3], const double n1[3],
                                                   const double t1[3], const double p1[3], double Q[4]) {
  const double w = dot3(n1, t0) / (1.0 + dot3(n0, n1));
  const double q0 = dot3(t1, t0) - w * dot3(t1, n0);
  const double q1 = (p1[0] * t0[0] + p1[1] * t0[1]) - w * (p1[0] * n0[0] + p1[1] * n0[1]);
  Q[0] = q0;
  Q[1] = -q1;
  Q[2] = q1;
  Q[3] = q0;
}

// o = Q A Q^T for the plane rotation Q = [[q0, -q1], [q1, q0]]: the parts
// (a00 + a11, a10 - a01) of A are kept and (a00 - a11, a01 + a10) turn by
// twice the angle of Q
__device__ __forceinline__ void rotate_2x2(double q0, double q1, const double A[4], double o[4]) {
  const double c2 = 0.5 * fma(q0, q0, -q1 * q1), s2 = q0 * q1;   // halves of cos, sin of twice the angle
  const double sm = A[0] + A[3], sk = A[2] - A[1], df = A[0] - A[3], sy = A[1] + A[2];
  const double e = fma(c2, df, -s2 * sy), f = fma(s2, df, c2 * sy);
  o[0] = fma(0.5, sm, e);
  o[3] = fma(0.5, sm, -e);
  o[1] = fma(-0.5, sk, f);
  o[2] = fma(0.5, sk, f);
}

template <bool kMG>
__global__ void k_ray_step(RayPtrs R, MGView V, clc_derivs M, int nside_maps, StepCoef sc) {
  const int64_t n = R.n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double x[3], be[3], A[4], Ap[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) { x[c] = R.x[c * n + k]; be[c] = R.beta[c * n + k]; }
#pragma unroll
    for (int c = 0; c < 4; ++c) { A[c] = R.A[c * n + k]; Ap[c] = R.Ap[c * n + k]; }
    // the ray is on the sphere of radius chi_n (where the previous step or the
    // initialisation put it): its direction is x / chi_n
    const double nv[3] = {x[0] * sc.ichi_n, x[1] * sc.ichi_n, x[2] * sc.ichi_n};
    double t[3], q[3];
    tangent_basis(nv, t, q);
    double L[5];
    if (kMG) patch_lens_fields(V, R.bundle[k], nv, t, q, L);
    else map_lens_fields(M, nside_maps, nv, L);
    // Eq. Atraj in the basis at n
    const double U[4] = {L[2], L[4], L[4], L[3]};
    double An[4];
    An[0] = (1.0 - sc.c) * Ap[0] + sc.c * A[0] - sc.d * (U[0] * A[0] + U[1] * A[2]);
    An[1] = (1.0 - sc.c) * Ap[1] + sc.c * A[1] - sc.d * (U[0] * A[1] + U[1] * A[3]);
    An[2] = (1.0 - sc.c) * Ap[2] + sc.c * A[2] - sc.d * (U[2] * A[0] + U[3] * A[2]);
    An[3] = (1.0 - sc.c) * Ap[3] + sc.c * A[3] - sc.d * (U[2] * A[1] + U[3] * A[3]);
    // Eq. betaprop: rotate beta about n x alpha by |alpha|
    const double av[3] = {L[0] * t[0] + L[1] * q[0], L[0] * t[1] + L[1] * q[1], L[0] * t[2]};
    double kk[3], bn[3];
    cross3(nv, av, kk);
    rotate_by_deflection(be, kk, dot3(av, av), bn);
    // Eq. posprop: the root lambda > 0 of |x + lambda beta|^2 = chi_next^2
    // (beta is nearly radial, x . beta close to chi_n, so the difference of
    // the two terms keeps all but log2(chi_n / (chi_next - chi_n)) bits)
    const double xb = dot3(x, bn);
    const double lam = sqrt(fma(xb, xb, sc.dchi2)) - xb;
    double x1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) x1[c] = fma(lam, bn[c], x[c]);
    const double n1[3] = {x1[0] * sc.ichi_next, x1[1] * sc.ichi_next, x1[2] * sc.ichi_next};
    // Appendix B: transport A^(n+1) and A^(n) to the basis at the new point
    double t1[3], p1[3], Q[4], Ao[4], Apo[4];
    tangent_basis(n1, t1, p1);
    transport_q_closed(nv, t, n1, t1, p1, Q);
    rotate_2x2(Q[0], Q[2], An, Ao);
    rotate_2x2(Q[0], Q[2], A, Apo);
#pragma unroll
    for (int c = 0; c < 3; ++c) { R.x[c * n + k] = x1[c]; R.beta[c * n + k] = bn[c]; }
#pragma unroll
    for (int c = 0; c < 4; ++c) { R.A[c * n + k] = Ao[c]; R.Ap[c * n + k] = Apo[c]; }
  }
}

static RayPtrs ray_ptrs(const clc_rays* r) {
  RayPtrs p;
  p.x = r->x; p.beta = r->beta; p.A = r->A; p.Ap = r->Ap; p.bundle = r->bundle; p.n = r->n;
  return p;
}

static int rays_ok(clc_ctx* ctx, const clc_rays* r) {
  if (!r || r->n < 0) return set_err(ctx, CLC_EINVAL, "bad ray state");
  if (r->n > 0 && (!r->x || !r->beta || !r->A || !r->Ap)) return set_err(ctx, CLC_EINVAL, "null ray arrays");
  return CLC_OK;
}

static int blocks(clc_ctx* ctx, int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms(ctx) * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace clc

using namespace clc;

extern "C" int clc_rays_init(clc_ctx* ctx, const double* z, const double* phi, double chi0, int nb, clc_rays* r) {
  if (!ctx) return CLC_EINVAL;
  int rc = rays_ok(ctx, r);
  if (rc) return rc;
  if (!(chi0 > 0) || (nb > 0 && !valid_nside(nb))) return set_err(ctx, CLC_EINVAL, "clc_rays_init: bad chi0 / nside");
  if (r->n == 0) return CLC_OK;
  if (!z || !phi) return set_err(ctx, CLC_EINVAL, "clc_rays_init: null positions");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_rays_init", k_rays_init, blocks(ctx, r->n, 256), 256, 0, z, phi, chi0, nb, ray_ptrs(r));
  return launch_check(ctx, "k_rays_init");
}

extern "C" int clc_rays_init_pixels(clc_ctx* ctx, int nside, double chi0, int nb, clc_rays* r) {
  if (!ctx) return CLC_EINVAL;
  int rc = rays_ok(ctx, r);
  if (rc) return rc;
  if (!valid_nside(nside) || !(chi0 > 0) || (nb > 0 && (!valid_nside(nb) || nb > nside)) ||
      r->n != 12ll * nside * nside)
    return set_err(ctx, CLC_EINVAL, "clc_rays_init_pixels: need n = 12 nside^2, chi0 > 0, nside_bundle <= nside");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_rays_init", k_rays_init_pixels, 4 * nside - 1, 256, 0, nside, chi0, nb, ray_ptrs(r));
  return launch_check(ctx, "k_rays_init_pixels");
}

extern "C" int clc_ray_step(clc_ctx* ctx, const clc_plane_solution* sol, const clc_derivs* maps, int nside_maps,
                            double chi_prev, double chi_n, double chi_next, clc_rays* r) {
  if (!ctx) return CLC_EINVAL;
  int rc = rays_ok(ctx, r);
  if (rc) return rc;
  if (!(chi_prev >= 0 && chi_n > chi_prev && chi_next > chi_n))
    return set_err(ctx, CLC_EINVAL, "clc_ray_step: need 0 <= chi_prev < chi_n < chi_next");
  if (!sol && (!maps || !maps->a_th || !maps->a_ph || !maps->u_tt || !maps->u_pp || !maps->u_tp || !valid_nside(nside_maps)))
    return set_err(ctx, CLC_EINVAL, "clc_ray_step: need a solution or five lens maps");
  if (sol && !r->bundle && r->n > 0) return set_err(ctx, CLC_EINVAL, "clc_ray_step: SHT+MG lookup needs ray bundles");
  if (r->n == 0) return CLC_OK;
  cudaSetDevice(ctx->device);
  StepCoef sc;
  sc.c = (chi_n / chi_next) * ((chi_next - chi_prev) / (chi_n - chi_prev));
  sc.d = (chi_next - chi_n) / chi_next;
  sc.dchi2 = (chi_next - chi_n) * (chi_next + chi_n);
  sc.ichi_n = 1.0 / chi_n;
  sc.ichi_next = 1.0 / chi_next;
  clc_derivs M{};
  if (maps) M = *maps;
  if (sol) {
    CLC_LAUNCH(ctx, "k_ray_step", k_ray_step<true>, blocks(ctx, r->n, 128), 128, 0, ray_ptrs(r), mg_view(sol), M, 0, sc);
  } else {
    MGView V{};
    CLC_LAUNCH(ctx, "k_ray_step", k_ray_step<false>, blocks(ctx, r->n, 128), 128, 0, ray_ptrs(r), V, M, nside_maps, sc);
  }
  return launch_check(ctx, "k_ray_step");
}

extern "C" int clc_raytrace_planes(clc_ctx* ctx, int solver, const clc_mg_params* mg,
                                   const double* const* kappa_planes, int nplanes, int nside, const double* chi,
                                   clc_rays* r) {
  if (!ctx) return CLC_EINVAL;
  int rc = rays_ok(ctx, r);
  if (rc) return rc;
  if (!mg || !kappa_planes || !chi || nplanes < 1 || !valid_nside(nside) ||
      (solver != CLC_SOLVER_SHT && solver != CLC_SOLVER_SHTMG))
    return set_err(ctx, CLC_EINVAL, "clc_raytrace_planes: bad arguments");
  for (int m = 0; m < nplanes; ++m)
    if (!kappa_planes[m] || !(chi[m + 1] > chi[m]) || !(chi[m] > 0))
      return set_err(ctx, CLC_EINVAL, "clc_raytrace_planes: null plane or non-increasing chi");
  cudaSetDevice(ctx->device);
  if (solver == CLC_SOLVER_SHT) {
    const size_t np = 12ull * nside * nside;
    double* maps = (double*)scratch(ctx, 4, 5 * np * sizeof(double));
    if (!maps) return CLC_ENOMEM;
    clc_derivs d{maps, maps + np, maps + 2 * np, maps + 3 * np, maps + 4 * np};
    for (int m = 0; m < nplanes; ++m) {
      if ((rc = clc_poisson_sht(ctx, kappa_planes[m], nside, mg->lmax, CLC_FP64, nullptr, &d))) return rc;
      if ((rc = clc_ray_step(ctx, nullptr, &d, nside, m > 0 ? chi[m - 1] : 0.0, chi[m], chi[m + 1], r))) return rc;
    }
    return CLC_OK;
  }
  clc_plane_solution* sol = nullptr;
  if ((rc = clc_solution_create(ctx, nside, mg, &sol))) return rc;
  int status = CLC_OK;
  for (int m = 0; m < nplanes && (status == CLC_OK || status == CLC_ENOTCONVERGED); ++m) {
    rc = clc_poisson_shtmg(ctx, kappa_planes[m], nside, mg, sol, nullptr);
    if (rc != CLC_OK && rc != CLC_ENOTCONVERGED) {
      status = rc;
      break;
    }
    if (rc == CLC_ENOTCONVERGED) status = rc;
    rc = clc_ray_step(ctx, sol, nullptr, 0, m > 0 ? chi[m - 1] : 0.0, chi[m], chi[m + 1], r);
    if (rc) {
      status = rc;
      break;
    }
  }
  clc_solution_destroy(sol);
  return status;
}
