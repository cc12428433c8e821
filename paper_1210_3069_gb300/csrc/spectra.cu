// Convergence, E/B-mode shear and rotation power spectra of the final
// inverse magnification matrices (paper Sec. 5, Eq. invmagmat).
//
// The shear gamma_1 + i gamma_2 ((theta-hat, phi-hat) basis) is a spin-2
// field.  With eth^2 Y_lm = (A_lm - B_lm) e^{i m phi} and
// eth-bar^2 Y_lm = (A_lm + B_lm) e^{i m phi},
//   A_lm = -2 cot t dlambda_lm - (l(l+1) - 2 m^2 / sin^2 t) lambda_lm,
//   B_lm = (2 m / sin t)(dlambda_lm - cot t lambda_lm),
// the E and B coefficients follow from the ring Fourier coefficients F1, F2 of
// gamma_1 and gamma_2 as
//   E_lm = sum_r [A F1 - i B F2] / N_l,  B_lm = sum_r [A F2 + i B F1] / N_l,
// N_l = sqrt((l+2)! / (l-2)!), so that a potential's shear gamma = eth^2 psi / 2
// has E_lm = N_l psi_lm / 2 and no B.  dlambda comes from the lambda table
// (sin t dlambda_lm = l eps_{l+1,m} lambda_{l+1,m} - (l+1) eps_lm lambda_{l-1,m}).
// Under theta -> pi - theta, A keeps the parity (-1)^{l+m} of lambda_lm and B
// takes the opposite one, which fixes the north/south combinations.
#include "fft.cuh"
#include "legendre.cuh"
#include "sphere.cuh"

int clc_sht_analysis(clc_ctx*, const double*, int, int, double*);

namespace clc {

__device__ __forceinline__ double eps_lm(int l, int m) {
  if (l <= m) return 0.0;
  return sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
}

// block (l-block, m): warp per l (8 l per warp), lanes over the northern
// rings, taken in chunks of kEbChunk rings staged in shared memory (the
// ring sums of each l accumulate across chunks in registers)
constexpr int kEbChunk = 1024;

__global__ void k_legendre_eb(int nside, int lmax, int R, const long long* __restrict__ off,
                              const double* __restrict__ tab, const double2* __restrict__ F1,
                              const double2* __restrict__ F2, int ldf, double2* __restrict__ E,
                              double2* __restrict__ B) {
  extern __shared__ double2 V[];  // [4][kEbChunk]: F1 even/odd, F2 even/odd
  const int m = blockIdx.y;
  const int l0 = m + blockIdx.x * 64;
  if (l0 > lmax) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* col = tab + off[m];
  double acc[8][4];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.0;
  for (int c0 = 0; c0 < R; c0 += kEbChunk) {
    const int cn = min(kEbChunk, R - c0);
    __syncthreads();   // the previous chunk is consumed
    for (int rr = threadIdx.x; rr < cn; rr += blockDim.x) {
      const int i = c0 + rr + 1;
      const bool eq = i == 2 * nside;
      const double2 a = F1[(size_t)m * ldf + i - 1], c = F2[(size_t)m * ldf + i - 1];
      double2 as = make_double2(0.0, 0.0), cs = make_double2(0.0, 0.0);
      if (!eq) {
        as = F1[(size_t)m * ldf + 4 * nside - i - 1];
        cs = F2[(size_t)m * ldf + 4 * nside - i - 1];
      }
      V[rr] = make_double2(a.x + as.x, a.y + as.y);
      V[kEbChunk + rr] = make_double2(a.x - as.x, a.y - as.y);
      V[2 * kEbChunk + rr] = make_double2(c.x + cs.x, c.y + cs.y);
      V[3 * kEbChunk + rr] = make_double2(c.x - cs.x, c.y - cs.y);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int l = l0 + warp + 8 * k;
      if (l > lmax || l < 2) continue;
      const double* row = col + (size_t)(l - m) * R;
      const double* rowp = row + R;                              // l + 1 (table holds lmax + 1)
      const double* rowm = l > m ? row - R : nullptr;            // l - 1
      const double e1 = (double)l * eps_lm(l + 1, m), e0 = (l + 1.0) * eps_lm(l, m);
      const double ll1 = (double)l * (l + 1.0), m2 = 2.0 * m * m, m_2 = 2.0 * m;
      const int p = (l + m) & 1;
      const double2* VA1 = V + (p ? kEbChunk : 0);          // F1 with A's parity
      const double2* VB1 = V + (p ? 0 : kEbChunk);          // F1 with B's parity
      const double2* VA2 = V + 2 * kEbChunk + (p ? kEbChunk : 0);
      const double2* VB2 = V + 2 * kEbChunk + (p ? 0 : kEbChunk);
      double ex = 0, ey = 0, bx = 0, by = 0;
      for (int rr = lane; rr < cn; rr += 32) {
        const int r = c0 + rr;
        const Ring g = ring_geom(nside, r + 1);
        const double is = 1.0 / g.s, cot = g.z * is;
        const double lam = row[r];
        const double dl = (e1 * rowp[r] - (rowm ? e0 * rowm[r] : 0.0)) * is;
        const double A = -2.0 * cot * dl - (ll1 - m2 * is * is) * lam;
        const double Bf = m_2 * is * (dl - cot * lam);
        const double2 a1 = VA1[rr], b1 = VB1[rr], a2 = VA2[rr], b2 = VB2[rr];
        // E += A F1 - i B F2 ; B += A F2 + i B F1
        ex += A * a1.x + Bf * b2.y;
        ey += A * a1.y - Bf * b2.x;
        bx += A * a2.x - Bf * b1.y;
        by += A * a2.y + Bf * b1.x;
      }
      acc[k][0] += ex;
      acc[k][1] += ey;
      acc[k][2] += bx;
      acc[k][3] += by;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int l = l0 + warp + 8 * k;
    if (l > lmax || l >= l0 + 64) continue;
    const size_t li = alm_idx(lmax, l, m);
    if (l < 2) {
      if (lane == 0) {
        E[li] = make_double2(0.0, 0.0);
        B[li] = make_double2(0.0, 0.0);
      }
      continue;
    }
    double ex = acc[k][0], ey = acc[k][1], bx = acc[k][2], by = acc[k][3];
    for (int o = 16; o > 0; o >>= 1) {
      ex += __shfl_xor_sync(0xffffffffu, ex, o);
      ey += __shfl_xor_sync(0xffffffffu, ey, o);
      bx += __shfl_xor_sync(0xffffffffu, bx, o);
      by += __shfl_xor_sync(0xffffffffu, by, o);
    }
    if (lane == 0) {
      const double inv = 1.0 / sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0));
      E[li] = make_double2(ex * inv, ey * inv);
      B[li] = make_double2(bx * inv, by * inv);
    }
  }
}

// C_l = (a_l0 b_l0* + 2 sum_{m>0} Re a_lm b_lm*) / (2l+1), one thread per l
__global__ void k_cl(const double2* __restrict__ a, const double2* __restrict__ b, int lmax, double* __restrict__ cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  double acc = 0.0;
  for (int m = 0; m <= l; ++m) {
    const double2 x = a[alm_idx(lmax, l, m)], y = b[alm_idx(lmax, l, m)];
    acc += (m ? 2.0 : 1.0) * (x.x * y.x + x.y * y.y);
  }
  cl[l] = acc / (2.0 * l + 1.0);
}

// kappa, gamma_1, gamma_2, omega maps of A (SoA A[4][n], Eq. invmagmat)
__global__ void k_decompose_A(const double* __restrict__ A, int64_t n, double* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double a = A[k], b = A[n + k], c = A[2 * n + k], d = A[3 * n + k];
    out[k] = 1.0 - 0.5 * (a + d);
    out[n + k] = -0.5 * (a - d);
    out[2 * n + k] = -0.5 * (b + c);
    out[3 * n + k] = 0.5 * (b - c);
  }
}

// The same decomposition after carrying each ray's A from the tangent basis
// at its source-sphere position x to the basis at its image position, the
// centre of RING pixel k (Appendix B transport along the geodesic between
// them).  One CTA per ring, like the ray initialisation: the ring geometry
// once, longitudes by sincospi.  kappa and omega are invariant under the
// rotation; the shear turns by twice its angle.
__global__ void k_decompose_A_image(const double* __restrict__ x, const double* __restrict__ A, int nside, int64_t n,
                                    double* __restrict__ out) {
  const int i = blockIdx.x + 1;
  const Ring r = ring_geom(nside, i);
  const double inv = 1.0 / (double)r.npix;
  const int shift = r.phi0 != 0.0 ? 1 : 0;
  for (int j = threadIdx.x; j < r.npix; j += blockDim.x) {
    const int64_t k = r.first + j;
    double sp, cp;
    sincospi((double)(2 * j + shift) * inv, &sp, &cp);
    const double n0[3] = {r.s * cp, r.s * sp, r.z};
    const double xv[3] = {x[k], x[n + k], x[2 * n + k]};
    const double ix = rsqrt(dot3(xv, xv));
    const double nx[3] = {xv[0] * ix, xv[1] * ix, xv[2] * ix};
    double t[3], q[3], Q[4], Ai[4];
    tangent_basis(nx, t, q);
    transport_q(nx, t, n0, Q);
    const double Ak[4] = {A[k], A[n + k], A[2 * n + k], A[3 * n + k]};
    qaqt(Q, Ak, Ai);
    out[k] = 1.0 - 0.5 * (Ai[0] + Ai[3]);
    out[n + k] = -0.5 * (Ai[0] - Ai[3]);
    out[2 * n + k] = -0.5 * (Ai[1] + Ai[2]);
    out[3 * n + k] = 0.5 * (Ai[1] - Ai[2]);
  }
}

int eb_analysis(clc_ctx* ctx, const double* g1, const double* g2, int nside, int lmax, double2* E, double2* B) {
  int rc;
  auto plan = get_fft_plan(ctx, nside, &rc);
  if (rc) return rc;
  auto T = get_legendre_table(ctx, nside, lmax, &rc);
  if (rc) return rc;
  const int ldf = 4 * nside - 1;
  double2* F = (double2*)scratch(ctx, 0, 2 * sizeof(double2) * (size_t)ldf * (lmax + 1));
  if (!F) return CLC_ENOMEM;
  double2* F2 = F + (size_t)ldf * (lmax + 1);
  const double w = 4.0 * kPi / (12.0 * (double)nside * nside);
  if ((rc = ring_analysis(ctx, *plan, g1, lmax, w, F, ldf))) return rc;
  if ((rc = ring_analysis(ctx, *plan, g2, lmax, w, F2, ldf))) return rc;
  dim3 grid((lmax + 1 + 63) / 64, lmax + 1);
  const int smem = 4 * kEbChunk * (int)sizeof(double2);
  cudaFuncSetAttribute(k_legendre_eb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_legendre_eb", k_legendre_eb, grid, 256, smem, nside, lmax, T->R, (const long long*)T->offsets.p,
             (const double*)T->data.p, F, F2, ldf, E, B);
  return launch_check(ctx, "k_legendre_eb");
}

}  // namespace clc

using namespace clc;

extern "C" int clc_eb_analysis(clc_ctx* ctx, const double* g1, const double* g2, int nside, int lmax, double* E,
                               double* B) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside) || nside > 4096 || lmax < 0 || lmax > 4 * nside)
    return set_err(ctx, CLC_EINVAL, "clc_eb_analysis: bad nside / lmax");
  if (!g1 || !g2 || !E || !B) return set_err(ctx, CLC_EINVAL, "clc_eb_analysis: null pointer");
  cudaSetDevice(ctx->device);
  return eb_analysis(ctx, g1, g2, nside, lmax, (double2*)E, (double2*)B);
}

extern "C" int clc_power_spectrum(clc_ctx* ctx, const double* alm, const double* alm2, int lmax, double* cl) {
  if (!ctx) return CLC_EINVAL;
  if (lmax < 0 || !alm || !cl) return set_err(ctx, CLC_EINVAL, "clc_power_spectrum: bad arguments");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_cl", k_cl, (lmax + 128) / 128, 128, 0, (const double2*)alm,
             (const double2*)(alm2 ? alm2 : alm), lmax, cl);
  return launch_check(ctx, "k_cl");
}

extern "C" int clc_lensing_spectra(clc_ctx* ctx, const double* x, const double* A, int nside, int lmax,
                                   double* cl_out) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside) || nside > 4096 || lmax < 2 || lmax > 4 * nside || !A || !cl_out)
    return set_err(ctx, CLC_EINVAL, "clc_lensing_spectra: bad arguments");
  cudaSetDevice(ctx->device);
  const int64_t np = 12ll * nside * nside;
  const size_t na = (size_t)(lmax + 1) * (lmax + 2) / 2;
  double* maps = (double*)scratch(ctx, 5, 4 * np * sizeof(double) + 4 * na * sizeof(double2));
  if (!maps) return CLC_ENOMEM;
  double2* alm = (double2*)(maps + 4 * np);
  int rc;
  if (x)
    CLC_LAUNCH(ctx, "k_decompose_A", k_decompose_A_image, 4 * nside - 1, 256, 0, x, A, nside, np, maps);
  else
    CLC_LAUNCH(ctx, "k_decompose_A", k_decompose_A, 1024, 256, 0, A, np, maps);
  if ((rc = launch_check(ctx, "k_decompose_A"))) return rc;
  if ((rc = clc_sht_analysis(ctx, maps, nside, lmax, (double*)alm))) return rc;                    // kappa
  if ((rc = clc_sht_analysis(ctx, maps + 3 * np, nside, lmax, (double*)(alm + na)))) return rc;    // omega
  if ((rc = eb_analysis(ctx, maps + np, maps + 2 * np, nside, lmax, alm + 2 * na, alm + 3 * na))) return rc;
  for (int q = 0; q < 4; ++q) {
    // output order: kappa, E, B, omega
    const int src = q == 0 ? 0 : (q == 1 ? 2 : (q == 2 ? 3 : 1));
    if ((rc = clc_power_spectrum(ctx, (const double*)(alm + src * na), nullptr, lmax, cl_out + (size_t)q * (lmax + 1))))
      return rc;
  }
  return CLC_OK;
}
