// Legendre step of the SHT (paper Sec. 3.2; the associated-Legendre
// recurrence of Press et al. 2007 Sec. 6.7) in FP64.
//
// The table lambda_lm(z_r) is built once per (Nside, lmax) with the
// three-term recurrence in l, started from
// lambda_mm = (-1)^m sqrt((2m+1)!! / (4 pi (2m)!!)) sin^m(theta) carried as a
// mantissa and a power-of-two exponent (sin^m theta underflows FP64 near the
// poles at large m).  Analysis and synthesis are then per-m matrix-vector
// products over the northern rings, using lambda_lm(-z) = (-1)^(l+m) lambda_lm(z)
// for the southern mirror rings.  Layout [m][l][r] keeps ring index r
// contiguous: the build writes, the synthesis reads (thread per ring) and the
// analysis reads (warp per l, lanes over rings) all coalesced.
#include <cmath>

#include "legendre.cuh"

namespace clc {

// p * 2^e, exact unless the result is subnormal or zero (one final rounding);
// |p| < 2^410 and e <= 64 here.
__device__ __forceinline__ double scale_pow2(double p, int e) {
  if (e >= -1022) return p * __longlong_as_double((long long)(e + 1023) << 52);
  if (e < -1600) return 0.0;
  return (p * __longlong_as_double((long long)(e + 600 + 1023) << 52)) * 0x1p-600;
}

__global__ void k_legendre_build(int nside, int lmax, int R, const long long* __restrict__ off,
                                 const double* __restrict__ lognorm, const double2* __restrict__ ab,
                                 double* __restrict__ tab, int m0) {
  const int m = m0 + blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const Ring g = ring_geom(nside, r + 1);
  const double z = g.z;
  const int lt = lmax + 1;  // table band limit
  double* col = tab + off[m - m0];
  const double l2 = lognorm[m] + (double)m * log2(g.s);
  int e = (int)floor(l2);
  double p2 = exp2(l2 - (double)e);
  if (m & 1) p2 = -p2;
  col[r] = scale_pow2(p2, e);
  if (lt < m + 1) return;
  double p1 = sqrt(2.0 * m + 3.0) * z * p2;
  col[(size_t)R + r] = scale_pow2(p1, e);
  const double big = 0x1p400, small = 0x1p-400;
  for (int l = m + 2; l <= lt; ++l) {
    const double2 c = ab[alm_idx(lt, l, m)];
    double p0 = c.x * (z * p1 - c.y * p2);
    if (fabs(p0) > big) {
      p0 *= small;
      p1 *= small;
      e += 400;
    }
    col[(size_t)(l - m) * R + r] = scale_pow2(p0, e);
    p2 = p1;
    p1 = p0;
  }
}

size_t legendre_table_bytes(int nside, int lmax, int m0, int m1) {
  const int lt = lmax + 1;
  size_t e = 0;
  for (int m = m0; m < m1; ++m) e += (size_t)(lt - m + 1) * 2 * nside;
  return e * sizeof(double);
}

int build_legendre_table(clc_ctx* ctx, int nside, int lmax, int m0, int m1, LegendreTable* T) {
  T->nside = nside;
  T->lmax = lmax;
  T->R = 2 * nside;
  T->m0 = m0;
  T->m1 = m1;
  const int lt = lmax + 1;
  T->h_offsets.resize(m1 - m0);
  long long acc = 0;
  for (int m = m0; m < m1; ++m) {
    T->h_offsets[m - m0] = acc;
    acc += (long long)(lt - m + 1) * T->R;
  }
  T->elems = (size_t)acc;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const size_t bytes = T->elems * sizeof(double);
  if (bytes + (size_t)(1ull << 30) > freeb)
    return set_err(ctx, CLC_ENOMEM, "Legendre table of " + std::to_string(bytes >> 20) + " MiB does not fit");
  // recurrence coefficients a_lm = sqrt((4l^2 - 1) / (l^2 - m^2)),
  // b_lm = sqrt(((l-1)^2 - m^2) / (4 (l-1)^2 - 1)), packed with band limit lt
  std::vector<double2> ab((size_t)alm_idx(lt, lt, lt) + 1);
  for (int m = 0; m <= lt; ++m)
    for (int l = m; l <= lt; ++l) {
      double a = 0, b = 0;
      if (l >= m + 2) {
        a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      }
      ab[alm_idx(lt, l, m)] = make_double2(a, b);
    }
  // log2 of sqrt((2m+1)!! / (4 pi (2m)!!))
  std::vector<double> lognorm(lmax + 1);
  double ln = 0.5 * std::log2(1.0 / (4.0 * kPi));
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) ln += 0.5 * std::log2((2.0 * m + 1.0) / (2.0 * m));
    lognorm[m] = ln;
  }
  Buffer d_ab, d_ln;
  auto alloc = [&](Buffer& b, size_t n) -> bool {
    b.bytes = n;
    if (cudaMalloc(&b.p, n) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return false;
    }
    return true;
  };
  if (!alloc(T->data, bytes) || !alloc(T->offsets, sizeof(long long) * (m1 - m0)) ||
      !alloc(d_ab, sizeof(double2) * ab.size()) || !alloc(d_ln, sizeof(double) * lognorm.size()))
    return set_err(ctx, CLC_ENOMEM, "Legendre table allocation failed");
  cudaMemcpyAsync(T->offsets.p, T->h_offsets.data(), sizeof(long long) * (m1 - m0), cudaMemcpyHostToDevice,
                  ctx->stream);
  cudaMemcpyAsync(d_ab.p, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(d_ln.p, lognorm.data(), sizeof(double) * lognorm.size(), cudaMemcpyHostToDevice, ctx->stream);
  dim3 grid((T->R + 127) / 128, m1 - m0);
  CLC_LAUNCH(ctx, "k_legendre_build", k_legendre_build, grid, 128, 0, nside, lmax, T->R, (const long long*)T->offsets.p,
             (const double*)d_ln.p, (const double2*)d_ab.p, (double*)T->data.p, m0);
  const int rc = launch_check(ctx, "k_legendre_build");
  // the coefficient buffers are freed when this function returns: wait for the build
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

std::shared_ptr<LegendreTable> get_legendre_table(clc_ctx* ctx, int nside, int lmax, int* rc) {
  const auto key = std::make_tuple(nside, lmax, 0);
  auto it = ctx->leg_tables.find(key);
  if (it != ctx->leg_tables.end()) {
    *rc = CLC_OK;
    return it->second;
  }
  auto T = std::make_shared<LegendreTable>();
  *rc = build_legendre_table(ctx, nside, lmax, 0, lmax + 1, T.get());
  if (*rc) return nullptr;
  ctx->leg_tables[key] = T;
  return T;
}

// Block (l-block, m): 8 warps, each warp one l at a time; lanes over rings.
__global__ void k_legendre_analysis(int nside, int lmax, int R, const long long* __restrict__ off,
                                    const double* __restrict__ tab, const double2* __restrict__ F, int ldf,
                                    double2* __restrict__ alm, int ltop, int lpack, int m0) {
  extern __shared__ double2 V[];  // V[0..R) even (N + S), V[R..2R) odd (N - S)
  const int m = m0 + blockIdx.y;
  const int l0 = m + blockIdx.x * 64;
  if (l0 > ltop) return;
  const double2* Fm = F + (size_t)m * ldf;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const int i = r + 1;
    const double2 fn = Fm[i - 1];
    double2 fs = make_double2(0.0, 0.0);
    if (i != 2 * nside) fs = Fm[4 * nside - i - 1];
    V[r] = make_double2(fn.x + fs.x, fn.y + fs.y);
    V[R + r] = make_double2(fn.x - fs.x, fn.y - fs.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* col = tab + off[m - m0];
  for (int l = l0 + warp; l <= ltop && l < l0 + 64; l += 8) {
    const double* row = col + (size_t)(l - m) * R;
    const double2* v = V + (((l + m) & 1) ? R : 0);
    double ax = 0.0, ay = 0.0;
    for (int r = lane; r < R; r += 32) {
      const double lam = row[r];
      const double2 x = v[r];
      ax = fma(lam, x.x, ax);
      ay = fma(lam, x.y, ay);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) alm[alm_idx(lpack, l, m)] = make_double2(ax, ay);
  }
}

int legendre_analysis(clc_ctx* ctx, const LegendreTable& T, const double2* F, int ldf, double2* alm, int ltop) {
  const int L = T.lmax;
  if (ltop < 0) ltop = L;
  dim3 grid((ltop + 1 + 63) / 64, T.m1 - T.m0);
  const int smem = 2 * T.R * (int)sizeof(double2);
  cudaFuncSetAttribute(k_legendre_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_legendre_analysis", k_legendre_analysis, grid, 256, smem, T.nside, L, T.R, (const long long*)T.offsets.p,
                                                        (const double*)T.data.p, F, ldf, alm, ltop, ltop, T.m0);
  return launch_check(ctx, "k_legendre_analysis");
}

struct SynthRhs {
  const double2* rhs;
  int nq;
  int lq[3];
};

// Block (ring chunk, m); thread per northern ring; the alm columns of this m
// are staged in shared memory.
__global__ void k_legendre_synthesis(int nside, int lmax, int R, const long long* __restrict__ off,
                                     const double* __restrict__ tab, SynthRhs s, double2* __restrict__ G, int ld,
                                     int m0) {
  extern __shared__ double2 A[];  // A[q * (lt - m + 1) + (l - m)]
  const int m = m0 + blockIdx.y;
  const int lt = lmax + 1;
  const int nl = lt - m + 1;
  for (int t = threadIdx.x; t < s.nq * nl; t += blockDim.x) {
    const int q = t / nl, l = m + t % nl;
    const size_t qoff = (size_t)q * (alm_idx(lt, lt, lt) + 1);
    A[t] = (l <= s.lq[q]) ? s.rhs[qoff + alm_idx(lt, l, m)] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int lmax_used = 0;
  for (int q = 0; q < s.nq; ++q) lmax_used = max(lmax_used, s.lq[q]);
  const double* col = tab + off[m - m0];
  double acc[3][2][2];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int p = 0; p < 2; ++p) acc[q][p][0] = acc[q][p][1] = 0.0;
  for (int l = m; l <= lmax_used; ++l) {
    const double lam = col[(size_t)(l - m) * R + r];
    const int p = (l + m) & 1;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q < s.nq) {
        const double2 a = A[q * nl + (l - m)];
        if (p) {
          acc[q][1][0] = fma(lam, a.x, acc[q][1][0]);
          acc[q][1][1] = fma(lam, a.y, acc[q][1][1]);
        } else {
          acc[q][0][0] = fma(lam, a.x, acc[q][0][0]);
          acc[q][0][1] = fma(lam, a.y, acc[q][0][1]);
        }
      }
    }
  }
  const int i = r + 1;
  const size_t qstride = (size_t)ld * (lmax + 2);
  for (int q = 0; q < s.nq; ++q) {
    double2* Gq = G + q * qstride + (size_t)m * ld;
    Gq[i - 1] = make_double2(acc[q][0][0] + acc[q][1][0], acc[q][0][1] + acc[q][1][1]);
    if (i != 2 * nside) Gq[4 * nside - i - 1] = make_double2(acc[q][0][0] - acc[q][1][0], acc[q][0][1] - acc[q][1][1]);
  }
}

int legendre_synthesis(clc_ctx* ctx, const LegendreTable& T, const double2* rhs, int nq, const int* lq, double2* G,
                       int ld) {
  const int L = T.lmax;
  SynthRhs s;
  s.rhs = rhs;
  s.nq = nq;
  for (int q = 0; q < 3; ++q) s.lq[q] = q < nq ? lq[q] : 0;
  dim3 grid((T.R + 127) / 128, T.m1 - T.m0);
  const int smem = nq * (L + 2) * (int)sizeof(double2);
  cudaFuncSetAttribute(k_legendre_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_legendre_synthesis", k_legendre_synthesis, grid, 128, smem, T.nside, L, T.R, (const long long*)T.offsets.p,
                                                         (const double*)T.data.p, s, G, ld, T.m0);
  return launch_check(ctx, "k_legendre_synthesis");
}

}  // namespace clc
