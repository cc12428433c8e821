// Mixed-precision, batched Legendre transforms of the SHT Poisson solve on the
// tcgen05 tensor cores (paper Sec. 3.2 transforms; the split-precision
// contraction follows the precision design of this library: FP64 only for the
// recurrence that builds the table, the ring FFTs and the final unpacking).
//
// For every m the lambda table is split by the parity p of l - m (rows l = m +
// p + 2k), because the southern mirror ring enters with sign (-1)^(l+m).  The
// table holds 2^10 lambda_lm as FP16 hi + lo (|lambda_lm| <= sqrt((2l+1)/4 pi)
// < 52 for l <= 16385, so the scaled values stay below the FP16 maximum 65504
// and small values keep more bits before lo turns subnormal), rows padded with
// zeros to a multiple of 64, laid out [m][p][k][ring] with the 2 Nside
// northern rings contiguous.  A batch of P planes of the same (Nside, lmax) shares it:
//   analysis   D[k][col]   = sum_ring T[m,p][k][ring] V[m,p][col][ring]
//              (col = plane, re/im; V = F_north +- F_south),
//   synthesis  D_p[ring][col] = sum_k T[m,p][k][ring] S[m,p][col][k]
//              (col = right-hand side, plane, re/im), both parities in one
//              CTA with two TMEM accumulators, combined in the epilogue into
//              the northern (even + odd) and southern (even - odd) rings.
// Data operands are split into FP16 hi + lo after scaling each column by a
// power of two (max -> [2^13, 2^14)); products hi*hi + hi*lo + lo*hi
// accumulate in FP32 in TMEM.
#include <algorithm>
#include <map>

#include "ring_fft.cuh"
#include "legendre.cuh"
#include "umma.cuh"

namespace clc {

constexpr long long kTcWaitPolls = 1ll << 26;
constexpr int kTabExp = 10;   // table values are 2^kTabExp lambda_lm

struct TcTable {
  int nside = 0, lmax = 0, R = 0;
  std::vector<long long> h_off;   // [2 (L+1)] row offset of group (m, p)
  std::vector<int> h_rows;        // [2 (L+1)] rows of group (m, p) (l <= lmax + 1), before padding
  std::vector<int> h_pad;         // [2 (L+1)] padded rows (multiple of 64)
  Buffer off, rows, pad;          // device copies
  Buffer hi, lo;                  // __half [total_rows + 128][R]
  Buffer items;                   // int4 (m, p, 128-row tile, 0) work items of the analysis
  int nitems = 0;
  long long total_rows = 0;
};

// ---------------------------------------------------------------------------
// table build: the FP64 scaled recurrence of legendre.cu, written as FP16 hi/lo

__device__ __forceinline__ double tc_scale_pow2(double p, int e) {
  if (e >= -1022) return p * __longlong_as_double((long long)(e + 1023) << 52);
  if (e < -1600) return 0.0;
  return (p * __longlong_as_double((long long)(e + 600 + 1023) << 52)) * 0x1p-600;
}

__device__ __forceinline__ void put_split(__half* hi, __half* lo, size_t i, double v) {
  const __half h = __double2half(v);
  hi[i] = h;
  lo[i] = __double2half(v - (double)__half2float(h));
}

__global__ void k_tc_table_build(int nside, int lmax, int R, const long long* __restrict__ off,
                                 const double* __restrict__ lognorm, const double2* __restrict__ ab,
                                 __half* __restrict__ hi, __half* __restrict__ lo) {
  const int m = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const Ring g = ring_geom(nside, r + 1);
  const double z = g.z;
  const int lt = lmax + 1;
  const double l2 = lognorm[m] + (double)m * log2(g.s);
  int e = (int)floor(l2);
  double p2 = exp2(l2 - (double)e);
  if (m & 1) p2 = -p2;
  auto store = [&](int l, double p) {
    const int par = (l - m) & 1;
    const size_t row = off[2 * m + par] + (l - m - par) / 2;
    put_split(hi, lo, row * R + r, tc_scale_pow2(p, e + kTabExp));
  };
  store(m, p2);
  if (lt < m + 1) return;
  double p1 = sqrt(2.0 * m + 3.0) * z * p2;
  store(m + 1, p1);
  for (int l = m + 2; l <= lt; ++l) {
    const double2 c = ab[alm_idx(lt, l, m)];
    double p0 = c.x * (z * p1 - c.y * p2);
    if (fabs(p0) > 0x1p400) {
      p0 *= 0x1p-400;
      p1 *= 0x1p-400;
      e += 400;
    }
    store(l, p0);
    p2 = p1;
    p1 = p0;
  }
}

std::shared_ptr<TcTable> get_tc_table(clc_ctx* ctx, int nside, int lmax, int* rc);

// ---------------------------------------------------------------------------
// operand packing

// One warp per (m, p, col): the column's values v_r, a power-of-two scale
// 2^e with max |v| 2^e in [2^13, 2^14), then FP16 hi/lo of v 2^e.
__device__ __forceinline__ int col_exponent(double mx) {
  if (!(mx > 0.0)) return 0;
  int ex;
  frexp(mx, &ex);          // mx in [2^(ex-1), 2^ex)
  return 14 - ex;
}

// analysis data: V[(2m+p)][col][r] from per-plane ring coefficients F[pl][m][ring]
__global__ void k_tc_pack_analysis(const float2* __restrict__ F, int ldf, size_t fstride, int nside, int lmax, int P,
                                   int N, int R, __half* __restrict__ vh, __half* __restrict__ vl,
                                   int* __restrict__ vexp) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int ngroups = 2 * (lmax + 1);
  if (gw >= ngroups * N) return;
  const int col = gw % N, grp = gw / N;
  const int m = grp >> 1, p = grp & 1;
  const int pl = col >> 1, im = col & 1;
  const size_t base = ((size_t)grp * N + col) * R;
  if (pl >= P) {
    for (int r = lane; r < R; r += 32) vh[base + r] = vl[base + r] = __double2half(0.0);
    if (lane == 0) vexp[grp * N + col] = 0;
    return;
  }
  const float2* Fm = F + pl * fstride + (size_t)m * ldf;
  auto val = [&](int r) -> double {
    const int i = r + 1;
    const float2 fn = Fm[i - 1];
    float2 fs = make_float2(0.f, 0.f);
    if (i != 2 * nside) fs = Fm[4 * nside - i - 1];
    const double a = im ? fn.y : fn.x, b = im ? fs.y : fs.x;
    return p ? a - b : a + b;
  };
  double mx = 0.0;
  for (int r = lane; r < R; r += 32) mx = fmax(mx, fabs(val(r)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = col_exponent(mx);
  const double sc = ldexp(1.0, e);
  for (int r = lane; r < R; r += 32) put_split(vh, vl, base + r, val(r) * sc);
  if (lane == 0) vexp[grp * N + col] = e;
}

// synthesis right-hand sides from per-plane a_lm (kappa): psi_lm, b_lm (theta
// derivative) and kappa_bl, laid out S[(2m+p)][col][k] (k = (l - m - p) / 2,
// padded rows zero), col = (q * P + pl) * 2 + re/im
__device__ __forceinline__ double2 tc_psi(const double2* a, int lmax, int l, int m) {
  if (l < m || l > lmax || l == 0) return make_double2(0.0, 0.0);
  const double2 k = a[alm_idx(lmax, l, m)];
  const double d = -1.0 / ((double)l * (l + 1.0));
  return make_double2(k.x * d, k.y * d);
}

__device__ __forceinline__ double tc_eps(int l, int m) {
  if (l <= m) return 0.0;
  return sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
}

__global__ void k_tc_pack_synthesis(const double2* __restrict__ alm, size_t astride, int lmax, int P, int nq, int N,
                                    const long long* __restrict__ soff, const int* __restrict__ pad,
                                    __half* __restrict__ sh, __half* __restrict__ sl, int* __restrict__ sexp) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int ngroups = 2 * (lmax + 1);
  if (gw >= ngroups * N) return;
  const int col = gw % N, grp = gw / N;
  const int m = grp >> 1, p = grp & 1;
  const int K = pad[grp];
  const size_t base = soff[grp] + (size_t)col * K;
  const int im = col & 1, qp = col >> 1, q = qp / P, pl = qp % P;
  if (q >= nq || K == 0) {
    for (int k = lane; k < K; k += 32) sh[base + k] = sl[base + k] = __double2half(0.0);
    if (lane == 0) sexp[grp * N + col] = 0;
    return;
  }
  const double2* a = alm + pl * astride;
  auto val = [&](int k) -> double {
    const int l = m + p + 2 * k;
    if (l > lmax + 1) return 0.0;
    double2 v;
    if (q == 0) {
      v = tc_psi(a, lmax, l, m);
    } else if (q == 1) {
      const double2 pm = tc_psi(a, lmax, l - 1, m), pp = tc_psi(a, lmax, l + 1, m);
      const double c1 = (l - 1.0) * tc_eps(l, m), c2 = (l + 2.0) * tc_eps(l + 1, m);
      v = make_double2(c1 * pm.x - c2 * pp.x, c1 * pm.y - c2 * pp.y);
    } else {
      const double2 ps = tc_psi(a, lmax, l, m);
      const double f = -(double)l * (l + 1.0);
      v = make_double2(f * ps.x, f * ps.y);
    }
    if (m == 0) v.y = 0.0;
    return im ? v.y : v.x;
  };
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(val(k)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = col_exponent(mx);
  const double sc = ldexp(1.0, e);
  for (int k = lane; k < K; k += 32) put_split(sh, sl, base + k, val(k) * sc);
  if (lane == 0) sexp[grp * N + col] = e;
}

// ---------------------------------------------------------------------------
// tensor-core contractions

struct TcAnalysisArgs {
  const __half *th, *tl;          // table
  const __half *vh, *vl;          // packed data
  const int* vexp;
  const long long* off;
  const int* rows;
  const int4* items;              // (m, p, tile, 0)
  double2* alm;                   // [P][nalm]
  size_t astride;
  int R, N, P, lmax;
};

__global__ void __launch_bounds__(128) k_tc_analysis(TcAnalysisArgs g, int* d_err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const uint32_t raw = umma::smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int N = g.N;
  uint8_t* sAh = base;
  uint8_t* sAl = sAh + 16384;
  uint8_t* sBh = sAl + 16384;
  uint8_t* sBl = sBh + ((N * 128 + 1023) & ~1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 it = g.items[blockIdx.x];
  const int m = it.x, p = it.y, tile = it.z;
  const int grp = 2 * m + p;
  const size_t row0 = g.off[grp] + (size_t)tile * 128;
  const __half* Vh = g.vh + (size_t)grp * N * g.R;
  const __half* Vl = g.vl + (size_t)grp * N * g.R;
  int ncols = 32;
  while (ncols < N) ncols <<= 1;
  if (threadIdx.x == 0) {
    umma::mbar_init(&mbar, 1);
    abort_flag = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tmem_base, ncols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma::idesc_f16_f32(128, N);
  uint32_t phase = 0;
  for (int k0 = 0; k0 < g.R; k0 += 64) {
    for (int t = threadIdx.x; t < 128 * 8; t += blockDim.x) {
      const int r = t >> 3, c = t & 7;
      const size_t o = (row0 + r) * g.R + k0 + c * 8;
      *reinterpret_cast<uint4*>(sAh + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(g.th + o);
      *reinterpret_cast<uint4*>(sAl + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(g.tl + o);
    }
    for (int t = threadIdx.x; t < N * 8; t += blockDim.x) {
      const int r = t >> 3, c = t & 7;
      const size_t o = (size_t)r * g.R + k0 + c * 8;
      *reinterpret_cast<uint4*>(sBh + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Vh + o);
      *reinterpret_cast<uint4*>(sBl + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Vl + o);
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma::fence_after_sync();
      const uint64_t dAh = umma::desc_sw128(umma::smem_u32(sAh)), dAl = umma::desc_sw128(umma::smem_u32(sAl));
      const uint64_t dBh = umma::desc_sw128(umma::smem_u32(sBh)), dBl = umma::desc_sw128(umma::smem_u32(sBl));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t adv = (uint64_t)(kk * 32) >> 4;
        umma::mma_f16(tmem, dAh + adv, dBh + adv, idesc, (k0 | kk) != 0);
        umma::mma_f16(tmem, dAh + adv, dBl + adv, idesc, 1);
        umma::mma_f16(tmem, dAl + adv, dBh + adv, idesc, 1);
      }
      umma::commit(&mbar);
    }
    if (!umma::mbar_wait(&mbar, phase, kTcWaitPolls)) {
      if (lane == 0) atomicCAS(d_err, 0, kDevTimeout);
      abort_flag = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
  }
  umma::fence_after_sync();
  if (!abort_flag) {
    const int k = tile * 128 + warp * 32 + lane;
    const int l = m + p + 2 * k;
    const bool valid = k < g.rows[grp] && l <= g.lmax;
    const int* ve = g.vexp + (size_t)grp * N;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (valid) {
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const int pl = (c0 + i) >> 1;
          if (pl < g.P) {
            const double re = ldexp((double)v[i], -kTabExp - ve[c0 + i]);
            const double imv = ldexp((double)v[i + 1], -kTabExp - ve[c0 + i + 1]);
            g.alm[pl * g.astride + alm_idx(g.lmax, l, m)] = make_double2(re, imv);
          }
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

struct TcSynthesisArgs {
  const __half *th, *tl;
  const __half *sh, *sl;
  const int* sexp;
  const long long *off, *soff;
  const int* pad;
  float2* G;                      // [P][nq][lmax + 2][ld]
  size_t gstride, qstride;
  int R, N, P, nq, lmax, nside, ld;
};

// Block (ring tile, m): both parities, accumulators at TMEM columns [0, N) and [N, 2N)
__global__ void __launch_bounds__(128) k_tc_synthesis(TcSynthesisArgs g, int* d_err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const uint32_t raw = umma::smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int N = g.N;
  uint8_t* sAh = base;
  uint8_t* sAl = sAh + 16384;
  uint8_t* sBh = sAl + 16384;
  uint8_t* sBl = sBh + ((N * 128 + 1023) & ~1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, m = blockIdx.y;
  const int ring0 = tile * 128;
  int ncols = 32;
  while (ncols < 2 * N) ncols <<= 1;
  if (threadIdx.x == 0) {
    umma::mbar_init(&mbar, 1);
    abort_flag = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tmem_base, ncols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma::idesc_f16_f32_amn(128, N);
  uint32_t phase = 0;
  for (int p = 0; p < 2 && !abort_flag; ++p) {
    const int grp = 2 * m + p;
    const int K = g.pad[grp];
    const size_t trow0 = g.off[grp];
    const __half* Sh = g.sh + g.soff[grp];
    const __half* Sl = g.sl + g.soff[grp];
    for (int k0 = 0; k0 < K; k0 += 64) {
      // A = T^T as an MN-major operand, copied without transposition: table
      // rows k0..k0+63 (K) x rings ring0..ring0+127 (M), two 64-ring atoms
      // columns 8 KB apart, each [k row][64 rings] in the 128-byte swizzle
      for (int t = threadIdx.x; t < 64 * 16; t += blockDim.x) {
        const int kk = t >> 4, rc = t & 15;
        const size_t o = (trow0 + k0 + kk) * g.R + ring0 + rc * 8;
        const uint32_t so = (uint32_t)(rc >> 3) * 8192u + umma::sw128_offset(kk, rc & 7);
        *reinterpret_cast<uint4*>(sAh + so) = *reinterpret_cast<const uint4*>(g.th + o);
        *reinterpret_cast<uint4*>(sAl + so) = *reinterpret_cast<const uint4*>(g.tl + o);
      }
      for (int t = threadIdx.x; t < N * 8; t += blockDim.x) {
        const int r = t >> 3, c = t & 7;
        const size_t o = (size_t)r * K + k0 + c * 8;
        *reinterpret_cast<uint4*>(sBh + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Sh + o);
        *reinterpret_cast<uint4*>(sBl + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Sl + o);
      }
      umma::fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        umma::fence_after_sync();
        const uint64_t dAh = umma::desc_sw128_mn(umma::smem_u32(sAh), 8192, 1024);
        const uint64_t dAl = umma::desc_sw128_mn(umma::smem_u32(sAl), 8192, 1024);
        const uint64_t dBh = umma::desc_sw128(umma::smem_u32(sBh)), dBl = umma::desc_sw128(umma::smem_u32(sBl));
        const uint32_t td = tmem + (uint32_t)(p * N);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t adva = (uint64_t)(kk * 2048) >> 4;   // two 8-row K atoms
          const uint64_t advb = (uint64_t)(kk * 32) >> 4;     // 16 fp16 along the K-major row
          umma::mma_f16(td, dAh + adva, dBh + advb, idesc, (k0 | kk) != 0);
          umma::mma_f16(td, dAh + adva, dBl + advb, idesc, 1);
          umma::mma_f16(td, dAl + adva, dBh + advb, idesc, 1);
        }
        umma::commit(&mbar);
      }
      if (!umma::mbar_wait(&mbar, phase, kTcWaitPolls)) {
        if (lane == 0) atomicCAS(d_err, 0, kDevTimeout);
        abort_flag = 1;
      }
      phase ^= 1u;
      __syncthreads();
      if (abort_flag) break;
    }
  }
  umma::fence_after_sync();
  if (!abort_flag) {
    const int r = ring0 + warp * 32 + lane;
    const int i = r + 1;
    const bool has_s = i != 2 * g.nside;
    const int* ee = g.sexp + (size_t)(2 * m) * N;
    const int* eo = g.sexp + (size_t)(2 * m + 1) * N;
    const bool odd_exists = g.pad[2 * m + 1] > 0;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float ve[16], vo[16];
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, ve);
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(N + c0), vo);
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const int qp = (c0 + c) >> 1;
        const int q = qp / g.P, pl = qp % g.P;
        if (q >= g.nq) continue;
        const double er = ldexp((double)ve[c], -kTabExp - ee[c0 + c]), ei = ldexp((double)ve[c + 1], -kTabExp - ee[c0 + c + 1]);
        double orr = 0.0, oi = 0.0;
        if (odd_exists) {
          orr = ldexp((double)vo[c], -kTabExp - eo[c0 + c]);
          oi = ldexp((double)vo[c + 1], -kTabExp - eo[c0 + c + 1]);
        }
        float2* Gq = g.G + pl * g.gstride + q * g.qstride + (size_t)m * g.ld;
        Gq[i - 1] = make_float2((float)(er + orr), (float)(ei + oi));
        if (has_s) Gq[4 * g.nside - i - 1] = make_float2((float)(er - orr), (float)(ei - oi));
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// host

std::shared_ptr<TcTable> get_tc_table(clc_ctx* ctx, int nside, int lmax, int* rc) {
  const auto key = std::make_pair(nside, lmax);
  auto it = ctx->tc_tables.find(key);
  if (it != ctx->tc_tables.end()) {
    *rc = CLC_OK;
    return it->second;
  }
  auto T = std::make_shared<TcTable>();
  T->nside = nside;
  T->lmax = lmax;
  T->R = 2 * nside;
  const int lt = lmax + 1;
  const int G = 2 * (lmax + 1);
  T->h_off.resize(G);
  T->h_rows.resize(G);
  T->h_pad.resize(G);
  long long acc = 0;
  for (int m = 0; m <= lmax; ++m)
    for (int p = 0; p < 2; ++p) {
      const int rows = (m + p <= lt) ? (lt - m - p) / 2 + 1 : 0;
      const int pad = (rows + 63) / 64 * 64;
      T->h_off[2 * m + p] = acc;
      T->h_rows[2 * m + p] = rows;
      T->h_pad[2 * m + p] = pad;
      acc += pad;
    }
  T->total_rows = acc;
  const size_t bytes = (size_t)(acc + 128) * T->R * sizeof(__half);
  size_t fb = 0, tb = 0;
  cudaMemGetInfo(&fb, &tb);
  if (2 * bytes + (2ull << 30) > fb) {
    *rc = set_err(ctx, CLC_ENOMEM, "tensor-core Legendre table of " + std::to_string(2 * bytes >> 20) + " MiB does not fit");
    return nullptr;
  }
  auto alloc = [&](Buffer& b, size_t n) -> bool {
    b.bytes = n;
    if (cudaMalloc(&b.p, n) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return false;
    }
    return true;
  };
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
  std::vector<double> lognorm(lmax + 1);
  double ln = 0.5 * std::log2(1.0 / (4.0 * kPi));
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) ln += 0.5 * std::log2((2.0 * m + 1.0) / (2.0 * m));
    lognorm[m] = ln;
  }
  std::vector<int4> items;
  for (int m = 0; m <= lmax; ++m)
    for (int p = 0; p < 2; ++p)
      for (int t = 0; t * 128 < T->h_rows[2 * m + p]; ++t)
        if (m + p + 2 * (t * 128) <= lmax) items.push_back(make_int4(m, p, t, 0));
  T->nitems = (int)items.size();
  Buffer d_ab, d_ln;
  if (!alloc(T->items, sizeof(int4) * items.size()) || !alloc(T->hi, bytes) || !alloc(T->lo, bytes) || !alloc(T->off, sizeof(long long) * G) ||
      !alloc(T->rows, sizeof(int) * G) || !alloc(T->pad, sizeof(int) * G) || !alloc(d_ab, sizeof(double2) * ab.size()) ||
      !alloc(d_ln, sizeof(double) * lognorm.size())) {
    *rc = set_err(ctx, CLC_ENOMEM, "tensor-core Legendre table allocation failed");
    return nullptr;
  }
  cudaMemsetAsync(T->hi.p, 0, bytes, ctx->stream);
  cudaMemsetAsync(T->lo.p, 0, bytes, ctx->stream);
  cudaMemcpyAsync(T->off.p, T->h_off.data(), sizeof(long long) * G, cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(T->rows.p, T->h_rows.data(), sizeof(int) * G, cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(T->pad.p, T->h_pad.data(), sizeof(int) * G, cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(d_ab.p, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(d_ln.p, lognorm.data(), sizeof(double) * lognorm.size(), cudaMemcpyHostToDevice, ctx->stream);
  cudaMemcpyAsync(T->items.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, ctx->stream);
  dim3 grid((T->R + 127) / 128, lmax + 1);
  CLC_LAUNCH(ctx, "k_tc_table_build", k_tc_table_build, grid, 128, 0, nside, lmax, T->R,
             (const long long*)T->off.p, (const double*)d_ln.p, (const double2*)d_ab.p, (__half*)T->hi.p,
             (__half*)T->lo.p);
  *rc = launch_check(ctx, "k_tc_table_build");
  cudaStreamSynchronize(ctx->stream);
  if (*rc) return nullptr;
  ctx->tc_tables[key] = T;
  return T;
}

static int round16(int v) { return (v + 15) / 16 * 16; }

// Mixed-precision pure-SHT Poisson solve of P planes of the same (nside, lmax):
// kappa[pl] (device maps), outputs psi[pl] and the five lens fields per plane.
int poisson_sht_tc(clc_ctx* ctx, const double* const* kappa, int P, int nside, int lmax, double* const* psi,
                   const clc_derivs* out) {
  int rc;
  if (nside < 64) return set_err(ctx, CLC_EINVAL, "CLC_MIXED needs nside >= 64");
  const bool derivs = out != nullptr;
  const int nq = derivs ? 3 : 1;
  const int Na = round16(2 * P), Ns = round16(2 * nq * P);
  if (Na > 256 || 2 * Ns > 256) return set_err(ctx, CLC_EINVAL, "CLC_MIXED: too many planes in one batch");
  auto plan = get_fft_plan(ctx, nside, &rc);
  if (rc) return rc;
  auto T = get_tc_table(ctx, nside, lmax, &rc);
  if (rc) return rc;
  const int R = T->R, G = 2 * (lmax + 1);
  const int ldf = 4 * nside - 1;
  const size_t fstride = (size_t)ldf * (lmax + 1);
  const size_t na = (size_t)(lmax + 1) * (lmax + 2) / 2;
  long long spad_total = 0;
  std::vector<long long> soff(G);
  for (int g = 0; g < G; ++g) {
    soff[g] = spad_total;
    spad_total += (long long)Ns * T->h_pad[g];
  }
  const size_t qstride = (size_t)ldf * (lmax + 2);
  const size_t gstride = nq * qstride;
  // scratch: F (P planes), packed V (hi, lo), exponents, alm (P), packed S, G (P planes)
  const size_t bF = sizeof(float2) * fstride * P;
  const size_t bV = sizeof(__half) * (size_t)G * Na * R;
  const size_t bVe = sizeof(int) * (size_t)G * Na;
  const size_t bA = sizeof(double2) * na * P;
  const size_t bS = sizeof(__half) * (size_t)spad_total;
  const size_t bSe = sizeof(int) * (size_t)G * Ns;
  const size_t bG = sizeof(float2) * gstride * P;
  const size_t bSo = sizeof(long long) * G;
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t total = r256(bF) + 2 * r256(bV) + r256(bVe) + r256(bA) + 2 * r256(bS) + r256(bSe) + r256(bG) + r256(bSo);
  uint8_t* w = (uint8_t*)scratch(ctx, 6, total);
  if (!w) return CLC_ENOMEM;
  float2* F = (float2*)w; w += r256(bF);
  __half* vh = (__half*)w; w += r256(bV);
  __half* vl = (__half*)w; w += r256(bV);
  int* vexp = (int*)w; w += r256(bVe);
  double2* alm = (double2*)w; w += r256(bA);
  __half* sh = (__half*)w; w += r256(bS);
  __half* sl = (__half*)w; w += r256(bS);
  int* sexp = (int*)w; w += r256(bSe);
  float2* Gm = (float2*)w; w += r256(bG);
  long long* d_soff = (long long*)w;
  cudaMemcpyAsync(d_soff, soff.data(), bSo, cudaMemcpyHostToDevice, ctx->stream);
  // 1. ring FFTs (FP32) of every plane, quadrature weight included
  const double wq = 4.0 * kPi / (12.0 * (double)nside * nside);
  for (int pl = 0; pl < P; ++pl)
    if ((rc = ring_analysis_t<float>(ctx, *plan, kappa[pl], lmax, wq, (C2<float>*)(F + pl * fstride), ldf))) return rc;
  // 2. pack the analysis operand
  {
    const long long warps = (long long)G * Na;
    CLC_LAUNCH(ctx, "k_tc_pack_analysis", k_tc_pack_analysis, (int)((warps * 32 + 255) / 256), 256, 0, F, ldf,
               fstride, nside, lmax, P, Na, R, vh, vl, vexp);
  }
  // 3. analysis on the tensor cores: one CTA per (m, p, 128-row tile)
  {
    TcAnalysisArgs a;
    a.th = (const __half*)T->hi.p;
    a.tl = (const __half*)T->lo.p;
    a.vh = vh;
    a.vl = vl;
    a.vexp = vexp;
    a.off = (const long long*)T->off.p;
    a.rows = (const int*)T->rows.p;
    a.items = (const int4*)T->items.p;
    a.alm = alm;
    a.astride = na;
    a.R = R;
    a.N = Na;
    a.P = P;
    a.lmax = lmax;
    const int smem = 1024 + 2 * 16384 + 2 * ((Na * 128 + 1023) & ~1023);
    cudaFuncSetAttribute(k_tc_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    CLC_LAUNCH(ctx, "k_tc_analysis", k_tc_analysis, T->nitems, 128, smem, a, ctx->d_err);
    if ((rc = launch_check(ctx, "k_tc_analysis"))) return rc;
  }
  // 4. Poisson solve and synthesis right-hand sides
  {
    const long long warps = (long long)G * Ns;
    CLC_LAUNCH(ctx, "k_tc_pack_synthesis", k_tc_pack_synthesis, (int)((warps * 32 + 255) / 256), 256, 0, alm, na,
               lmax, P, nq, Ns, d_soff, (const int*)T->pad.p, sh, sl, sexp);
  }
  // 5. synthesis on the tensor cores: one CTA per (128-ring tile, m)
  {
    TcSynthesisArgs s;
    s.th = (const __half*)T->hi.p;
    s.tl = (const __half*)T->lo.p;
    s.sh = sh;
    s.sl = sl;
    s.sexp = sexp;
    s.off = (const long long*)T->off.p;
    s.soff = d_soff;
    s.pad = (const int*)T->pad.p;
    s.G = Gm;
    s.gstride = gstride;
    s.qstride = qstride;
    s.R = R;
    s.N = Ns;
    s.P = P;
    s.nq = nq;
    s.lmax = lmax;
    s.nside = nside;
    s.ld = ldf;
    const int smem = 1024 + 2 * 16384 + 2 * ((Ns * 128 + 1023) & ~1023);
    cudaFuncSetAttribute(k_tc_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    CLC_LAUNCH(ctx, "k_tc_synthesis", k_tc_synthesis, dim3(R / 128, lmax + 1), 128, smem, s, ctx->d_err);
    if ((rc = launch_check(ctx, "k_tc_synthesis"))) return rc;
  }
  // 6. ring FFT synthesis (FP32) of every plane
  for (int pl = 0; pl < P; ++pl) {
    double* o[6] = {psi ? psi[pl] : nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (derivs) {
      o[1] = out[pl].a_th;
      o[2] = out[pl].a_ph;
      o[3] = out[pl].u_tt;
      o[4] = out[pl].u_pp;
      o[5] = out[pl].u_tp;
    }
    if ((rc = ring_synthesis_t<float>(ctx, *plan, (const C2<float>*)(Gm + pl * gstride), ldf, lmax, derivs ? 1 : 0, o)))
      return rc;
  }
  return CLC_OK;
}

}  // namespace clc

using namespace clc;

// planes per tensor-core batch: the synthesis holds two accumulators of
// round16(2 nq P) FP32 columns each in at most 256 TMEM columns
int tc_planes_per_batch(bool derivs) { return derivs ? 21 : 64; }

extern "C" int clc_poisson_sht_batch(clc_ctx* ctx, const double* const* kappa, int nplanes, int nside, int lmax,
                                     int precision, double* const* psi, const clc_derivs* out) {
  if (!ctx) return CLC_EINVAL;
  if (!kappa || nplanes < 1 || !valid_nside(nside) || nside > 4096 || lmax < 1 || lmax > 4 * nside)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: bad arguments");
  for (int i = 0; i < nplanes; ++i)
    if (!kappa[i]) return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: null kappa plane");
  if (precision != CLC_FP64 && precision != CLC_MIXED)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_sht_batch: precision must be CLC_FP64 or CLC_MIXED");
  cudaSetDevice(ctx->device);
  if (precision == CLC_FP64) {
    for (int i = 0; i < nplanes; ++i) {
      const int rc = clc_poisson_sht(ctx, kappa[i], nside, lmax, CLC_FP64, psi ? psi[i] : nullptr, out ? &out[i] : nullptr);
      if (rc) return rc;
    }
    return CLC_OK;
  }
  if (!psi && !out) return CLC_OK;
  const int per = tc_planes_per_batch(out != nullptr);
  for (int i0 = 0; i0 < nplanes; i0 += per) {
    const int P = std::min(per, nplanes - i0);
    const int rc = poisson_sht_tc(ctx, kappa + i0, P, nside, lmax, psi ? psi + i0 : nullptr, out ? out + i0 : nullptr);
    if (rc) return rc;
  }
  return CLC_OK;
}
