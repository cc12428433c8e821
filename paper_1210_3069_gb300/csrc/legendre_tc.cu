// Mixed-precision, batched Legendre transforms of the SHT Poisson solve on the
// tcgen05 tensor cores (paper Sec. 3.2 transforms).  FP64 is used only by the
// scaled associated-Legendre recurrence that builds the table; the ring FFTs
// run in FP32 and the contractions as split FP16 hi + lo products with FP32
// accumulation in tensor memory.
//
// For every m the lambda table is split by the parity p of l - m (rows
// l = m + p + 2k), because the southern mirror ring enters with sign
// (-1)^(l+m).  The table holds 2^10 lambda_lm as FP16 hi + lo
// (|lambda_lm| <= sqrt((2l+1)/4 pi) < 52 for l <= 16385, so the scaled values
// stay below the FP16 maximum and small values keep more bits before lo turns
// subnormal).  All planes of a batch class share it:
//   analysis   D[k][col]      = sum_ring T[m,p][k][ring] V[m,p][col][ring]
//              (col = plane, re/im; V = F_north +- F_south),
//   synthesis  D_p[ring][col] = sum_k T[m,p][k][ring] S[m,p][col][k]
//              (col = right-hand side, plane, re/im), both parities in one
//              CTA with two TMEM accumulators, combined in the epilogue into
//              the northern (even + odd) and southern (even - odd) rings.
// Data operands are split into FP16 hi + lo after scaling each column by a
// power of two (max -> [2^13, 2^14)); products hi*hi + hi*lo + lo*hi
// accumulate in FP32.  Every operand tile lives in global memory already in
// the 128-byte-swizzled shared-memory layout, so a pipeline stage is a few
// contiguous bulk copies (TMA engine) completing on an mbarrier; one thread
// issues the copies, another the MMAs, and the four warps read the
// accumulators back.  All kernels are persistent: each CTA walks a work list
// spanning every class of the batch.
#include <algorithm>
#include <map>

#include "legendre_tc.cuh"
#include "ring_fft.cuh"
#include "legendre.cuh"
#include "umma.cuh"

namespace clc {

constexpr long long kTcWaitPolls = 1ll << 26;
constexpr int kTcMaxStages = 4;

// half offset of element (row r, column c < 64) inside a tile of 64-half rows
// in the 128-byte swizzle (8-row groups of 1024 bytes)
__host__ __device__ __forceinline__ uint32_t atom_off(int r, int c) {
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + (((c >> 3) ^ (r & 7)) << 3) + (c & 7));
}

// FP32 x * 2^e, exact while the result is a normal float
__device__ __forceinline__ float times_pow2f(float x, int e) {
  if (e >= -126 && e <= 127) return x * __int_as_float((e + 127) << 23);
  return ldexpf(x, e);
}

// power-of-two exponent that brings a column maximum into [2^13, 2^14)
__device__ __forceinline__ int col_exponent(float mx) {
  if (!(mx > 0.f)) return 0;
  int ex;
  frexpf(mx, &ex);
  return 14 - ex;
}

__device__ __forceinline__ void put_split2(__half* hi, __half* lo, size_t i, float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  *reinterpret_cast<__half2*>(hi + i) = h;
  *reinterpret_cast<__half2*>(lo + i) = __floats2half2_rn(a - hf.x, b - hf.y);
}

// ---------------------------------------------------------------------------
// table build: the FP64 scaled recurrence of legendre.cu, written as FP16 hi/lo

__device__ __forceinline__ double tc_scale_pow2(double p, int e) {
  if (e >= -1022) return p * __longlong_as_double((long long)(e + 1023) << 52);
  if (e < -1600) return 0.0;
  return (p * __longlong_as_double((long long)(e + 600 + 1023) << 52)) * 0x1p-600;
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
  const size_t ratoms = (size_t)(R >> 6);
  auto store = [&](int l, double p) {
    const int par = (l - m) & 1;
    const long long row = off[2 * m + par] + (l - m - par) / 2;
    const size_t i = ((size_t)(row >> 6) * ratoms + (size_t)(r >> 6)) * 4096 + atom_off((int)(row & 63), r & 63);
    const double v = tc_scale_pow2(p, e + kTabExp);
    const __half h = __double2half(v);
    hi[i] = h;
    lo[i] = __double2half(v - (double)__half2float(h));
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
    *rc = set_err(ctx, CLC_ENOMEM,
                  "tensor-core Legendre table of " + std::to_string(2 * bytes >> 20) + " MiB does not fit");
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
  Buffer d_ab, d_ln;
  if (!alloc(T->hi, bytes) || !alloc(T->lo, bytes) || !alloc(T->off, sizeof(long long) * G) ||
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
  dim3 grid((T->R + 127) / 128, lmax + 1);
  CLC_LAUNCH(ctx, "k_tc_table_build", k_tc_table_build, grid, 128, 0, nside, lmax, T->R,
             (const long long*)T->off.p, (const double*)d_ln.p, (const double2*)d_ab.p, (__half*)T->hi.p,
             (__half*)T->lo.p);
  *rc = launch_check(ctx, "k_tc_table_build");
  // the coefficient buffers are freed on return: wait for the build
  cudaStreamSynchronize(ctx->stream);
  if (*rc) return nullptr;
  ctx->tc_tables[key] = T;
  return T;
}

// ---------------------------------------------------------------------------
// flat item spaces over the classes of a batch

__device__ __forceinline__ int find_class(const TcBatchDev& b, long long idx, long long TcClass::*first) {
  int c = 0;
  while (c + 1 < b.ncls && idx >= b.cls[c + 1].*first) ++c;
  return c;
}

// ---------------------------------------------------------------------------
// ring FFTs (FP32) of every plane of every class; one ring per CTA at a time
// (512 threads for the six-field synthesis, 256 for the analysis)

constexpr int kRingThreads = 512;

__global__ void k_tc_ring_analysis(TcBatchDev b) {
  extern __shared__ __align__(16) unsigned char smem_ra[];
  C2<float>* s = reinterpret_cast<C2<float>*>(smem_ra);
  for (long long it = blockIdx.x; it < b.n_ring; it += gridDim.x) {
    const TcClass& C = b.cls[find_class(b, it, &TcClass::ring0)];
    const long long loc = it - C.ring0;
    const int nr = 4 * C.nside - 1;
    const int pl = (int)(loc / nr), i = (int)(loc % nr) + 1;
    ring_analysis_ring<float>(b.kappa[C.plane0 + pl], C.nside, C.lmax, C.wq,
                              reinterpret_cast<C2<float>*>(C.F + pl * C.fstride), C.ldf, C.fft, i, s);
  }
}

__global__ void __launch_bounds__(kRingThreads, 2) k_tc_ring_synthesis(TcBatchDev b) {
  extern __shared__ __align__(16) unsigned char smem_rs[];
  C2<float>* s = reinterpret_cast<C2<float>*>(smem_rs);
  for (long long it = blockIdx.x; it < b.n_ring; it += gridDim.x) {
    const TcClass& C = b.cls[find_class(b, it, &TcClass::ring0)];
    const long long loc = it - C.ring0;
    const int nr = 4 * C.nside - 1;
    const int pl = (int)(loc / nr), i = (int)(loc % nr) + 1;
    SynthArgsT<float> a;
    const float2* Gp = C.G + pl * C.gstride;
    a.G0 = reinterpret_cast<const C2<float>*>(Gp);
    a.G1 = reinterpret_cast<const C2<float>*>(Gp + C.qstride);
    a.G2 = reinterpret_cast<const C2<float>*>(Gp + 2 * C.qstride);
    a.sm = 4ll * C.ldf;
    a.sr = 4;
    a.quad = 1;
    a.P01 = b.mode ? reinterpret_cast<const C2<double>*>(C.G01 + (size_t)pl * C.nq * 2 * C.ldf) : nullptr;
    a.p01q = 2ll * C.ldf;
    a.p01m = C.ldf;
    a.ncap = C.ncap;
    a.nring = C.ldf;
    double* const* o = b.out + (size_t)(C.plane0 + pl) * 6;
    for (int f = 0; f < 6; ++f) a.out[f] = o[f];
    ring_synthesis_ring<float>(a, C.nside, C.lmax, b.mode, C.fft, i, s, s + fft_buf_len<float>(C.mmax));
  }
}

// ---------------------------------------------------------------------------
// FP64 Legendre sums of the orders m = 0, 1 (derivative mode).  At the rings
// next to the poles the Hessian terms of these two orders are differences of
// 1/sin^2(theta)-sized parts, so the synthesis takes them from these sums
// instead of the tensor-core ones (the FP32 rounding of the latter would be
// amplified by up to Nside^2).  Only the ncap rings next to each pole
// (sin theta < 0.29) need them.  One thread per (plane, northern cap ring,
// which also gives its southern mirror); the unscaled recurrence is safe for
// m <= 1.

__global__ void k_tc_low_orders(TcBatchDev b) {
  for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < b.n_low;
       it += (long long)gridDim.x * blockDim.x) {
    const TcClass& C = b.cls[find_class(b, it, &TcClass::low0)];
    const long long loc = it - C.low0;
    const int ns = C.nside, L = C.lmax;
    const int pl = (int)(loc / C.ncap), i = (int)(loc % C.ncap) + 1;
    const Ring g = ring_geom(ns, i);
    const double z = g.z;
    const bool has_s = i != 2 * ns;
    const float2* a = C.alm + pl * C.astride;
    double2* out = C.G01 + (size_t)pl * C.nq * 2 * C.ldf;
    for (int m = 0; m <= 1; ++m) {
      const double* co = C.co01 + (size_t)m * (L + 3) * 4;
      auto kap = [&](int l) -> double2 {
        if (l < m || l > L || l < 1) return make_double2(0.0, 0.0);
        const float2 v = a[alm_idx(L, l, m)];
        return make_double2((double)v.x, m ? (double)v.y : 0.0);
      };
      auto psi = [&](int l) -> double2 {
        const double2 k = kap(l);
        const double d = (l >= 1 && l <= L) ? co[4 * l + 3] : 0.0;
        return make_double2(k.x * d, k.y * d);
      };
      double2 n0 = make_double2(0, 0), n1 = n0, n2 = n0, s0 = n0, s1 = n0, s2 = n0;
      double p2 = m == 0 ? 0.28209479177387814347 : -0.34549414947133547927 * g.s;   // lambda_mm
      double p1 = 0.0;
      double2 pm1 = psi(m - 1), p0 = psi(m), pp1 = psi(m + 1);
      for (int l = m; l <= L + 1; ++l) {
        double lam;
        if (l == m) {
          lam = p2;
        } else if (l == m + 1) {
          p1 = sqrt(2.0 * m + 3.0) * z * p2;
          lam = p1;
        } else {
          lam = co[4 * l] * (z * p1 - co[4 * l + 1] * p2);
          p2 = p1;
          p1 = lam;
        }
        const double c1 = (l - 1.0) * co[4 * l + 2], c2 = (l + 2.0) * co[4 * (l + 1) + 2];
        const double2 bl = make_double2(c1 * pm1.x - c2 * pp1.x, c1 * pm1.y - c2 * pp1.y);
        const double2 kb = (l >= 1 && l <= L) ? kap(l) : make_double2(0.0, 0.0);
        const double sg = ((l + m) & 1) ? -1.0 : 1.0;
        n0.x += p0.x * lam; n0.y += p0.y * lam;
        n1.x += bl.x * lam; n1.y += bl.y * lam;
        n2.x += kb.x * lam; n2.y += kb.y * lam;
        s0.x += sg * p0.x * lam; s0.y += sg * p0.y * lam;
        s1.x += sg * bl.x * lam; s1.y += sg * bl.y * lam;
        s2.x += sg * kb.x * lam; s2.y += sg * kb.y * lam;
        pm1 = p0;
        p0 = pp1;
        pp1 = psi(l + 2);
      }
      const size_t q = 2 * (size_t)C.ldf, mo = (size_t)m * C.ldf;
      out[mo + i - 1] = n0;
      out[q + mo + i - 1] = n1;
      out[2 * q + mo + i - 1] = n2;
      if (has_s) {
        const size_t j = 4 * ns - i - 1;
        out[mo + j] = s0;
        out[q + mo + j] = s1;
        out[2 * q + mo + j] = s2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// operand packing (FP32 arithmetic)

// analysis operand of order m (both parities): V[2m+p][ring block][col][64],
// col = 2 plane + re/im, values F_north +- F_south of ring r
__global__ void k_tc_pack_analysis(TcBatchDev b) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long it = blockIdx.x; it < b.n_pa; it += gridDim.x) {
    const TcClass& C = b.cls[find_class(b, it, &TcClass::pa0)];
    const int m = (int)(it - C.pa0);
    const int R = C.R, N = C.Na, ns = C.nside;
    const size_t blk = (size_t)N * 64;
    const size_t be = (size_t)(2 * m) * (R / 64) * blk, bo = be + (size_t)(R / 64) * blk;
    for (int col = warp; col < N; col += nw) {
      const int pl = col >> 1, im = col & 1;
      if (pl >= C.P) {
        for (int r = 2 * lane; r < R; r += 64) {
          const size_t o = (size_t)(r >> 6) * blk + atom_off(col, r & 63);
          put_split2(C.vh, C.vl, be + o, 0.f, 0.f);
          put_split2(C.vh, C.vl, bo + o, 0.f, 0.f);
        }
        if (lane == 0) C.vexp[(2 * m) * N + col] = C.vexp[(2 * m + 1) * N + col] = 0;
        continue;
      }
      const float* Fm = reinterpret_cast<const float*>(C.F + pl * C.fstride + (size_t)m * C.ldf) + im;
      auto vals = [&](int r, float& e, float& o) {
        const float a = Fm[2 * r];
        const float s = (r + 1 != 2 * ns) ? Fm[2 * (4 * ns - r - 2)] : 0.f;
        e = a + s;
        o = a - s;
      };
      float mxe = 0.f, mxo = 0.f;
      for (int r = 2 * lane; r < R; r += 64) {
        float e0, o0, e1, o1;
        vals(r, e0, o0);
        vals(r + 1, e1, o1);
        mxe = fmaxf(mxe, fmaxf(fabsf(e0), fabsf(e1)));
        mxo = fmaxf(mxo, fmaxf(fabsf(o0), fabsf(o1)));
      }
      for (int o = 16; o > 0; o >>= 1) {
        mxe = fmaxf(mxe, __shfl_xor_sync(0xffffffffu, mxe, o));
        mxo = fmaxf(mxo, __shfl_xor_sync(0xffffffffu, mxo, o));
      }
      const int xe = col_exponent(mxe), xo = col_exponent(mxo);
      for (int r = 2 * lane; r < R; r += 64) {
        float e0, o0, e1, o1;
        vals(r, e0, o0);
        vals(r + 1, e1, o1);
        const size_t o = (size_t)(r >> 6) * blk + atom_off(col, r & 63);
        put_split2(C.vh, C.vl, be + o, times_pow2f(e0, xe), times_pow2f(e1, xe));
        put_split2(C.vh, C.vl, bo + o, times_pow2f(o0, xo), times_pow2f(o1, xo));
      }
      if (lane == 0) {
        C.vexp[(2 * m) * N + col] = xe;
        C.vexp[(2 * m + 1) * N + col] = xo;
      }
    }
  }
}

// synthesis right-hand sides of group (m, p): S[soff + t Ns 64][col][64],
// col = (q P + plane) 2 + re/im.  With psi_lm = -kappa_lm / (l (l + 1)):
//   q = 0: psi_lm                              = D0_l kappa_lm,
//   q = 1: b_lm = (l-1) eps_lm psi_{l-1,m} - (l+2) eps_{l+1,m} psi_{l+1,m}
//               = A1_l kappa_{l-1,m} + A2_l kappa_{l+1,m},
//          A1_l = -eps_lm / l, A2_l = eps_{l+1,m} / (l + 1),
//   q = 2: kappa_bl = -l (l + 1) psi_lm        = kappa_lm for l >= 1,
// terms outside 1 <= l' <= lmax being zero; eps_lm = sqrt((l^2 - m^2) / (4 l^2 - 1)).
__device__ __forceinline__ float tc_epsf(int l, int m) {
  if (l <= m) return 0.f;
  return sqrtf((float)((l - m) * (l + m)) / (float)((2 * l - 1) * (2 * l + 1)));
}

__global__ void k_tc_pack_synthesis(TcBatchDev b) {
  extern __shared__ float coef[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (long long it = blockIdx.x; it < b.n_ps; it += gridDim.x) {
    const TcClass& C = b.cls[find_class(b, it, &TcClass::ps0)];
    const int grp = (int)(it - C.ps0);
    const int m = grp >> 1, p = grp & 1, lmax = C.lmax, N = C.Ns;
    const int K = C.pad[grp];
    float* D0 = coef;
    float* A1 = coef + K;
    float* A2 = coef + 2 * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const int l = m + p + 2 * k;
      float d0 = 0.f, a1 = 0.f, a2 = 0.f;
      if (l <= lmax + 1) {
        if (l >= 1 && l <= lmax) d0 = -1.f / ((float)l * (float)(l + 1));
        if (l - 1 >= 1 && l - 1 <= lmax) a1 = -tc_epsf(l, m) / (float)l;
        if (l + 1 <= lmax) a2 = tc_epsf(l + 1, m) / (float)(l + 1);
      }
      D0[k] = d0;
      A1[k] = a1;
      A2[k] = a2;
    }
    __syncthreads();
    const size_t base = C.soff[grp];
    const size_t blk = (size_t)N * 64;
    for (int col = warp; col < N; col += nw) {
      const int im = col & 1, qp = col >> 1, q = qp / C.P, pl = qp % C.P;
      if (q >= C.nq || (m == 0 && im)) {
        for (int k = 2 * lane; k < K; k += 64)
          put_split2(C.sh, C.sl, base + (size_t)(k >> 6) * blk + atom_off(col, k & 63), 0.f, 0.f);
        if (lane == 0) C.sexp[grp * N + col] = 0;
        continue;
      }
      const float* a = reinterpret_cast<const float*>(C.alm + pl * C.astride) + im;
      auto kap = [&](int l) -> float { return (l >= m && l <= lmax) ? a[2 * alm_idx(lmax, l, m)] : 0.f; };
      auto val = [&](int k) -> float {
        const int l = m + p + 2 * k;
        if (q == 0) return D0[k] * kap(l);
        if (q == 1) return A1[k] * kap(l - 1) + A2[k] * kap(l + 1);
        return D0[k] != 0.f ? kap(l) : 0.f;
      };
      float mx = 0.f;
      for (int k = 2 * lane; k < K; k += 64) mx = fmaxf(mx, fmaxf(fabsf(val(k)), fabsf(val(k + 1))));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int x = col_exponent(mx);
      for (int k = 2 * lane; k < K; k += 64)
        put_split2(C.sh, C.sl, base + (size_t)(k >> 6) * blk + atom_off(col, k & 63), times_pow2f(val(k), x),
                   times_pow2f(val(k + 1), x));
      if (lane == 0) C.sexp[grp * N + col] = x;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// tensor-core contractions: persistent, warp-specialised, bulk-copy pipelined
//
// Analysis item (class, group, 128-row tile): K runs over the R rings in
// stages of 64; A = two 8 KB table atoms (rows 0-63 and 64-127 of the tile),
// B = the group's operand block of the stage's ring block.
// Synthesis item (class, m, 128-ring tile): K runs over the padded rows of
// parity 0 then parity 1; A = the two adjacent atoms of the tile's 128 rings
// (MN-major), B = the right-hand-side block.
//
// The tensor cores add each MMA into the FP32 accumulator with truncation,
// an error that grows with the number of accumulation steps.  So the MMAs
// accumulate in TMEM only over a chunk of kFlush stages; the four epilogue
// warps then add the chunk into a running sum held in a second TMEM region
// with round-to-nearest FP32 adds, and release the chunk accumulator.
// Warps 0-3: epilogue (TMEM lanes 32w..32w+31), warp 4: bulk-copy producer,
// warp 5: MMA issuer.  TMEM columns: chunk [0, W), sum [W, 2W), W = Nmax
// (analysis) or 2 Nmax (synthesis, parity p at p Nmax), Nmax the widest
// operand of the launch: the next item's first chunk may be accumulating
// while the epilogue still reads the previous item's sums, so the regions
// must not move with the width of the item.

constexpr int kFlush = 2;   // pipeline stages per TMEM accumulation chunk

template <bool kSyn>
struct GemmItem {
  int nk, N, K0, nch0, nch;   // stages, columns, parity-0 stages, parity-0 chunks, chunks
  __device__ __forceinline__ void init(const TcBatchDev& b, int4 w) {
    const TcClass& C = b.cls[w.x];
    if (kSyn) {
      N = C.Ns;
      K0 = C.pad[2 * w.y] >> 6;
      const int K1 = C.pad[2 * w.y + 1] >> 6;
      nk = K0 + K1;
      nch0 = (K0 + kFlush - 1) / kFlush;
      nch = nch0 + (K1 + kFlush - 1) / kFlush;
    } else {
      N = C.Na;
      nk = K0 = C.R >> 6;
      nch0 = nch = (nk + kFlush - 1) / kFlush;
    }
  }
  // chunk of stage k, and whether k starts / ends its chunk
  __device__ __forceinline__ int chunk(int k) const { return k < K0 ? k / kFlush : nch0 + (k - K0) / kFlush; }
  __device__ __forceinline__ bool starts(int k) const { return k < K0 ? k % kFlush == 0 : (k - K0) % kFlush == 0; }
  __device__ __forceinline__ bool ends(int k) const {
    return k + 1 == nk || k + 1 == K0 || (k < K0 ? (k + 1) % kFlush == 0 : (k + 1 - K0) % kFlush == 0);
  }
};

template <bool kSyn>
__global__ void __launch_bounds__(192) k_tc_gemm(TcBatchDev b, const int4* __restrict__ items, int nitems, int S,
                                                 int bB, int nmax, int tcols, int* d_err) {
  extern __shared__ __align__(16) uint8_t smem_g[];
  __shared__ uint64_t full[kTcMaxStages], empty[kTcMaxStages], chunkb, freeb, drainb;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const uint32_t raw = umma::smem_u32(smem_g);
  uint8_t* base = smem_g + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t stage_bytes = 2u * 16384u + 2u * (uint32_t)bB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(&chunkb, 1);
    umma::mbar_init(&freeb, 128);
    umma::mbar_init(&drainb, 1);
    abort_flag = 0;
    umma::fence_mbar_init();
  }
  if (warp == 0) umma::tmem_alloc(&tmem_base, tcols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  auto fail = [&]() {
    atomicCAS(d_err, 0, kDevTimeout);
    abort_flag = 1;
  };

  if (warp == 4) {
    // ---- producer: bulk copies of every stage of every item
    if (lane == 0) {
      uint32_t it = 0;
      int last_it[kTcMaxStages];
      for (int s = 0; s < kTcMaxStages; ++s) last_it[s] = -1;
      for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
        const int4 w = items[item];
        const TcClass& C = b.cls[w.x];
        GemmItem<kSyn> gi;
        gi.init(b, w);
        const int RA = C.R >> 6;
        const uint32_t bbytes = (uint32_t)gi.N * 128u;
        for (int k = 0; k < gi.nk; ++k, ++it) {
          const int s = (int)(it % (uint32_t)S);
          const uint32_t u = it / (uint32_t)S;
          if (u > 0 && !umma::mbar_wait(&empty[s], (u - 1) & 1u, kTcWaitPolls)) {
            fail();
            break;
          }
          uint8_t* st = base + (size_t)s * stage_bytes;
          umma::mbar_arrive_expect_tx(&full[s], 2u * 16384u + 2u * bbytes);
          if (kSyn) {
            const int p = k < gi.K0 ? 0 : 1, t = p ? k - gi.K0 : k;
            const int grp = 2 * w.y + p;
            const size_t a = ((size_t)(C.off[grp] / 64 + t) * RA + 2 * w.z) * 4096;
            umma::bulk_g2s(st, C.th + a, 16384u, &full[s]);
            umma::bulk_g2s(st + 16384, C.tl + a, 16384u, &full[s]);
            const size_t bo = (size_t)C.soff[grp] + (size_t)t * gi.N * 64;
            umma::bulk_g2s(st + 32768, C.sh + bo, bbytes, &full[s]);
            umma::bulk_g2s(st + 32768 + bB, C.sl + bo, bbytes, &full[s]);
          } else {
            const size_t rb = (size_t)((C.off[w.y] + (long long)w.z * 128) / 64);
            const size_t a0 = (rb * RA + k) * 4096, a1 = ((rb + 1) * RA + k) * 4096;
            umma::bulk_g2s(st, C.th + a0, 8192u, &full[s]);
            umma::bulk_g2s(st + 8192, C.th + a1, 8192u, &full[s]);
            umma::bulk_g2s(st + 16384, C.tl + a0, 8192u, &full[s]);
            umma::bulk_g2s(st + 16384 + 8192, C.tl + a1, 8192u, &full[s]);
            const size_t bo = ((size_t)w.y * RA + k) * (size_t)gi.N * 64;
            umma::bulk_g2s(st + 32768, C.vh + bo, bbytes, &full[s]);
            umma::bulk_g2s(st + 32768 + bB, C.vl + bo, bbytes, &full[s]);
          }
          last_it[s] = (int)it;
        }
      }
      if (abort_flag)
        for (int s = 0; s < S; ++s)   // bounded drain of the copies in flight
          if (last_it[s] >= 0) umma::mbar_wait(&full[s], (uint32_t)(last_it[s] / S) & 1u, kTcWaitPolls);
    }
  } else if (warp == 5) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, nchunk = 0;
      for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
        const int4 w = items[item];
        GemmItem<kSyn> gi;
        gi.init(b, w);
        const int N = gi.N;
        const uint32_t idesc = kSyn ? umma::idesc_f16_f32_amn(128, N) : umma::idesc_f16_f32(128, N);
        for (int k = 0; k < gi.nk && !abort_flag; ++k, ++it) {
          const bool first = gi.starts(k);
          if (first && nchunk > 0 && !umma::mbar_wait(&freeb, (nchunk - 1) & 1u, kTcWaitPolls)) {
            fail();   // the epilogue has not released the chunk accumulator
            break;
          }
          const int s = (int)(it % (uint32_t)S);
          if (!umma::mbar_wait(&full[s], (it / (uint32_t)S) & 1u, kTcWaitPolls)) {
            fail();
            break;
          }
          umma::fence_after_sync();
          uint8_t* st = base + (size_t)s * stage_bytes;
          const uint32_t sa = umma::smem_u32(st), sb = umma::smem_u32(st + 32768);
          const int p = (kSyn && k >= gi.K0) ? 1 : 0;
          const uint32_t td = tmem + (uint32_t)(p * nmax);
          uint64_t dAh, dAl;
          if (kSyn) {
            dAh = umma::desc_sw128_mn(sa, 8192, 1024);
            dAl = umma::desc_sw128_mn(sa + 16384, 8192, 1024);
          } else {
            dAh = umma::desc_sw128(sa);
            dAl = umma::desc_sw128(sa + 16384);
          }
          const uint64_t dBh = umma::desc_sw128(sb), dBl = umma::desc_sw128(sb + (uint32_t)bB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adva = kSyn ? (uint64_t)(kk * 2048) >> 4 : (uint64_t)(kk * 32) >> 4;
            const uint64_t advb = (uint64_t)(kk * 32) >> 4;
            umma::mma_f16(td, dAh + adva, dBh + advb, idesc, (first && kk == 0) ? 0u : 1u);
            umma::mma_f16(td, dAh + adva, dBl + advb, idesc, 1);
            umma::mma_f16(td, dAl + adva, dBh + advb, idesc, 1);
          }
          umma::commit(&empty[s]);
          if (gi.ends(k)) {
            umma::commit(&chunkb);
            ++nchunk;
          }
        }
      }
      if (abort_flag) {   // bounded wait for the MMAs in flight
        umma::commit(&drainb);
        umma::mbar_wait(&drainb, 0, kTcWaitPolls);
      }
    }
  } else {
    // ---- epilogue warps 0-3: fold chunks into the running sums, then write out
    uint32_t nchunk = 0;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int item = blockIdx.x; item < nitems && !__any_sync(0xffffffffu, abort_flag); item += gridDim.x) {
      const int4 w = items[item];
      const TcClass& C = b.cls[w.x];
      GemmItem<kSyn> gi;
      gi.init(b, w);
      const int N = gi.N;
      const uint32_t W = kSyn ? 2u * (uint32_t)nmax : (uint32_t)nmax;
      bool ok = true;
      for (int c = 0; c < gi.nch; ++c, ++nchunk) {
        // warp-uniform decision: the TMEM accesses below are whole-warp operations
        const bool got = umma::mbar_wait(&chunkb, nchunk & 1u, kTcWaitPolls);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const int p = c < gi.nch0 ? 0 : 1;
        const bool first = c == 0 || c == gi.nch0;
        const uint32_t cc = (uint32_t)(p * nmax), sc = W + (uint32_t)(p * nmax);
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          umma::tmem_ld16(trow + cc + (uint32_t)c0, v);
          if (!first) {
            float t[16];
            umma::tmem_ld16(trow + sc + (uint32_t)c0, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += t[i];
          }
          umma::tmem_st16(trow + sc + (uint32_t)c0, v);
        }
        umma::fence_before_sync();
        umma::mbar_arrive(&freeb);
      }
      if (!ok) break;
      __syncwarp();
      if (!kSyn) {
        const int grp = w.y, m = grp >> 1, p = grp & 1;
        const int k = w.z * 128 + warp * 32 + lane;
        const int l = m + p + 2 * k;
        const bool valid = k < C.rows[grp] && l <= C.lmax;
        const int* ve = C.vexp + (size_t)grp * N;
        float2* out = C.alm + alm_idx(C.lmax, l < C.lmax ? l : C.lmax, m);
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          umma::tmem_ld16(trow + W + (uint32_t)c0, v);
          if (valid) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const int pl = (c0 + i) >> 1;
              if (pl < C.P)
                out[pl * C.astride] = make_float2(times_pow2f(v[i], -kTabExp - ve[c0 + i]),
                                                  times_pow2f(v[i + 1], -kTabExp - ve[c0 + i + 1]));
            }
          }
        }
      } else {
        const int m = w.y;
        const int i = w.z * 128 + warp * 32 + lane + 1;   // ring
        const bool has_s = i != 2 * C.nside;
        const int* ee = C.sexp + (size_t)(2 * m) * N;
        const int* eo = C.sexp + (size_t)(2 * m + 1) * N;
        for (int c0 = 0; c0 < N; c0 += 16) {
          float ve[16], vo[16];
          umma::tmem_ld16(trow + W + (uint32_t)c0, ve);
          umma::tmem_ld16(trow + W + (uint32_t)(nmax + c0), vo);
#pragma unroll
          for (int c = 0; c < 16; c += 2) {
            const int qp = (c0 + c) >> 1;
            const int q = qp / C.P, pl = qp % C.P;
            if (q >= C.nq) continue;
            const float er = times_pow2f(ve[c], -kTabExp - ee[c0 + c]);
            const float ei = times_pow2f(ve[c + 1], -kTabExp - ee[c0 + c + 1]);
            const float orr = times_pow2f(vo[c], -kTabExp - eo[c0 + c]);
            const float oi = times_pow2f(vo[c + 1], -kTabExp - eo[c0 + c + 1]);
            float2* Gq = C.G + pl * C.gstride + q * C.qstride + (size_t)(m >> 2) * 4 * C.ldf + (m & 3);
            Gq[(size_t)(i - 1) * 4] = make_float2(er + orr, ei + oi);
            if (has_s) Gq[(size_t)(4 * C.nside - i - 1) * 4] = make_float2(er - orr, ei - oi);
          }
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// ---------------------------------------------------------------------------
// host

static int pow2_cols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

static int stage_b_bytes(int nmax) { return (nmax * 128 + 1023) / 1024 * 1024; }

int tc_build_items(clc_ctx* ctx, const TcBatchDev& b, const std::vector<std::shared_ptr<TcTable>>& tabs,
                   TcItems* it) {
  std::vector<std::pair<int, int4>> an, sy;   // (stages, item): longer items first
  it->na_max = 16;
  it->ns_max = 16;
  it->fft_an_smem = it->fft_sy_smem = it->pack_s_smem = 0;
  for (int c = 0; c < b.ncls; ++c) {
    const TcClass& C = b.cls[c];
    const TcTable& T = *tabs[c];
    it->na_max = std::max(it->na_max, C.Na);
    it->ns_max = std::max(it->ns_max, C.Ns);
    it->fft_an_smem = std::max(it->fft_an_smem, fft_buf_len<float>(C.mmax) * (int)sizeof(float2));
    it->fft_sy_smem = std::max(it->fft_sy_smem, (fft_buf_len<float>(C.mmax) + 2 * C.nside + 1) * (int)sizeof(float2));
    it->pack_s_smem = std::max(it->pack_s_smem, 3 * T.h_pad[0] * (int)sizeof(float));
    for (int m = 0; m <= C.lmax; ++m)
      for (int p = 0; p < 2; ++p)
        for (int t = 0; t * 128 < T.h_rows[2 * m + p]; ++t)
          if (m + p + 2 * (t * 128) <= C.lmax) an.push_back({C.R / 64, make_int4(c, 2 * m + p, t, 0)});
    for (int m = 0; m <= C.lmax; ++m)
      for (int rt = 0; rt < C.R / 128; ++rt)
        sy.push_back({(T.h_pad[2 * m] + T.h_pad[2 * m + 1]) / 64, make_int4(c, m, rt, 0)});
  }
  auto by_len = [](const std::pair<int, int4>& x, const std::pair<int, int4>& y) { return x.first > y.first; };
  std::stable_sort(an.begin(), an.end(), by_len);
  std::stable_sort(sy.begin(), sy.end(), by_len);
  std::vector<int4> a, s;
  for (auto& x : an) a.push_back(x.second);
  for (auto& x : sy) s.push_back(x.second);
  it->n_an = (int)a.size();
  it->n_sy = (int)s.size();
  auto upload = [&](Buffer& buf, const std::vector<int4>& v) -> int {
    buf.bytes = sizeof(int4) * std::max<size_t>(v.size(), 1);
    if (cudaMalloc(&buf.p, buf.bytes) != cudaSuccess) {
      cudaGetLastError();
      buf.p = nullptr;
      return set_err(ctx, CLC_ENOMEM, "work-list allocation failed");
    }
    return cuda_check(ctx, cudaMemcpy(buf.p, v.data(), sizeof(int4) * v.size(), cudaMemcpyHostToDevice),
                      "work-list upload");
  };
  int rc = upload(it->an, a);
  if (rc) return rc;
  return upload(it->sy, s);
}

// persistent grid: per_sm CTAs on every SM, at most what stays resident
template <typename K>
static int grid_of(clc_ctx* ctx, K kern, int threads, int smem, long long items, int per_sm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  per_sm = std::max(1, std::min(per_sm, std::max(occ, 1)));
  const long long g = std::min<long long>(items, (long long)num_sms(ctx) * per_sm);
  return (int)std::max<long long>(g, 1);
}

int tc_run_stage(clc_ctx* ctx, const TcBatchDev& b, const TcItems& it, const TcLaunch& L, int stage) {
  switch (stage) {
    case 0: {
      cudaFuncSetAttribute(k_tc_ring_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, it.fft_an_smem);
      const int g = grid_of(ctx, k_tc_ring_analysis, 256, it.fft_an_smem, b.n_ring, L.fft_ctas);
      CLC_LAUNCH(ctx, "k_tc_ring_analysis", k_tc_ring_analysis, g, 256, it.fft_an_smem, b);
      return launch_check(ctx, "k_tc_ring_analysis");
    }
    case 1: {
      const int g = grid_of(ctx, k_tc_pack_analysis, 256, 0, b.n_pa, 8);
      CLC_LAUNCH(ctx, "k_tc_pack_analysis", k_tc_pack_analysis, g, 256, 0, b);
      return launch_check(ctx, "k_tc_pack_analysis");
    }
    case 2: {
      const int bB = stage_b_bytes(it.na_max);
      const int smem = 1024 + L.an_stages * (32768 + 2 * bB);
      cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      const int tcols = pow2_cols(2 * it.na_max);
      const int g = grid_of(ctx, k_tc_gemm<false>, 192, smem, it.n_an, std::min(L.an_ctas, 512 / tcols));
      CLC_LAUNCH(ctx, "k_tc_analysis", (k_tc_gemm<false>), g, 192, smem, b, (const int4*)it.an.p, it.n_an,
                 L.an_stages, bB, it.na_max, tcols, ctx->d_err);
      return launch_check(ctx, "k_tc_analysis");
    }
    case 3: {
      if (b.mode && b.n_low > 0) {
        const int g = (int)std::min<long long>((b.n_low + 127) / 128, (long long)num_sms(ctx) * 16);
        CLC_LAUNCH(ctx, "k_tc_low_orders", k_tc_low_orders, g, 128, 0, b);
        const int rc = launch_check(ctx, "k_tc_low_orders");
        if (rc) return rc;
      }
      cudaFuncSetAttribute(k_tc_pack_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, it.pack_s_smem);
      const int g = grid_of(ctx, k_tc_pack_synthesis, 256, it.pack_s_smem, b.n_ps, 4);
      CLC_LAUNCH(ctx, "k_tc_pack_synthesis", k_tc_pack_synthesis, g, 256, it.pack_s_smem, b);
      return launch_check(ctx, "k_tc_pack_synthesis");
    }
    case 4: {
      const int bB = stage_b_bytes(it.ns_max);
      const int smem = 1024 + L.sy_stages * (32768 + 2 * bB);
      cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      const int tcols = pow2_cols(4 * it.ns_max);
      const int g = grid_of(ctx, k_tc_gemm<true>, 192, smem, it.n_sy, std::min(L.sy_ctas, 512 / tcols));
      CLC_LAUNCH(ctx, "k_tc_synthesis", (k_tc_gemm<true>), g, 192, smem, b, (const int4*)it.sy.p, it.n_sy,
                 L.sy_stages, bB, it.ns_max, tcols, ctx->d_err);
      return launch_check(ctx, "k_tc_synthesis");
    }
    default: {
      cudaFuncSetAttribute(k_tc_ring_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, it.fft_sy_smem);
      const int g = grid_of(ctx, k_tc_ring_synthesis, kRingThreads, it.fft_sy_smem, b.n_ring, L.fft_ctas);
      CLC_LAUNCH(ctx, "k_tc_ring_synthesis", k_tc_ring_synthesis, g, kRingThreads, it.fft_sy_smem, b);
      return launch_check(ctx, "k_tc_ring_synthesis");
    }
  }
}

int tc_run(clc_ctx* ctx, const TcBatchDev& b, const TcItems& it, const TcLaunch& L) {
  for (int s = 0; s < 6; ++s) {
    const int rc = tc_run_stage(ctx, b, it, L, s);
    if (rc) return rc;
  }
  return CLC_OK;
}

}  // namespace clc
