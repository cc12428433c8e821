// Mixed-precision batched SHT Poisson solve on the tcgen05 tensor cores
// (paper Sec. 3.2): shared declarations of the kernels (legendre_tc.cu) and
// of the batch plans that run them (sht_batch.cu).
#pragma once

#include <cuda_fp16.h>

#include "fft.cuh"

namespace clc {

constexpr int kTcMaxClasses = 8;   // plane classes (same nside, lmax) in one batch
constexpr int kTabExp = 10;        // table values are 2^kTabExp lambda_lm

// FP16 hi + lo lambda table of one (nside, lmax), grouped by (m, parity of
// l - m): group g = 2m + p holds rows l = m + p + 2k (l <= lmax + 1), padded
// with zero rows to a multiple of 64.  Storage is in 8 KB atoms of 64 rows x
// 64 rings, each row 128 bytes with the 16-byte chunk index XOR (row mod 8):
// atom (row block b, ring block j) at element (b * R / 64 + j) * 4096.  The
// same atom is a K-major tile for the analysis (rows = M, rings = K) and an
// MN-major tile for the synthesis (rows = K, rings = M).
struct TcTable {
  int nside = 0, lmax = 0, R = 0;
  std::vector<long long> h_off;   // [G] first row of group g (multiple of 64)
  std::vector<int> h_rows;        // [G] rows with l <= lmax + 1
  std::vector<int> h_pad;         // [G] rows padded to a multiple of 64
  Buffer off, rows, pad;          // device copies
  Buffer hi, lo;                  // __half atoms, total_rows + 128 rows
  long long total_rows = 0;
  size_t bytes() const { return hi.bytes + lo.bytes; }
};

std::shared_ptr<TcTable> get_tc_table(clc_ctx* ctx, int nside, int lmax, int* rc);

// One (nside, lmax) class of a batch: P planes sharing the table.
struct TcClass {
  const __half* th;
  const __half* tl;
  const long long* off;
  const int* rows;
  const int* pad;
  int nside, lmax, R, P, nq, Na, Ns;
  int plane0;                     // first plane of the class in the batch pointer tables
  double wq;                      // quadrature weight 4 pi / Npix
  PlanDevT<float> fft;
  int mmax;                       // FFT buffer points of the ring kernels
  float2* F;                      // [P][lmax + 1][ldf] ring coefficients
  size_t fstride;
  int ldf;
  __half *vh, *vl;                // analysis operand [G][R / 64][Na x 64 swizzled]
  int* vexp;                      // [G][Na] column scale exponents
  float2* alm;                    // [P][nalm] kappa_lm
  size_t astride;
  __half *sh, *sl;                // synthesis operand [soff[g] + t Ns 64][Ns x 64 swizzled]
  int* sexp;                      // [G][Ns]
  const long long* soff;          // [G]
  float2* G;                      // [P][nq][m / 4][ring][m % 4] per-ring Legendre sums
  size_t gstride, qstride;
  int ldm;                        // lmax + 1 rounded up to a multiple of 4
  double2* G01;                   // [P][nq][m = 0, 1][ring] FP64 Legendre sums of the two lowest orders
  const double* co01;             // [m = 0, 1][l = 0 .. lmax + 2][4] recurrence a_lm, b_lm, eps_lm, -1/(l(l+1))
  int ncap;                       // rings from each pole that use the FP64 sums
  long long ring0, pa0, ps0, low0;  // first flat item of the class: ring FFTs, packs, low-order sums
};

struct TcBatchDev {
  int ncls;
  TcClass cls[kTcMaxClasses];
  const double* const* kappa;     // device array [nplanes]
  double* const* out;             // device array [nplanes][6]: psi, a_th, a_ph, u_tt, u_pp, u_tp (NULL = skip)
  long long n_ring, n_pa, n_ps, n_low;   // flat item counts
  int mode;                       // 0: psi only, 1: psi and derivatives
};

// Launch shapes picked by the autotuner (sht_batch.cu).
struct TcLaunch {
  int an_stages = 2, an_ctas = 2;     // analysis pipeline depth, resident CTAs per SM
  int sy_stages = 2, sy_ctas = 2;     // synthesis
  int fft_ctas = 4;                   // ring FFT kernels, resident CTAs per SM
};

// Device-side work lists of a batch (built once per batch layout).
struct TcItems {
  Buffer an, sy;                      // int4 items: analysis (cls, grp, tile, 0), synthesis (cls, m, ring tile, 0)
  int n_an = 0, n_sy = 0;
  int na_max = 16, ns_max = 16;       // widest operands (TMEM columns, stage sizes)
  int fft_an_smem = 0, fft_sy_smem = 0, pack_s_smem = 0;
};

int tc_build_items(clc_ctx* ctx, const TcBatchDev& b, const std::vector<std::shared_ptr<TcTable>>& tabs,
                   TcItems* it);
// The six launches of one mixed-precision Poisson pass over every plane of the batch.
int tc_run(clc_ctx* ctx, const TcBatchDev& b, const TcItems& it, const TcLaunch& L);
// Individual stages (the autotuner times them separately); stage 0..5.
int tc_run_stage(clc_ctx* ctx, const TcBatchDev& b, const TcItems& it, const TcLaunch& L, int stage);

}  // namespace clc
