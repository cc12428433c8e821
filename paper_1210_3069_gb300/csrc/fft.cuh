// Ring FFTs of the HEALPix SHT (paper Sec. 3.2: FFTs along iso-latitude rings).
#pragma once

#include "common.cuh"

namespace clc {

// complex value of the FFT arithmetic type (layout of double2 / float2)
template <typename T>
struct alignas(2 * sizeof(T)) C2 {
  T x, y;
};

struct FftPlan {
  int nside = 0;
  int mmax_fft = 0;        // largest complex FFT size used by any ring
  Buffer twiddle;          // double2[mmax_fft / 2]: e^{-2 pi i j / mmax_fft}
  Buffer cls;              // int4[nside]: per polar ring class k (1..nside-1): (M, logM, chirp off, filter off)
  Buffer chirp;            // double2: e^{i pi j^2 / N} per Bluestein class
  Buffer filter;           // double2: FFT_M of the Bluestein filter per class
  Buffer twiddle32, chirp32, filter32;   // the same tables rounded to FP32
  size_t chirp_n = 0, filt_n = 0;
};

template <typename T>
struct PlanDevT {
  const C2<T>* tw;
  const int4* cls;
  const C2<T>* chirp;
  const C2<T>* filter;
  int logmmax;
};

std::shared_ptr<FftPlan> get_fft_plan(clc_ctx* ctx, int nside, int* rc);

// The shared-memory FFT buffer is padded by one point per 128 bytes
// (index i stored at i + (i >> shift)) to spread strided butterfly accesses
// over the banks.
template <typename T>
__host__ __device__ constexpr int fft_pad_shift() { return sizeof(T) == 4 ? 4 : 3; }
template <typename T>
__host__ __device__ constexpr int fft_buf_len(int m) { return m + (m >> fft_pad_shift<T>()) + 1; }
template <typename T>
PlanDevT<T> plan_dev(const FftPlan& p);
// dynamic shared memory of the ring kernels (analysis: FFT buffer; synthesis:
// FFT buffer + N + 1 spectrum points)
template <typename T>
int ring_analysis_smem(const FftPlan& p) { return fft_buf_len<T>(p.mmax_fft) * (int)sizeof(C2<T>); }
template <typename T>
int ring_synthesis_smem(const FftPlan& p) { return (fft_buf_len<T>(p.mmax_fft) + 2 * p.nside + 1) * (int)sizeof(C2<T>); }

// F[m * ldf + (i - 1)] = sum_j map_j e^{-i m phi_j} over ring i, m = 0 .. lmax,
// times `weight` (all 4 nside - 1 rings; ldf >= 4 nside - 1).
template <typename T>
int ring_analysis_t(clc_ctx* ctx, const FftPlan& plan, const double* map, int lmax, double weight, C2<T>* F,
                    int ldf);

// Synthesis of real ring values from per-ring Fourier coefficients G_q[m][ring]
// (q = 0 .. nq-1; ld = row length; G_q at G + q * ld * (lmax + 2)).
// mode 0: out[0] = psi from G_0.  mode 1 (derivatives; G_0 = psi,
// G_1 = sin(t) d_t psi, G_2 = kappa_bl): out[0..5] = psi, alpha_t, alpha_p,
// u_tt, u_pp, u_tp (NULL entries skipped).
template <typename T>
int ring_synthesis_t(clc_ctx* ctx, const FftPlan& plan, const C2<T>* G, int ld, int lmax, int mode,
                     double* const out[6]);

// FP64 forms
inline int ring_analysis(clc_ctx* ctx, const FftPlan& plan, const double* map, int lmax, double weight,
                         double2* F, int ldf) {
  return ring_analysis_t<double>(ctx, plan, map, lmax, weight, reinterpret_cast<C2<double>*>(F), ldf);
}
inline int ring_synthesis(clc_ctx* ctx, const FftPlan& plan, const double2* G, int ld, int lmax, int mode,
                          double* const out[6]) {
  return ring_synthesis_t<double>(ctx, plan, reinterpret_cast<const C2<double>*>(G), ld, lmax, mode, out);
}

}  // namespace clc
