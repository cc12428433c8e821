// Ring FFTs of the HEALPix SHT (paper Sec. 3.2: FFTs along iso-latitude rings).
#pragma once

#include "common.cuh"

namespace clc {

struct FftPlan {
  int nside = 0;
  int mmax_fft = 0;        // largest complex FFT size used by any ring
  int smem_bytes = 0;      // dynamic shared memory of the ring kernels
  Buffer twiddle;          // double2[mmax_fft / 2]: e^{-2 pi i j / mmax_fft}
  Buffer cls;              // int4[nside]: per polar ring class k (1..nside-1): (M, logM, chirp off, filter off)
  Buffer chirp;            // double2: e^{i pi j^2 / N} per Bluestein class
  Buffer filter;           // double2: FFT_M of the Bluestein filter per class
};

std::shared_ptr<FftPlan> get_fft_plan(clc_ctx* ctx, int nside, int* rc);

// F[m * ldf + (i - 1)] = sum_j map_j e^{-i m phi_j} over ring i, m = 0 .. lmax,
// times `weight` (all 4 nside - 1 rings; ldf >= 4 nside - 1).
int ring_analysis(clc_ctx* ctx, const FftPlan& plan, const double* map, int lmax, double weight,
                  double2* F, int ldf);

// Synthesis of real ring values from per-ring Fourier coefficients G_q[m][ring]
// (q = 0 .. nq-1; ld = row length).  mode 0: out[0] = psi from G_0.
// mode 1 (derivatives; G_0 = psi, G_1 = sin(t) d_t psi, G_2 = kappa_bl):
// out[0..5] = psi, alpha_t, alpha_p, u_tt, u_pp, u_tp (NULL entries skipped).
int ring_synthesis(clc_ctx* ctx, const FftPlan& plan, const double2* G, int ld, int lmax, int mode,
                   double* const out[6]);

}  // namespace clc
