// Legendre transforms of the HEALPix SHT (paper Sec. 3.2).
#pragma once

#include "common.cuh"

namespace clc {

// lambda_lm(z_r) for the 2 nside northern rings (equator included), every
// m <= lmax and l = m .. lmax + 1, stored [m][l - m][r] (r contiguous).
struct LegendreTable {
  int nside = 0, lmax = 0, R = 0;
  int m0 = 0, m1 = 0;  // orders held: m0 <= m < m1 (offsets relative to m0)
  Buffer data;      // double
  Buffer offsets;   // int64[lmax + 1]: start of column m (in elements)
  std::vector<long long> h_offsets;
  size_t elems = 0;
};

// The whole table of (nside, lmax), cached in the context.
std::shared_ptr<LegendreTable> get_legendre_table(clc_ctx* ctx, int nside, int lmax, int* rc);
// A table of the orders m0 <= m < m1 only (caller-owned; for solves whose
// whole table does not fit in device memory).
int build_legendre_table(clc_ctx* ctx, int nside, int lmax, int m0, int m1, LegendreTable* T);
size_t legendre_table_bytes(int nside, int lmax, int m0, int m1);

// packed index of (l, m) for band limit lmax (m-major)
__host__ __device__ __forceinline__ long long alm_idx(int lmax, int l, int m) {
  return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// alm[idx(l, m)] = sum_r lambda_lm(r) V_m^{(l+m) % 2}(r) from ring Fourier
// coefficients F[m * ldf + ring] (weights already applied), for the table's
// orders and l <= ltop (lmax by default, at most lmax + 1), packed with band
// limit ltop.
int legendre_analysis(clc_ctx* ctx, const LegendreTable& T, const double2* F, int ldf, double2* alm, int ltop = -1);

// G_q[m][ring] = sum_l lambda_lm(ring) rhs_q[idx'(l, m)] for q < nq, where
// rhs_q is packed with band limit lmax + 1 (idx' = alm_idx(lmax + 1, l, m)) and
// lq[q] is the highest l used by rhs q.  G_q lives at G + q * ld * (lmax + 2).
int legendre_synthesis(clc_ctx* ctx, const LegendreTable& T, const double2* rhs, int nq, const int* lq,
                       double2* G, int ld);

}  // namespace clc
