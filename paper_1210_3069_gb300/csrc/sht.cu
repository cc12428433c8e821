// SHT entry points and the pure-SHT Poisson solve (paper Sec. 3.2):
// analysis of kappa, psi_lm = -kappa_lm / (l (l + 1)) with the l = 0 term set
// to zero, and synthesis of psi and of its derivatives.  The theta derivative
// is synthesised through the coefficients b_lm of sin(theta) d/dtheta psi,
//   sin t d/dt lambda_lm = l eps_{l+1,m} lambda_{l+1,m} - (l+1) eps_lm lambda_{l-1,m},
//   eps_lm = sqrt((l^2 - m^2) / (4 l^2 - 1)),
// phi derivatives multiply the ring Fourier coefficients by i m, and the
// theta-theta component of the Hessian follows from the Laplacian:
// U_tt = kappa_bl - U_pp with kappa_bl = sum -l(l+1) psi_lm Y_lm.
#include <algorithm>

#include "fft.cuh"
#include "legendre.cuh"

namespace clc {

int poisson_sht_tc(clc_ctx* ctx, const double* const* kappa, int P, int nside, int lmax, double* const* psi,
                   const clc_derivs* out);

// rhs_0 = psi_lm, rhs_1 = b_lm (l <= lmax + 1), rhs_2 = -l(l+1) psi_lm, all
// packed with band limit lmax + 1.
__global__ void k_poisson_rhs(const double2* __restrict__ klm, int lmax, double2* __restrict__ rhs, long long Q,
                              int m0) {
  const int m = m0 + blockIdx.y;
  const int lt = lmax + 1;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lt) return;
  auto psi = [&](int ll) -> double2 {
    if (ll < m || ll > lmax || ll == 0) return make_double2(0.0, 0.0);
    const double2 k = klm[alm_idx(lmax, ll, m)];
    const double d = -1.0 / ((double)ll * (ll + 1.0));
    return make_double2(k.x * d, k.y * d);
  };
  auto eps = [&](int ll) -> double {
    if (ll <= m) return 0.0;
    return sqrt(((double)ll * ll - (double)m * m) / (4.0 * ll * ll - 1.0));
  };
  const double2 p = psi(l);
  const double2 pm = psi(l - 1), pp = psi(l + 1);
  const double c1 = (l - 1.0) * eps(l), c2 = (l + 2.0) * eps(l + 1);
  const long long i = alm_idx(lt, l, m);
  rhs[i] = p;
  rhs[Q + i] = make_double2(c1 * pm.x - c2 * pp.x, c1 * pm.y - c2 * pp.y);
  const double ll1 = -(double)l * (l + 1.0);
  rhs[2 * Q + i] = make_double2(ll1 * p.x, ll1 * p.y);
}

// copy alm (band limit lmax) into the lmax + 1 packing, zero at l = lmax + 1
__global__ void k_alm_expand(const double2* __restrict__ alm, int lmax, double2* __restrict__ rhs) {
  const int m = blockIdx.y;
  const int lt = lmax + 1;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lt) return;
  double2 v = make_double2(0.0, 0.0);
  if (l <= lmax) v = alm[alm_idx(lmax, l, m)];
  if (m == 0) v.y = 0.0;
  rhs[alm_idx(lt, l, m)] = v;
}

static int check_sht_args(clc_ctx* ctx, int nside, int lmax, const char* who) {
  if (!valid_nside(nside) || nside > 4096) return set_err(ctx, CLC_EINVAL, std::string(who) + ": bad nside");
  if (lmax < 0 || lmax > 4 * nside) return set_err(ctx, CLC_EINVAL, std::string(who) + ": lmax must be in [0, 4 nside]");
  return CLC_OK;
}

// Run fn on FP64 Legendre tables covering every order m <= lmax: the cached
// whole table when it fits in device memory, otherwise tables of consecutive
// order ranges built one after the other (each freed before the next; the
// recurrence cost is then paid per call).
template <typename Fn>
static int for_each_table(clc_ctx* ctx, int nside, int lmax, Fn fn) {
  int rc;
  const bool cached = ctx->leg_tables.count(std::make_tuple(nside, lmax, 0)) > 0;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const size_t whole = legendre_table_bytes(nside, lmax, 0, lmax + 1);
  const bool limited = ctx->table_budget > 0 && whole > ctx->table_budget;
  if (!limited && (cached || whole + (2ull << 30) <= freeb)) {
    auto T = get_legendre_table(ctx, nside, lmax, &rc);
    if (rc) return rc;
    return fn(*T);
  }
  size_t budget = std::min<size_t>(freeb > (8ull << 30) ? freeb - (8ull << 30) : (freeb / 2), 48ull << 30);
  if (ctx->table_budget > 0) budget = std::min(budget, ctx->table_budget);
  int m0 = 0;
  while (m0 <= lmax) {
    int m1 = m0 + 1;
    size_t b = legendre_table_bytes(nside, lmax, m0, m1);
    while (m1 <= lmax) {
      const size_t nb = legendre_table_bytes(nside, lmax, m1, m1 + 1);
      if (b + nb > budget) break;
      b += nb;
      ++m1;
    }
    LegendreTable T;
    if ((rc = build_legendre_table(ctx, nside, lmax, m0, m1, &T))) return rc;
    if ((rc = fn(T))) return rc;
    if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "table chunk"))) return rc;
    m0 = m1;
  }
  return CLC_OK;
}

// analysis into a device alm buffer (band limit lmax)
int sht_analysis(clc_ctx* ctx, const double* map, int nside, int lmax, double2* alm) {
  int rc;
  auto plan = get_fft_plan(ctx, nside, &rc);
  if (rc) return rc;
  const int ldf = 4 * nside - 1;
  double2* F = (double2*)scratch(ctx, 0, sizeof(double2) * (size_t)ldf * (lmax + 1));
  if (!F) return CLC_ENOMEM;
  const double w = 4.0 * kPi / (12.0 * (double)nside * nside);
  if ((rc = ring_analysis(ctx, *plan, map, lmax, w, F, ldf))) return rc;
  return for_each_table(ctx, nside, lmax, [&](const LegendreTable& T) { return legendre_analysis(ctx, T, F, ldf, alm); });
}

// synthesis of nq right-hand sides (lmax + 1 packing) and the ring FFTs
int sht_synthesis_rhs(clc_ctx* ctx, const double2* rhs, int nq, const int* lq, int nside, int lmax, int mode,
                      double* const out[6]) {
  int rc;
  auto plan = get_fft_plan(ctx, nside, &rc);
  if (rc) return rc;
  const int ld = 4 * nside - 1;
  double2* G = (double2*)scratch(ctx, 3, sizeof(double2) * (size_t)nq * ld * (lmax + 2));
  if (!G) return CLC_ENOMEM;
  if ((rc = for_each_table(ctx, nside, lmax,
                           [&](const LegendreTable& T) { return legendre_synthesis(ctx, T, rhs, nq, lq, G, ld); })))
    return rc;
  return ring_synthesis(ctx, *plan, G, ld, lmax, mode, out);
}

}  // namespace clc

using namespace clc;

extern "C" int clc_set_table_budget(clc_ctx* ctx, size_t bytes) {
  if (!ctx) return CLC_EINVAL;
  ctx->table_budget = bytes;
  return CLC_OK;
}

extern "C" int clc_sht_analysis(clc_ctx* ctx, const double* map, int nside, int lmax, double* alm) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_sht_args(ctx, nside, lmax, "clc_sht_analysis");
  if (rc) return rc;
  if (!map || !alm) return set_err(ctx, CLC_EINVAL, "clc_sht_analysis: null pointer");
  cudaSetDevice(ctx->device);
  return sht_analysis(ctx, map, nside, lmax, (double2*)alm);
}

extern "C" int clc_sht_synthesis(clc_ctx* ctx, const double* alm, int nside, int lmax, double* map) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_sht_args(ctx, nside, lmax, "clc_sht_synthesis");
  if (rc) return rc;
  if (!map || !alm) return set_err(ctx, CLC_EINVAL, "clc_sht_synthesis: null pointer");
  cudaSetDevice(ctx->device);
  const long long Q = alm_idx(lmax + 1, lmax + 1, lmax + 1) + 1;
  double2* rhs = (double2*)scratch(ctx, 2, sizeof(double2) * Q);
  if (!rhs) return CLC_ENOMEM;
  dim3 grid((lmax + 2 + 127) / 128, lmax + 1);
  CLC_LAUNCH(ctx, "k_alm_expand", k_alm_expand, grid, 128, 0, (const double2*)alm, lmax, rhs);
  if ((rc = launch_check(ctx, "k_alm_expand"))) return rc;
  const int lq[1] = {lmax};
  double* out[6] = {map, nullptr, nullptr, nullptr, nullptr, nullptr};
  return sht_synthesis_rhs(ctx, rhs, 1, lq, nside, lmax, 0, out);
}

extern "C" int clc_poisson_sht(clc_ctx* ctx, const double* kappa, int nside, int lmax, int precision, double* psi,
                               const clc_derivs* d) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_sht_args(ctx, nside, lmax, "clc_poisson_sht");
  if (rc) return rc;
  if (!kappa) return set_err(ctx, CLC_EINVAL, "clc_poisson_sht: null kappa");
  if (precision != CLC_FP64 && precision != CLC_MIXED)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_sht: precision must be CLC_FP64 or CLC_MIXED");
  cudaSetDevice(ctx->device);
  const bool derivs = d && (d->a_th || d->a_ph || d->u_tt || d->u_pp || d->u_tp);
  if (!psi && !derivs) return CLC_OK;
  if (precision == CLC_MIXED) return poisson_sht_tc(ctx, &kappa, 1, nside, lmax, &psi, derivs ? d : nullptr);
  double2* klm = (double2*)scratch(ctx, 1, sizeof(double2) * (alm_idx(lmax, lmax, lmax) + 1));
  if (!klm) return CLC_ENOMEM;
  const long long Q = alm_idx(lmax + 1, lmax + 1, lmax + 1) + 1;
  double2* rhs = (double2*)scratch(ctx, 2, sizeof(double2) * Q * 3);
  if (!rhs) return CLC_ENOMEM;
  auto plan = get_fft_plan(ctx, nside, &rc);
  if (rc) return rc;
  const int ld = 4 * nside - 1;
  double2* F = (double2*)scratch(ctx, 0, sizeof(double2) * (size_t)ld * (lmax + 1));
  if (!F) return CLC_ENOMEM;
  const int nq = derivs ? 3 : 1;
  double2* G = (double2*)scratch(ctx, 3, sizeof(double2) * (size_t)nq * ld * (lmax + 2));
  if (!G) return CLC_ENOMEM;
  const double w = 4.0 * kPi / (12.0 * (double)nside * nside);
  if ((rc = ring_analysis(ctx, *plan, kappa, lmax, w, F, ld))) return rc;
  const int lq1[1] = {lmax};
  const int lq3[3] = {lmax, lmax + 1, lmax};
  // per table (or order range): analysis, Poisson right-hand sides, synthesis
  rc = for_each_table(ctx, nside, lmax, [&](const LegendreTable& T) {
    int r = legendre_analysis(ctx, T, F, ld, klm);
    if (r) return r;
    dim3 grid((lmax + 2 + 127) / 128, T.m1 - T.m0);
    CLC_LAUNCH(ctx, "k_poisson_rhs", k_poisson_rhs, grid, 128, 0, klm, lmax, rhs, Q, T.m0);
    if ((r = launch_check(ctx, "k_poisson_rhs"))) return r;
    return legendre_synthesis(ctx, T, rhs, nq, derivs ? lq3 : lq1, G, ld);
  });
  if (rc) return rc;
  if (!derivs) {
    double* out[6] = {psi, nullptr, nullptr, nullptr, nullptr, nullptr};
    return ring_synthesis(ctx, *plan, G, ld, lmax, 0, out);
  }
  double* out[6] = {psi, d->a_th, d->a_ph, d->u_tt, d->u_pp, d->u_tp};
  return ring_synthesis(ctx, *plan, G, ld, lmax, 1, out);
}
