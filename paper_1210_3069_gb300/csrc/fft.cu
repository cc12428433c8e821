// Ring FFT plans and single-map launches (paper Sec. 3.2: the SHT runs FFTs
// along iso-latitude rings, Press et al. 2007 Sec. 6.7).  The plan of one
// Nside holds the twiddles, the Bluestein chirps and filter spectra of the
// non-power-of-two polar rings (FP64, plus FP32 copies for the mixed path);
// the per-ring device code is in ring_fft.cuh.  One CTA per ring.
#include <algorithm>

#include "ring_fft.cuh"

namespace clc {

__global__ void k_twiddle(double2* tw, int mmax) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < mmax / 2; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)mmax, &sn, &cs);
    tw[j] = make_double2(cs, -sn);
  }
}

// One CTA per Bluestein ring class k: chirp w_j = e^{i pi j^2 / N}, N = 2k, and
// the spectrum of the circular filter b (b_j = w_j, b_{M-j} = w_j).
__global__ void k_bluestein_tables(int nside, PlanDevT<double> P, C2<double>* chirp, C2<double>* filter) {
  extern __shared__ C2<double> sb[];
  C2<double>* s = sb;
  const int k = blockIdx.x + 1;
  if (k >= nside) return;
  const int N = 2 * k;
  if (is_pow2(N)) return;
  const int4 c = P.cls[k];
  const int M = c.x, logM = c.y;
  C2<double>* w = chirp + c.z;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const long long t = ((long long)j * j) % (2ll * N);
    w[j] = expi_pi<double>((double)t / (double)N);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    C2<double> v = cx<double>(0.0, 0.0);
    if (j < N) v = w[j];
    else if (j > M - N) v = w[M - j];
    s[pidx<double>(brev(j, logM))] = v;
  }
  __syncthreads();
  fft_pow2<double>(s, logM, P);
  for (int j = threadIdx.x; j < M; j += blockDim.x) filter[c.w + j] = s[pidx<double>(j)];
}

__global__ void k_round_to_float(const double2* __restrict__ in, size_t n, float2* __restrict__ out) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    out[j] = make_float2((float)in[j].x, (float)in[j].y);
}

template <typename T>
__global__ void k_ring_analysis(const double* __restrict__ map, int nside, int lmax, double weight,
                                C2<T>* __restrict__ F, int ldf, PlanDevT<T> P) {
  extern __shared__ __align__(16) unsigned char smem_fft[];
  ring_analysis_ring<T>(map, nside, lmax, weight, F, ldf, P, blockIdx.x + 1, reinterpret_cast<C2<T>*>(smem_fft));
}

template <typename T>
__global__ void k_ring_synthesis(SynthArgsT<T> a, int nside, int lmax, int mode, int mmax_fft, PlanDevT<T> P) {
  extern __shared__ __align__(16) unsigned char smem_fft[];
  C2<T>* s = reinterpret_cast<C2<T>*>(smem_fft);
  ring_synthesis_ring<T>(a, nside, lmax, mode, P, blockIdx.x + 1, s, s + fft_buf_len<T>(mmax_fft));
}

template <>
PlanDevT<double> plan_dev<double>(const FftPlan& p) {
  PlanDevT<double> d;
  d.tw = (const C2<double>*)p.twiddle.p;
  d.cls = (const int4*)p.cls.p;
  d.chirp = (const C2<double>*)p.chirp.p;
  d.filter = (const C2<double>*)p.filter.p;
  d.logmmax = 0;
  while ((1 << d.logmmax) < p.mmax_fft) ++d.logmmax;
  return d;
}

template <>
PlanDevT<float> plan_dev<float>(const FftPlan& p) {
  PlanDevT<float> d;
  d.tw = (const C2<float>*)p.twiddle32.p;
  d.cls = (const int4*)p.cls.p;
  d.chirp = (const C2<float>*)p.chirp32.p;
  d.filter = (const C2<float>*)p.filter32.p;
  d.logmmax = 0;
  while ((1 << d.logmmax) < p.mmax_fft) ++d.logmmax;
  return d;
}

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

std::shared_ptr<FftPlan> get_fft_plan(clc_ctx* ctx, int nside, int* rc) {
  auto it = ctx->fft_plans.find(nside);
  if (it != ctx->fft_plans.end()) {
    *rc = CLC_OK;
    return it->second;
  }
  auto p = std::make_shared<FftPlan>();
  p->nside = nside;
  std::vector<int4> cls(std::max(nside, 1), make_int4(0, 0, 0, 0));
  int mmax = std::max(2 * nside, 1);
  size_t chirp_n = 0, filt_n = 0;
  for (int k = 1; k < nside; ++k) {
    const int N = 2 * k;
    if ((N & (N - 1)) == 0) continue;
    const int M = next_pow2(2 * N - 1);
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    cls[k] = make_int4(M, logM, (int)chirp_n, (int)filt_n);
    chirp_n += N;
    filt_n += M;
    mmax = std::max(mmax, M);
  }
  p->mmax_fft = mmax;
  p->chirp_n = chirp_n;
  p->filt_n = filt_n;
  auto alloc = [&](Buffer& b, size_t bytes) -> bool {
    b.bytes = std::max(bytes, (size_t)16);
    if (cudaMalloc(&b.p, b.bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return false;
    }
    return true;
  };
  if (!alloc(p->twiddle, sizeof(double2) * std::max(mmax / 2, 1)) || !alloc(p->cls, sizeof(int4) * cls.size()) ||
      !alloc(p->chirp, sizeof(double2) * chirp_n) || !alloc(p->filter, sizeof(double2) * filt_n) ||
      !alloc(p->twiddle32, sizeof(float2) * std::max(mmax / 2, 1)) || !alloc(p->chirp32, sizeof(float2) * chirp_n) ||
      !alloc(p->filter32, sizeof(float2) * filt_n)) {
    *rc = set_err(ctx, CLC_ENOMEM, "FFT plan allocation failed");
    return nullptr;
  }
  *rc = cuda_check(ctx, cudaMemcpyAsync(p->cls.p, cls.data(), sizeof(int4) * cls.size(), cudaMemcpyHostToDevice,
                                        ctx->stream), "plan upload");
  if (*rc) return nullptr;
  CLC_LAUNCH(ctx, "k_twiddle", k_twiddle, 64, 256, 0, (double2*)p->twiddle.p, mmax);
  PlanDevT<double> d = plan_dev<double>(*p);
  if (nside > 1 && chirp_n > 0) {
    const int smem = fft_buf_len<double>(mmax) * (int)sizeof(double2);
    cudaFuncSetAttribute(k_bluestein_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    CLC_LAUNCH(ctx, "k_bluestein_tables", k_bluestein_tables, nside - 1, 256, smem, nside, d, (C2<double>*)p->chirp.p,
               (C2<double>*)p->filter.p);
  }
  CLC_LAUNCH(ctx, "k_round_to_float", k_round_to_float, 64, 256, 0, (const double2*)p->twiddle.p,
             (size_t)std::max(mmax / 2, 1), (float2*)p->twiddle32.p);
  if (chirp_n > 0) {
    CLC_LAUNCH(ctx, "k_round_to_float", k_round_to_float, 256, 256, 0, (const double2*)p->chirp.p, chirp_n,
               (float2*)p->chirp32.p);
    CLC_LAUNCH(ctx, "k_round_to_float", k_round_to_float, 256, 256, 0, (const double2*)p->filter.p, filt_n,
               (float2*)p->filter32.p);
  }
  *rc = launch_check(ctx, "FFT plan build");
  if (*rc) return nullptr;
  ctx->fft_plans[nside] = p;
  return p;
}

template <typename T>
int ring_analysis_t(clc_ctx* ctx, const FftPlan& plan, const double* map, int lmax, double weight, C2<T>* F,
                    int ldf) {
  const int nside = plan.nside;
  const int smem = ring_analysis_smem<T>(plan);
  cudaFuncSetAttribute(k_ring_analysis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_ring_analysis", (k_ring_analysis<T>), 4 * nside - 1, 256, smem, map, nside, lmax, weight, F, ldf,
             plan_dev<T>(plan));
  return launch_check(ctx, "k_ring_analysis");
}

template <typename T>
int ring_synthesis_t(clc_ctx* ctx, const FftPlan& plan, const C2<T>* G, int ld, int lmax, int mode,
                     double* const out[6]) {
  const int nside = plan.nside;
  SynthArgsT<T> a;
  const size_t qstride = (size_t)ld * (lmax + 2);
  a.G0 = G;
  a.G1 = G + qstride;
  a.G2 = G + 2 * qstride;
  a.sm = ld;
  a.sr = 1;
  a.quad = 0;
  a.P01 = nullptr;
  a.p01q = a.p01m = 0;
  a.ncap = a.nring = 0;
  for (int f = 0; f < 6; ++f) a.out[f] = out[f];
  const int smem = ring_synthesis_smem<T>(plan);
  cudaFuncSetAttribute(k_ring_synthesis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_ring_synthesis", (k_ring_synthesis<T>), 4 * nside - 1, 256, smem, a, nside, lmax, mode,
             plan.mmax_fft, plan_dev<T>(plan));
  return launch_check(ctx, "k_ring_synthesis");
}

template int ring_analysis_t<double>(clc_ctx*, const FftPlan&, const double*, int, double, C2<double>*, int);
template int ring_analysis_t<float>(clc_ctx*, const FftPlan&, const double*, int, double, C2<float>*, int);
template int ring_synthesis_t<double>(clc_ctx*, const FftPlan&, const C2<double>*, int, int, int, double* const[6]);
template int ring_synthesis_t<float>(clc_ctx*, const FftPlan&, const C2<float>*, int, int, int, double* const[6]);

}  // namespace clc
