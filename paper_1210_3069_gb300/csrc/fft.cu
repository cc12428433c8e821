// Ring FFTs of the HEALPix SHT (paper Sec. 3.2: the SHT runs FFTs along
// iso-latitude rings, Press et al. 2007 Sec. 6.7).  One CTA per ring, the
// whole ring in shared memory.  A real ring of n = 4i (polar) or 4 Nside
// (equatorial) samples is transformed as a complex sequence of N = n / 2
// points: power-of-two N by an in-place radix-2 FFT, other N by Bluestein's
// chirp convolution with a power-of-two FFT of M >= 2N - 1 points whose chirp
// and filter spectrum are precomputed per ring length in the plan.
#include <algorithm>

#include "fft.cuh"

namespace clc {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 expi_pi(double t) {  // e^{i pi t}
  double sn, cs;
  sincospi(t, &sn, &cs);
  return make_double2(cs, sn);
}
__device__ __forceinline__ int brev(int j, int logM) { return logM == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - logM)); }
__device__ __forceinline__ bool is_pow2(int v) { return (v & (v - 1)) == 0; }

struct PlanDev {
  const double2* tw;
  const int4* cls;
  const double2* chirp;
  const double2* filter;
  int logmmax;
};

// In-place forward FFT (sign -1) of s[0..2^logM) given in bit-reversed order.
__device__ void fft_pow2(double2* s, int logM, const PlanDev& P) {
  const int M = 1 << logM;
  for (int lg = 1; lg <= logM; ++lg) {
    const int half = 1 << (lg - 1);
    const int sh = P.logmmax - lg;
    for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
      const int pos = t & (half - 1);
      const int i = ((t >> (lg - 1)) << lg) + pos;
      const int j = i + half;
      const double2 w = P.tw[pos << sh];
      const double2 v = cmul(s[j], w);
      const double2 u = s[i];
      s[i] = cadd(u, v);
      s[j] = csub(u, v);
    }
    __syncthreads();
  }
}

// Forward DFT of N points whose value at j is produced by load(j).
// Result Z_k (natural order) is left in s[0..N).
template <typename Load>
__device__ void dft_any(double2* s, int N, int ring_class, const PlanDev& P, Load load) {
  if (is_pow2(N)) {
    const int logN = 31 - __clz(N);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[brev(j, logN)] = load(j);
    __syncthreads();
    fft_pow2(s, logN, P);
    return;
  }
  const int4 c = P.cls[ring_class];
  const int M = c.x, logM = c.y;
  const double2* w = P.chirp + c.z;
  const double2* B = P.filter + c.w;
  for (int j = threadIdx.x; j < M; j += blockDim.x)
    s[brev(j, logM)] = (j < N) ? cmul(load(j), cconj(w[j])) : make_double2(0.0, 0.0);
  __syncthreads();
  fft_pow2(s, logM, P);
  for (int k = threadIdx.x; k < M; k += blockDim.x) s[k] = cconj(cmul(s[k], B[k]));
  __syncthreads();
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int kr = brev(k, logM);
    if (k < kr) {
      const double2 t = s[k];
      s[k] = s[kr];
      s[kr] = t;
    }
  }
  __syncthreads();
  fft_pow2(s, logM, P);
  const double invM = 1.0 / (double)M;
  for (int k = threadIdx.x; k < N; k += blockDim.x) s[k] = cmul(cscale(cconj(s[k]), invM), cconj(w[k]));
  __syncthreads();
}

__global__ void k_twiddle(double2* tw, int mmax) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < mmax / 2; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)mmax, &sn, &cs);
    tw[j] = make_double2(cs, -sn);
  }
}

// One CTA per Bluestein ring class k: chirp w_j = e^{i pi j^2 / N}, N = 2k, and
// the spectrum of the circular filter b (b_j = w_j, b_{M-j} = w_j).
__global__ void k_bluestein_tables(int nside, PlanDev P, double2* chirp, double2* filter) {
  extern __shared__ double2 s[];
  const int k = blockIdx.x + 1;
  if (k >= nside) return;
  const int N = 2 * k;
  if (is_pow2(N)) return;
  const int4 c = P.cls[k];
  const int M = c.x, logM = c.y;
  double2* w = chirp + c.z;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const long long t = ((long long)j * j) % (2ll * N);
    w[j] = expi_pi((double)t / (double)N);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (j < N) v = w[j];
    else if (j > M - N) v = w[M - j];
    s[brev(j, logM)] = v;
  }
  __syncthreads();
  fft_pow2(s, logM, P);
  for (int j = threadIdx.x; j < M; j += blockDim.x) filter[c.w + j] = s[j];
}

__device__ __forceinline__ int ring_class_of(int nside, int i) {
  const int ip = i < 2 * nside ? i : 4 * nside - i;
  return ip < nside ? ip : 0;
}

__global__ void k_ring_analysis(const double* __restrict__ map, int nside, int lmax, double weight,
                                double2* __restrict__ F, int ldf, PlanDev P) {
  extern __shared__ double2 s[];
  const int i = blockIdx.x + 1;
  const Ring r = ring_geom(nside, i);
  const int n = r.npix, N = n / 2;
  const double* x = map + r.first;
  dft_any(s, N, ring_class_of(nside, i), P, [&](int j) { return make_double2(x[2 * j], x[2 * j + 1]); });
  const bool shifted = r.phi0 != 0.0;
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    const int k = m % n;
    const bool cj = k > N;
    const int kk = cj ? n - k : k;
    const double2 Zk = s[kk % N];
    const double2 Zn = cconj(s[(N - kk) % N]);
    const double2 A = cscale(cadd(Zk, Zn), 0.5);
    const double2 Bv = cscale(csub(Zk, Zn), 0.5);
    const double2 tw = cconj(expi_pi(2.0 * (double)kk / (double)n));   // e^{-2 pi i kk / n}
    const double2 tB = cmul(tw, Bv);
    double2 X = make_double2(A.x + tB.y, A.y - tB.x);                  // A - i tw Bv
    if (cj) X = cconj(X);
    if (shifted) X = cmul(X, cconj(expi_pi((double)(m % (2 * n)) / (double)n)));  // e^{-i m phi0}
    F[(size_t)m * ldf + (i - 1)] = cscale(X, weight);
  }
}

struct SynthArgs {
  const double2* G0;
  const double2* G1;
  const double2* G2;
  int ld;
  double* out[6];
};

__device__ __forceinline__ double2 spec_of(const SynthArgs& a, int mode, int f, int m, int ring0, double s,
                                           double c) {
  const size_t idx = (size_t)m * a.ld + ring0;
  const double2 g0 = a.G0[idx];
  if (mode == 0 || f == 0) return g0;
  const double2 g1 = a.G1[idx];
  const double dm = (double)m;
  const double is = 1.0 / s, is2 = is * is;
  switch (f) {
    case 1: return make_double2(-g1.x * is, -g1.y * is);                        // alpha_t
    case 2: return make_double2(dm * g0.y * is, -dm * g0.x * is);                // alpha_p = -i m g0 / s
    case 3: {                                                                    // u_tt
      const double2 g2 = a.G2[idx];
      const double2 upp = make_double2((-dm * dm * g0.x + c * g1.x) * is2, (-dm * dm * g0.y + c * g1.y) * is2);
      return make_double2(g2.x - upp.x, g2.y - upp.y);
    }
    case 4: return make_double2((-dm * dm * g0.x + c * g1.x) * is2, (-dm * dm * g0.y + c * g1.y) * is2);
    default: {                                                                   // u_tp = i m (g1 - c g0) / s^2
      const double2 d = make_double2(g1.x - c * g0.x, g1.y - c * g0.y);
      return make_double2(-dm * d.y * is2, dm * d.x * is2);
    }
  }
}

__global__ void k_ring_synthesis(SynthArgs a, int nside, int lmax, int mode, int mmax_fft, PlanDev P) {
  extern __shared__ double2 sm[];
  double2* s = sm;
  double2* Xs = sm + mmax_fft;
  const int i = blockIdx.x + 1;
  const Ring r = ring_geom(nside, i);
  const int n = r.npix, N = n / 2;
  const int ring0 = i - 1;
  const bool shifted = r.phi0 != 0.0;
  const int nf = mode ? 6 : 1;
  for (int f = 0; f < nf; ++f) {
    double* out = a.out[f];
    if (!out) continue;
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
      double2 X = make_double2(0.0, 0.0);
      for (int m = k; m <= lmax; m += n) {
        double2 g = spec_of(a, mode, f, m, ring0, r.s, r.z);
        if (shifted) g = cmul(g, expi_pi((double)(m % (2 * n)) / (double)n));
        if (m == 0) g.y = 0.0;
        X = cadd(X, g);
      }
      for (int m = (k == 0 ? n : n - k); m <= lmax; m += n) {
        double2 g = spec_of(a, mode, f, m, ring0, r.s, r.z);
        if (shifted) g = cmul(g, expi_pi((double)(m % (2 * n)) / (double)n));
        X = cadd(X, cconj(g));
      }
      Xs[k] = X;
    }
    __syncthreads();
    // P_k = conj(X_k) + X_{N-k} + i e^{-2 pi i k / n} (conj(X_k) - X_{N-k});
    // the forward DFT of P packs x_{2j} + i x_{2j+1}
    dft_any(s, N, ring_class_of(nside, i), P, [&](int k) {
      const double2 a1 = cconj(Xs[k]);
      const double2 b1 = Xs[N - k];
      const double2 d = csub(a1, b1);
      const double2 tw = cconj(expi_pi(2.0 * (double)k / (double)n));
      const double2 t = cmul(tw, d);
      return make_double2(a1.x + b1.x - t.y, a1.y + b1.y + t.x);
    });
    double* x = out + r.first;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      x[2 * j] = s[j].x;
      x[2 * j + 1] = s[j].y;
    }
    __syncthreads();
  }
}

static PlanDev plan_dev(const FftPlan& p) {
  PlanDev d;
  d.tw = (const double2*)p.twiddle.p;
  d.cls = (const int4*)p.cls.p;
  d.chirp = (const double2*)p.chirp.p;
  d.filter = (const double2*)p.filter.p;
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
  const int synth_smem = (mmax + 2 * nside + 1) * (int)sizeof(double2);
  p->smem_bytes = synth_smem;
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
      !alloc(p->chirp, sizeof(double2) * chirp_n) || !alloc(p->filter, sizeof(double2) * filt_n)) {
    *rc = set_err(ctx, CLC_ENOMEM, "FFT plan allocation failed");
    return nullptr;
  }
  *rc = cuda_check(ctx, cudaMemcpyAsync(p->cls.p, cls.data(), sizeof(int4) * cls.size(), cudaMemcpyHostToDevice,
                                        ctx->stream), "plan upload");
  if (*rc) return nullptr;
  CLC_LAUNCH(ctx, "k_twiddle", k_twiddle, 64, 256, 0, (double2*)p->twiddle.p, mmax);
  PlanDev d = plan_dev(*p);
  if (nside > 1 && chirp_n > 0) {
    const int smem = mmax * (int)sizeof(double2);
    cudaFuncSetAttribute(k_bluestein_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    CLC_LAUNCH(ctx, "k_bluestein_tables", k_bluestein_tables, nside - 1, 256, smem, nside, d, (double2*)p->chirp.p, (double2*)p->filter.p);
  }
  *rc = launch_check(ctx, "FFT plan build");
  if (*rc) return nullptr;
  ctx->fft_plans[nside] = p;
  return p;
}

int ring_analysis(clc_ctx* ctx, const FftPlan& plan, const double* map, int lmax, double weight, double2* F,
                  int ldf) {
  const int nside = plan.nside;
  const int smem = plan.mmax_fft * (int)sizeof(double2);
  cudaFuncSetAttribute(k_ring_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_ring_analysis", k_ring_analysis, 4 * nside - 1, 256, smem, map, nside, lmax, weight, F, ldf, plan_dev(plan));
  return launch_check(ctx, "k_ring_analysis");
}

int ring_synthesis(clc_ctx* ctx, const FftPlan& plan, const double2* G, int ld, int lmax, int mode,
                   double* const out[6]) {
  const int nside = plan.nside;
  SynthArgs a;
  const size_t qstride = (size_t)ld * (lmax + 2);
  a.G0 = G;
  a.G1 = G + qstride;
  a.G2 = G + 2 * qstride;
  a.ld = ld;
  for (int f = 0; f < 6; ++f) a.out[f] = out[f];
  const int smem = plan.smem_bytes;
  cudaFuncSetAttribute(k_ring_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  CLC_LAUNCH(ctx, "k_ring_synthesis", k_ring_synthesis, 4 * nside - 1, 256, smem, a, nside, lmax, mode, plan.mmax_fft, plan_dev(plan));
  return launch_check(ctx, "k_ring_synthesis");
}

}  // namespace clc
