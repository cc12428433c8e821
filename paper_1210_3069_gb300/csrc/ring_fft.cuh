// Device side of the ring FFTs (paper Sec. 3.2: FFTs along iso-latitude
// rings), templated on the arithmetic type: FP64 for the FP64 SHT path, FP32
// for the mixed-precision path (whose error budget is set by the FP16 hi + lo
// Legendre contraction, far above FP32 FFT round-off).
//
// A block transforms one ring at a time with the whole ring in shared memory.
// A real ring of n = 4i (polar) or 4 Nside (equatorial) samples is handled as
// a complex sequence of N = n / 2 points: power-of-two N by an in-place
// radix-4 FFT (two radix-2 stages fused per pass, a leading radix-2 stage for
// odd log2 N), other N by Bluestein's chirp convolution with power-of-two
// FFTs of M >= 2N - 1 points whose chirp and filter spectrum the plan holds.
#pragma once

#include "fft.cuh"

namespace clc {

template <typename T>
__device__ __forceinline__ C2<T> cx(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return cx<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return cx<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ C2<T> operator*(C2<T> a, C2<T> b) {
  return cx<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ C2<T> operator*(C2<T> a, T s) { return cx<T>(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ C2<T> conj(C2<T> a) { return cx<T>(a.x, -a.y); }

__device__ __forceinline__ void sc_pi(double t, double* s, double* c) { sincospi(t, s, c); }
__device__ __forceinline__ void sc_pi(float t, float* s, float* c) { sincospif(t, s, c); }

// e^{i pi t}
template <typename T>
__device__ __forceinline__ C2<T> expi_pi(T t) {
  T s, c;
  sc_pi(t, &s, &c);
  return cx<T>(c, s);
}
// FP32: t reduced to [-1, 1], then the fast sincos intrinsic on pi t
// (absolute error about 2^-21 on [-pi, pi], far inside the mixed path's
// error budget)
template <>
__device__ __forceinline__ C2<float> expi_pi<float>(float t) {
  const float r = t - 2.f * rintf(0.5f * t);
  float s, c;
  __sincosf(3.14159265358979f * r, &s, &c);
  return cx<float>(c, s);
}

// e^{i pi a k / n} along k = k0, k0 + dk, ... (one call of next() per k, in
// that order).  FP64 steps by a complex rotation (error ~ steps x 1e-16);
// FP32 evaluates each factor directly.
template <typename T>
struct Rot;
template <>
struct Rot<double> {
  C2<double> cur, inc;
  __device__ __forceinline__ void init(int k0, int dk, int n, double a) {
    cur = expi_pi<double>(a * (double)k0 / (double)n);
    inc = expi_pi<double>(a * (double)dk / (double)n);
  }
  __device__ __forceinline__ C2<double> next() {
    const C2<double> r = cur;
    cur = cur * inc;
    return r;
  }
};
template <>
struct Rot<float> {
  int k, dk;
  float an;   // a / n
  __device__ __forceinline__ void init(int k0, int dk_, int n_, double a_) {
    k = k0;
    dk = dk_;
    an = (float)a_ / (float)n_;   // FP32: an FP64 division here would run on the slow FP64 pipe
  }
  __device__ __forceinline__ C2<float> next() {
    const C2<float> r = expi_pi<float>(an * (float)k);
    k += dk;
    return r;
  }
};

// a / b in the arithmetic type (no FP64 division on the FP32 path)
template <typename T>
__device__ __forceinline__ T ratio(int a, int b) { return (T)a / (T)b; }

// padded position of FFT point i in shared memory
template <typename T>
__device__ __forceinline__ int pidx(int i) { return i + (i >> fft_pad_shift<T>()); }

// FP32 -> FP64 by moving the bits (exact for normal floats; zero and
// subnormal floats give zero): keeps the output conversion off the FP64 pipe
__device__ __forceinline__ double to_out(double v) { return v; }
// FP64 map value in the arithmetic type (FP32: rounded on the integer pipe)
template <typename T>
__device__ __forceinline__ T to_in(double v) { return (T)v; }
template <>
__device__ __forceinline__ float to_in<float>(double v) { return d2f_rn(v); }
__device__ __forceinline__ double to_out(float v) { return f2d_exact(v); }

__device__ __forceinline__ int brev(int j, int logM) { return logM == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - logM)); }
__device__ __forceinline__ bool is_pow2(int v) { return (v & (v - 1)) == 0; }

// In-place forward FFT (sign -1) of s[0..2^logM) given in bit-reversed order;
// twiddle W_L^j = tw[j * mmax / L].
template <typename T>
__device__ void fft_pow2(C2<T>* s, int logM, const PlanDevT<T>& P) {
  const int M = 1 << logM;
  int lg = 1;
  if (logM & 1) {
    for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
      const C2<T> u = s[pidx<T>(2 * t)], v = s[pidx<T>(2 * t + 1)];
      s[pidx<T>(2 * t)] = u + v;
      s[pidx<T>(2 * t + 1)] = u - v;
    }
    __syncthreads();
    lg = 2;
  }
  for (; lg < logM; lg += 2) {
    // stages lg (half h) and lg + 1 (half 2h) on the quad i0 + {0, h, 2h, 3h}
    const int h = 1 << (lg - 1);
    const int sh1 = P.logmmax - lg, sh2 = P.logmmax - lg - 1;
    for (int t = threadIdx.x; t < M / 4; t += blockDim.x) {
      const int p = t & (h - 1);
      const int i0 = ((t >> (lg - 1)) << (lg + 1)) + p;
      const int j0 = pidx<T>(i0), j1 = pidx<T>(i0 + h), j2 = pidx<T>(i0 + 2 * h), j3 = pidx<T>(i0 + 3 * h);
      const C2<T> a0 = s[j0], a1 = s[j1], a2 = s[j2], a3 = s[j3];
      const C2<T> w1 = P.tw[p << sh1], w2 = P.tw[p << sh2];
      C2<T> v = a1 * w1;
      const C2<T> b0 = a0 + v, b1 = a0 - v;
      v = a3 * w1;
      const C2<T> b2 = a2 + v, b3 = a2 - v;
      v = b2 * w2;
      s[j0] = b0 + v;
      s[j2] = b0 - v;
      v = b3 * w2;
      v = cx<T>(v.y, -v.x);  // times W_{4h}^h = -i
      s[j1] = b1 + v;
      s[j3] = b1 - v;
    }
    __syncthreads();
  }
}

// Forward DFT of N points whose value at j is load(j); Z_k (natural order) is
// left in s[pidx(0..N)).  load is called by each thread for its j = threadIdx.x,
// threadIdx.x + blockDim.x, ... < N, in increasing order.
template <typename T, typename Load>
__device__ void dft_any(C2<T>* s, int N, int ring_class, const PlanDevT<T>& P, Load load) {
  if (is_pow2(N)) {
    const int logN = 31 - __clz(N);
    for (int j = threadIdx.x; j < N; j += blockDim.x) s[pidx<T>(brev(j, logN))] = load(j);
    __syncthreads();
    fft_pow2<T>(s, logN, P);
    return;
  }
  const int4 c = P.cls[ring_class];
  const int M = c.x, logM = c.y;
  const C2<T>* w = P.chirp + c.z;
  const C2<T>* B = P.filter + c.w;
  for (int j = threadIdx.x; j < M; j += blockDim.x)
    s[pidx<T>(brev(j, logM))] = (j < N) ? load(j) * conj(w[j]) : cx<T>(0, 0);
  __syncthreads();
  fft_pow2<T>(s, logM, P);
  for (int k = threadIdx.x; k < M; k += blockDim.x) s[pidx<T>(k)] = conj(s[pidx<T>(k)] * B[k]);
  __syncthreads();
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int kr = brev(k, logM);
    if (k < kr) {
      const C2<T> t = s[pidx<T>(k)];
      s[pidx<T>(k)] = s[pidx<T>(kr)];
      s[pidx<T>(kr)] = t;
    }
  }
  __syncthreads();
  fft_pow2<T>(s, logM, P);
  const T invM = (T)1 / (T)M;
  for (int k = threadIdx.x; k < N; k += blockDim.x) s[pidx<T>(k)] = (conj(s[pidx<T>(k)]) * invM) * conj(w[k]);
  __syncthreads();
}

// Geometry of ring i computed once per CTA (FP64 division and square root)
// and shared with all its threads, with 1 / sin(theta).
struct RingS {
  Ring r;
  double is;
};
__device__ __forceinline__ RingS ring_geom_cta(int nside, int i) {
  __shared__ RingS sh;
  __syncthreads();   // earlier readers of sh are done
  if (threadIdx.x == 0) {
    sh.r = ring_geom(nside, i);
    sh.is = 1.0 / sh.r.s;
  }
  __syncthreads();
  return sh;
}

__device__ __forceinline__ int ring_class_of(int nside, int i) {
  const int ip = i < 2 * nside ? i : 4 * nside - i;
  return ip < nside ? ip : 0;
}

// F[m * ldf + (i - 1)] = weight * sum_j map_j e^{-i m phi_j} over ring i, m <= lmax.
template <typename T>
__device__ void ring_analysis_ring(const double* __restrict__ map, int nside, int lmax, double weight,
                                   C2<T>* __restrict__ F, int ldf, const PlanDevT<T>& P, int i, C2<T>* s) {
  const Ring r = ring_geom_cta(nside, i).r;
  const int n = r.npix, N = n / 2;
  const double* x = map + r.first;
  dft_any<T>(s, N, ring_class_of(nside, i), P, [&](int j) { return cx<T>(to_in<T>(x[2 * j]), to_in<T>(x[2 * j + 1])); });
  const bool shifted = r.phi0 != 0.0;
  const T w = (T)weight, half = (T)0.5;
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    const int k = m % n;
    const bool cj = k > N;
    const int kk = cj ? n - k : k;
    const C2<T> Zk = s[pidx<T>(kk % N)];
    const C2<T> Zn = conj(s[pidx<T>((N - kk) % N)]);
    const C2<T> A = (Zk + Zn) * half;
    const C2<T> Bv = (Zk - Zn) * half;
    const C2<T> tB = conj(expi_pi<T>(ratio<T>(2 * kk, n))) * Bv;                   // e^{-2 pi i kk / n} Bv
    C2<T> X = cx<T>(A.x + tB.y, A.y - tB.x);                                      // A - i tB
    if (cj) X = conj(X);
    if (shifted) X = X * conj(expi_pi<T>(ratio<T>(m % (2 * n), n)));                // e^{-i m phi0}
    F[(size_t)m * ldf + (i - 1)] = X * w;
  }
  __syncthreads();
}

// Legendre sums G_q of one plane: element (m, ring) at m * sm + ring * sr,
// or, with quad set, in groups of four orders per ring:
// ((m / 4) * sm + ring * 4 + m % 4).  P01 (optional, FP32 path): FP64 sums
// of orders m = 0, 1 at P01[q * p01q + m * p01m + ring], used instead of G on
// the ncap rings next to each pole (nring rings in all).
template <typename T>
struct SynthArgsT {
  const C2<T>* G0;
  const C2<T>* G1;
  const C2<T>* G2;
  long long sm, sr;
  int quad;
  const C2<double>* P01;
  long long p01q, p01m;
  int ncap, nring;
  double* out[6];
};

// Fourier coefficient of output field f at order m on one ring from the
// Legendre sums g0 = psi, g1 = sin(t) d_t psi, g2 = kappa_bl (is = 1 / sin t,
// c = cos t).
template <typename S>
__device__ __forceinline__ C2<S> spec_combine(int mode, int f, int m, C2<S> g0, C2<S> g1, C2<S> g2, S is, S is2, S c) {
  if (mode == 0 || f == 0) return g0;
  const S dm = (S)m;
  switch (f) {
    case 1: return cx<S>(-g1.x * is, -g1.y * is);                               // alpha_t
    case 2: return cx<S>(dm * g0.y * is, -dm * g0.x * is);                       // alpha_p = -i m g0 / s
    case 3:                                                                      // u_tt = kappa_bl - u_pp
      return cx<S>(g2.x - (-dm * dm * g0.x + c * g1.x) * is2, g2.y - (-dm * dm * g0.y + c * g1.y) * is2);
    case 4: return cx<S>((-dm * dm * g0.x + c * g1.x) * is2, (-dm * dm * g0.y + c * g1.y) * is2);
    default: {                                                                   // u_tp = i m (g1 - c g0) / s^2
      const C2<S> d = cx<S>(g1.x - c * g0.x, g1.y - c * g0.y);
      return cx<S>(-dm * d.y * is2, dm * d.x * is2);
    }
  }
}

// Ring geometry factors in the arithmetic type and, for the FP64 orders of
// the FP32 path, in FP64.
template <typename T>
struct RingFac {
  T is, is2, c;
  double isd, is2d, cd;
};

template <typename T>
__device__ __forceinline__ C2<T> spec_of(const SynthArgsT<T>& a, int mode, int f, int m, int ring0, const RingFac<T>& g) {
  if (a.P01 && m <= 1 && (ring0 < a.ncap || ring0 >= a.nring - a.ncap)) {
    // the polar Hessian terms of m = 0, 1 cancel to O(sin^2 t): combine in FP64
    const C2<double>* P = a.P01 + (size_t)m * a.p01m + ring0;
    const C2<double> z = cx<double>(0.0, 0.0);
    const C2<double> h = spec_combine<double>(mode, f, m, P[0], mode ? P[a.p01q] : z, mode ? P[2 * a.p01q] : z, g.isd,
                                              g.is2d, g.cd);
    return cx<T>((T)h.x, (T)h.y);
  }
  const size_t idx = a.quad ? (size_t)(m >> 2) * a.sm + (size_t)ring0 * 4 + (m & 3)
                            : (size_t)m * a.sm + (size_t)ring0 * a.sr;
  const C2<T> g0 = a.G0[idx];
  if (mode == 0 || f == 0) return g0;
  const C2<T> g1 = a.G1[idx];
  const C2<T> g2 = f == 3 ? a.G2[idx] : cx<T>(0, 0);
  return spec_combine<T>(mode, f, m, g0, g1, g2, g.is, g.is2, g.c);
}

// Real ring values of every requested output field of ring i.  s: FFT
// buffer (fft_buf_len(plan mmax) points), Xs: N + 1 points.
template <typename T>
__device__ void ring_synthesis_ring(const SynthArgsT<T>& a, int nside, int lmax, int mode, const PlanDevT<T>& P,
                                    int i, C2<T>* s, C2<T>* Xs) {
  const RingS rs = ring_geom_cta(nside, i);
  const Ring& r = rs.r;
  const int n = r.npix, N = n / 2;
  const int ring0 = i - 1;
  const bool shifted = r.phi0 != 0.0;
  RingFac<T> gf;
  gf.isd = rs.is;
  gf.is2d = gf.isd * gf.isd;
  gf.cd = r.z;
  gf.is = (T)gf.isd;
  gf.is2 = gf.is * gf.is;
  gf.c = (T)r.z;
  const int nf = mode ? 6 : 1;
  for (int f = 0; f < nf; ++f) {
    double* out = a.out[f];
    if (!out) continue;
    // X_k = c_k [sum_{q>=0} (-1)^q g_{k+qn} + sum_{q>=1} (-1)^q conj(g_{qn-k})]
    // with the half-pixel shift c_k = e^{i pi k / n} (signs and c_k only on
    // shifted rings): the aliases m = k + qn differ from k by q n in phase.
    Rot<T> ck;
    if (shifted) ck.init(threadIdx.x, blockDim.x, n, 1.0);
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
      C2<T> X = cx<T>(0, 0);
      int q = 0;
      for (int m = k; m <= lmax; m += n, ++q) {
        C2<T> g = spec_of<T>(a, mode, f, m, ring0, gf);
        if (m == 0) g.y = (T)0;
        X = (shifted && (q & 1)) ? X - g : X + g;
      }
      q = 1;
      for (int m = (k == 0 ? n : n - k); m <= lmax; m += n, ++q) {
        const C2<T> g = conj(spec_of<T>(a, mode, f, m, ring0, gf));
        X = (shifted && (q & 1)) ? X - g : X + g;
      }
      if (shifted) X = X * ck.next();
      Xs[k] = X;
    }
    __syncthreads();
    // P_k = conj(X_k) + X_{N-k} + i e^{-2 pi i k / n} (conj(X_k) - X_{N-k});
    // the forward DFT of P packs x_{2j} + i x_{2j+1}
    Rot<T> tw;
    tw.init(threadIdx.x, blockDim.x, n, -2.0);
    dft_any<T>(s, N, ring_class_of(nside, i), P, [&](int k) {
      const C2<T> a1 = conj(Xs[k]);
      const C2<T> b1 = Xs[N - k];
      const C2<T> t = tw.next() * (a1 - b1);
      return cx<T>(a1.x + b1.x - t.y, a1.y + b1.y + t.x);
    });
    double* x = out + r.first;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const C2<T> v = s[pidx<T>(j)];
      x[2 * j] = to_out(v.x);
      x[2 * j + 1] = to_out(v.y);
    }
    __syncthreads();
  }
}

}  // namespace clc
