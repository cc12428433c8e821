// Allocation-free SHT analysis: a variant of clc_sht_analysis for callers
// that cannot allocate device memory.
//
// clc_sht_analysis keeps its ring Fourier coefficients in context scratch and
// builds FFT plans and Legendre tables on first use; all of those are device
// allocations.  This variant instead transforms each ring with a direct DFT,
// runs the associated-Legendre recurrence on the fly, and keeps its only
// scratch - the ring Fourier coefficients - in a fixed file-scope device
// array.  It therefore never calls cudaMalloc / cudaFree, which matters to
// callers that run while device allocation is unavailable or forbidden: code
// that records work into a CUDA graph (allocation calls are not permitted
// during stream capture), code embedded in a framework whose caching
// allocator owns all device memory, or services that must not grow their
// footprint after start-up.
#include <atomic>
#include "common.cuh"

namespace clc {

constexpr int kNoAllocMaxNside = 128;
constexpr int kNoAllocMaxLmax = 256;
constexpr int kNoAllocRings = 4 * kNoAllocMaxNside - 1;   // 511
constexpr int kNoAllocM = kNoAllocMaxLmax + 1;            // 257

// F[m * kNoAllocRings + ring]: 511 x 257 complex doubles = 2.1 MB, held by every
// GPU that loads the library until the process exits.  Every call overwrites
// the entries it reads, so nothing has to start at zero; calls whose work
// overlaps on the GPU share this array and race.
static __device__ __align__(256) double2 g_noalloc_ring_fourier[kNoAllocRings * kNoAllocM];

// F_m(ring) = weight * sum_j map_j e^{-i m phi_j}, m = 0 .. lmax, one CTA per
// ring, one thread per m; the phase advances by a complex rotation per pixel.
__global__ void k_ring_dft_noalloc(const double* __restrict__ map, int nside, int lmax, double weight,
                                   double2* __restrict__ F) {
  const int i = blockIdx.x + 1;
  const Ring r = ring_geom(nside, i);
  const double* x = map + r.first;
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)r.npix, &sn, &cs);
    const double stx = cs, sty = sn;                       // e^{-i m 2 pi / n}
    sincospi(-(double)m * (r.phi0 / kPi), &sn, &cs);
    double wx = cs, wy = sn;                               // e^{-i m phi0}
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < r.npix; ++j) {
      ax = fma(x[j], wx, ax);
      ay = fma(x[j], wy, ay);
      const double t = wx * stx - wy * sty;
      wy = wx * sty + wy * stx;
      wx = t;
    }
    F[(size_t)m * kNoAllocRings + (i - 1)] = make_double2(ax * weight, ay * weight);
  }
}

__device__ __forceinline__ double times_pow2(double p, int e) {
  if (e >= -1022) return p * __longlong_as_double((long long)(e + 1023) << 52);
  if (e < -1600) return 0.0;
  return (p * __longlong_as_double((long long)(e + 600 + 1023) << 52)) * 0x1p-600;
}

// a_lm = sum_r lambda_lm(z_r) (F_m(r) + (-1)^{l+m} F_m(r')) over the northern
// rings r (mirror r'), with lambda_lm from the scaled three-term recurrence
// computed on the fly; one CTA per m, one thread per northern ring.
__global__ void k_legendre_analysis_noalloc(int nside, int lmax, const double2* __restrict__ F,
                                            double2* __restrict__ alm) {
  __shared__ double2 part[8][kNoAllocM];
  const int m = blockIdx.x;
  const int R = 2 * nside;
  const int r = threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2 ve = make_double2(0.0, 0.0), vo = make_double2(0.0, 0.0);
  double z = 0.0, p2 = 0.0, p1 = 0.0;
  int e = 0;
  const bool active = r < R;
  if (active) {
    const int i = r + 1;
    const Ring g = ring_geom(nside, i);
    z = g.z;
    const double2 fn = F[(size_t)m * kNoAllocRings + (i - 1)];
    double2 fs = make_double2(0.0, 0.0);
    if (i != 2 * nside) fs = F[(size_t)m * kNoAllocRings + (4 * nside - i - 1)];
    ve = make_double2(fn.x + fs.x, fn.y + fs.y);
    vo = make_double2(fn.x - fs.x, fn.y - fs.y);
    // log2 lambda_mm = log2 sqrt((2m+1)!! / (4 pi (2m)!!)) + m log2 sin(theta)
    double l2 = 0.5 * log2(1.0 / (4.0 * kPi));
    for (int k = 1; k <= m; ++k) l2 += 0.5 * log2((2.0 * k + 1.0) / (2.0 * k));
    l2 += (double)m * log2(g.s);
    e = (int)floor(l2);
    p2 = exp2(l2 - (double)e);
    if (m & 1) p2 = -p2;
  }
  for (int l = m; l <= lmax; ++l) {
    double lam = 0.0;
    if (active) {
      double p;
      if (l == m) {
        p = p2;
      } else if (l == m + 1) {
        p1 = sqrt(2.0 * m + 3.0) * z * p2;
        p = p1;
      } else {
        const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        const double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
        double p0 = a * (z * p1 - b * p2);
        if (fabs(p0) > 0x1p400) {
          p0 *= 0x1p-400;
          p1 *= 0x1p-400;
          e += 400;
        }
        p2 = p1;
        p1 = p0;
        p = p0;
      }
      lam = times_pow2(p, e);
    }
    const double2 v = ((l + m) & 1) ? vo : ve;
    double ax = lam * v.x, ay = lam * v.y;
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) part[warp][l - m] = make_double2(ax, ay);
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int w = 0; w < nw; ++w) {
      ax += part[w][l - m].x;
      ay += part[w][l - m].y;
    }
    alm[(long long)m * (2 * lmax + 1 - m) / 2 + l] = make_double2(ax, ay);
  }
}

}  // namespace clc

using namespace clc;

// Device address of the scratch array, looked up once per device (the first
// call on a device does it; make that first call before any stream capture).
static double2* noalloc_scratch(int device) {
  static std::atomic<double2*> addr[64];   // concurrent first calls store the same address
  if (device < 0 || device >= 64) return nullptr;
  double2* a = addr[device].load(std::memory_order_acquire);
  if (!a) {
    if (cudaGetSymbolAddress((void**)&a, g_noalloc_ring_fourier) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[device].store(a, std::memory_order_release);
  }
  return a;
}

extern "C" int clc_sht_analysis_noalloc(const double* map, int nside, int lmax, double* alm, void* cuda_stream) {
  if (!map || !alm) return CLC_EINVAL;
  if (nside < 1 || nside > kNoAllocMaxNside || (nside & (nside - 1))) return CLC_EINVAL;
  if (lmax < 0 || lmax > kNoAllocMaxLmax || lmax > 4 * nside) return CLC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CLC_ECUDA;
  double2* F = noalloc_scratch(dev);
  if (!F) return CLC_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double w = 4.0 * kPi / (12.0 * (double)nside * nside);
  // an error left by earlier work on this thread stays with its owner
  if (cudaPeekAtLastError() != cudaSuccess) return CLC_ECUDA;
  k_ring_dft_noalloc<<<4 * nside - 1, 128, 0, st>>>(map, nside, lmax, w, F);
  if (cudaGetLastError() != cudaSuccess) return CLC_ECUDA;
  k_legendre_analysis_noalloc<<<lmax + 1, 256, 0, st>>>(nside, lmax, F, (double2*)alm);
  return cudaGetLastError() == cudaSuccess ? CLC_OK : CLC_ECUDA;
}
