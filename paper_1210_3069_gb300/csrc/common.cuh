// Shared definitions of the lens-plane library: context, error handling and
// HEALPix geometry on the device (Gorski et al. 2005; paper Sec. 3, 3.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/calclens.h"

namespace clc {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoOverPi = 0x1.45f306dc9c883p-1;  // double nearest 2/pi
constexpr double kTwoThirds = 0x1.5555555555555p-1;  // double nearest 2/3

// device-side error codes recorded in the context's error word
enum DevErr { kDevOk = 0, kDevBadIndex = 1, kDevTimeout = 2, kDevNonFinite = 3 };

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
  ~Buffer() { if (p) cudaFree(p); }
};

struct FftPlan;       // ring FFT plan of one Nside (fft.cu)
struct LegendreTable; // lambda_lm table of one (Nside, lmax) (legendre.cu)
struct TcTable;       // FP16 hi/lo lambda_lm table for the tensor cores (legendre_tc.cu)
struct TcBatch;       // buffers and launches of a mixed-precision SHT batch (sht_batch.cu)

}  // namespace clc

struct clc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int* d_err = nullptr;  // device error word
  // launch accounting and optional per-kernel CUDA-event timing
  long long launches = 0;
  // first launch error not yet reported (taken right after each launch, so a
  // later runtime call that returns it cannot lose it)
  cudaError_t launch_err = cudaSuccess;
  const char* launch_err_kernel = nullptr;
  bool prof = false;
  std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  std::map<int, std::shared_ptr<clc::FftPlan>> fft_plans;
  std::map<std::tuple<int, int, int>, std::shared_ptr<clc::LegendreTable>> leg_tables;
  std::map<std::pair<int, int>, std::shared_ptr<clc::TcTable>> tc_tables;
  size_t table_budget = 0;  // FP64 Legendre table limit in bytes (0: device memory decides)
  std::map<std::tuple<int, int, int, int>, std::shared_ptr<clc::TcBatch>> tc_batches;
  // growable scratch buffers, reused across calls on this context's stream
  clc::Buffer scratch[8];
};

namespace clc {

int set_err(clc_ctx* ctx, int code, const std::string& msg);
cudaEvent_t pool_event(clc_ctx* ctx);

// Counts every kernel launch of a context and, while profiling is enabled,
// brackets it with CUDA events on the context's stream.
struct LaunchScope {
  clc_ctx* ctx;
  const char* name;
  cudaEvent_t start = nullptr;
  LaunchScope(clc_ctx* c, const char* n) : ctx(c), name(n) {
    ++ctx->launches;
    if (ctx->prof) {
      start = pool_event(ctx);
      if (start) cudaEventRecord(start, ctx->stream);
    }
  }
  ~LaunchScope() {
    if (start) {
      cudaEvent_t stop = pool_event(ctx);
      if (stop) {
        cudaEventRecord(stop, ctx->stream);
        ctx->prof_ev[name].push_back({start, stop});
      }
    }
  }
};

inline void note_launch(clc_ctx* ctx, cudaError_t e, const char* name) {
  if (e != cudaSuccess && ctx->launch_err == cudaSuccess) {
    ctx->launch_err = e;
    ctx->launch_err_kernel = name;
  }
}

#define CLC_LAUNCH(ctx, name, kern, g, b, s, ...)                    \
  do {                                                               \
    ::clc::LaunchScope _clc_ls((ctx), (name));                       \
    kern<<<(g), (b), (s), (ctx)->stream>>>(__VA_ARGS__);             \
    ::clc::note_launch((ctx), cudaGetLastError(), (name));           \
  } while (0)
int cuda_check(clc_ctx* ctx, cudaError_t e, const char* what);
// Grow scratch buffer `slot` to at least `bytes`; returns nullptr on failure
// (the context's error is set).
void* scratch(clc_ctx* ctx, int slot, size_t bytes);
int launch_check(clc_ctx* ctx, const char* what);
bool valid_nside(int nside);
int num_sms(clc_ctx* ctx);

// ---------------------------------------------------------------------------
// HEALPix on the device.  ang2pix uses only correctly rounded, unfused FP64
// operations (__dadd_rn etc. are never contracted into FMAs), in exactly the
// order documented in the oracle, so indices match it bit for bit.

__device__ __forceinline__ double wrap_tt(double phi) {
  double tt = __dmul_rn(phi, kTwoOverPi);
  if (tt >= 4.0) tt = __dsub_rn(tt, 4.0);
  return tt;
}

__device__ __forceinline__ int64_t imod(int64_t a, int64_t b) {
  int64_t r = a % b;
  return r < 0 ? r + b : r;
}

__device__ __forceinline__ int64_t ang2pix_ring(int nside, double z, double phi) {
  const int64_t n = nside;
  const double nd = (double)nside;
  const double za = fabs(z);
  const double tt = wrap_tt(phi);
  if (za <= kTwoThirds) {
    const double t1 = __dmul_rn(nd, __dadd_rn(0.5, tt));
    const double t2 = __dmul_rn(nd, __dmul_rn(0.75, z));
    const int64_t jp = (int64_t)__dsub_rn(t1, t2);
    const int64_t jm = (int64_t)__dadd_rn(t1, t2);
    const int64_t ir = n + 1 + jp - jm;
    const int64_t kshift = 1 - (ir & 1);
    int64_t ip = (jp + jm - n + kshift + 1) >> 1;
    ip = imod(ip, 4 * n);
    return 2 * n * (n - 1) + (ir - 1) * 4 * n + ip;
  }
  const double tp = __dsub_rn(tt, trunc(tt));
  const double tmp = __dmul_rn(nd, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
  const int64_t jp = (int64_t)__dmul_rn(tp, tmp);
  const int64_t jm = (int64_t)__dmul_rn(__dsub_rn(1.0, tp), tmp);
  const int64_t ir = jp + jm + 1;
  int64_t ip = (int64_t)__dmul_rn(tt, (double)ir);
  ip = imod(ip, 4 * ir);
  if (z > 0) return 2 * ir * (ir - 1) + ip;
  return 12 * n * n - 2 * ir * (ir + 1) + ip;
}

__device__ __forceinline__ int64_t spread_bits(int64_t v) {
  uint64_t x = (uint64_t)v & 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return (int64_t)x;
}

__device__ __forceinline__ int64_t compress_bits(int64_t v) {
  uint64_t x = (uint64_t)v & 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x | (x >> 16)) & 0x00000000ffffffffull;
  return (int64_t)x;
}

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }

__device__ __forceinline__ int64_t ang2pix_nest(int nside, double z, double phi) {
  const int64_t n = nside;
  const int order = ilog2(nside);
  const double nd = (double)nside;
  const double za = fabs(z);
  const double tt = wrap_tt(phi);
  int64_t face, ix, iy;
  if (za <= kTwoThirds) {
    const double t1 = __dmul_rn(nd, __dadd_rn(0.5, tt));
    const double t2 = __dmul_rn(nd, __dmul_rn(0.75, z));
    int64_t jp = (int64_t)__dsub_rn(t1, t2);
    int64_t jm = (int64_t)__dadd_rn(t1, t2);
    if (jp >= 4 * n && jm >= 4 * n) { jp -= 4 * n; jm -= 4 * n; }
    const int64_t ifp = jp >> order, ifm = jm >> order;
    if (ifp == ifm) face = (ifp == 4) ? 4 : ifp + 4;
    else if (ifp < ifm) face = ifp;
    else face = ifm + 8;
    ix = jm & (n - 1);
    iy = n - (jp & (n - 1)) - 1;
  } else {
    int64_t ntt = (int64_t)trunc(tt);
    if (ntt > 3) ntt = 3;
    const double tp = __dsub_rn(tt, (double)ntt);
    const double tmp = __dmul_rn(nd, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
    int64_t jp = (int64_t)__dmul_rn(tp, tmp);
    int64_t jm = (int64_t)__dmul_rn(__dsub_rn(1.0, tp), tmp);
    if (jp > n - 1) jp = n - 1;
    if (jm > n - 1) jm = n - 1;
    if (z >= 0) { face = ntt; ix = n - jm - 1; iy = n - jp - 1; }
    else { face = ntt + 8; ix = jp; iy = jm; }
  }
  return face * n * n + spread_bits(ix) + (spread_bits(iy) << 1);
}

// RING index of a NEST pixel (base-face coordinates -> ring, position)
__device__ __forceinline__ int64_t nest2ring(int nside, int64_t pix) {
  const int64_t n = nside;
  const int order = ilog2(nside);
  const int64_t face = pix >> (2 * order);
  const int64_t ipf = pix & (n * n - 1);
  const int64_t ix = compress_bits(ipf), iy = compress_bits(ipf >> 1);
  // ring of the face's lowest corner (units of Nside) and longitude index of
  // the face centre (units of pi/4)
  const int jrll = (face < 4) ? 2 : (face < 8 ? 3 : 4);
  const int jpll = (face < 4) ? (int)(2 * face + 1) : (face < 8 ? (int)(2 * (face - 4)) : (int)(2 * (face - 8) + 1));
  const int64_t jr = jrll * n - ix - iy - 1;
  int64_t nr, nbefore, kshift;
  if (jr < n) { nr = jr; nbefore = 2 * nr * (nr - 1); kshift = 0; }
  else if (jr > 3 * n) { nr = 4 * n - jr; nbefore = 12 * n * n - 2 * nr * (nr + 1); kshift = 0; }
  else { nr = n; nbefore = 2 * n * (n - 1) + (jr - n) * 4 * n; kshift = (jr - n) & 1; }
  int64_t jp = (jpll * nr + ix - iy + 1 + kshift) / 2;
  if (jp > 4 * n) jp -= 4 * n;
  if (jp < 1) jp += 4 * n;
  return nbefore + jp - 1;
}

// NEST index of the RING pixel at position j (0-based) of ring i (1-based):
// base face and in-face coordinates by inverting the ring / position
// formulas of nest2ring, integer arithmetic only.  In the polar caps the face
// is j / (pixels per face in the ring); in the equatorial belt the face row
// (north, equatorial, south faces) follows from the ring, and the face is the
// one whose in-face coordinates (S +- D) / 2 lie inside [0, nside).
__device__ __forceinline__ int64_t ring_pos2nest(int nside, int i, int64_t j) {
  const int64_t n = nside;
  int64_t f = 0, ix = 0, iy = 0;
  if (i < nside) {                 // north cap, faces 0..3: ring i holds i pixels of each
    const int64_t nr = i;
    f = j / nr;
    const int64_t b = j - f * nr;
    ix = n - nr + b;
    iy = n - 1 - b;
  } else if (i > 3 * nside) {      // south cap, faces 8..11
    const int64_t nr = 4 * n - i;
    const int64_t q = j / nr;
    f = 8 + q;
    ix = j - q * nr;
    iy = nr - 1 - ix;
  } else {                         // equatorial belt
    const int kshift = (i - nside) & 1;
    const int64_t t = 2 * j + 1 - kshift;
    bool found = false;
    for (int row = 2; row <= 4 && !found; ++row) {
      const int64_t S = row * n - i - 1;   // ix + iy on this face row
      if (S < 0 || S > 2 * n - 2) continue;
      for (int q = 0; q < 4; ++q) {
        const int64_t jpll = row == 3 ? 2 * q : 2 * q + 1;
        int64_t D = t - jpll * n;         // ix - iy, up to a multiple of 8 nside
        if (D > 4 * n) D -= 8 * n;
        if (D <= -4 * n) D += 8 * n;
        if (((S + D) & 1) == 0 && D <= S && -D <= S && D <= 2 * n - 2 - S && -D <= 2 * n - 2 - S) {
          f = 4 * (row - 2) + q;
          ix = (S + D) / 2;
          iy = (S - D) / 2;
          found = true;
          break;
        }
      }
    }
  }
  return f * n * n + spread_bits(ix) + (spread_bits(iy) << 1);
}

// Geometry of ring i (1-based, 1 <= i <= 4 nside - 1)
struct Ring {
  double z, s;      // cos / sin theta of the ring
  int64_t first;    // RING index of its first pixel
  int npix;         // pixels in the ring
  double phi0;      // longitude of its first pixel
};

__device__ __host__ __forceinline__ Ring ring_geom(int nside, int i) {
  Ring r;
  const int64_t n = nside;
  const bool north = i < nside, south = i > 3 * nside;
  if (north || south) {
    const int64_t ip = north ? i : 4 * n - i;
    const double a = ((double)ip * (double)ip) / (3.0 * (double)n * (double)n);
    r.z = north ? 1.0 - a : a - 1.0;
    r.s = sqrt(a * (2.0 - a));
    r.npix = (int)(4 * ip);
    r.first = north ? 2 * ip * (ip - 1) : 12 * n * n - 2 * ip * (ip + 1);
    r.phi0 = kPi / (double)r.npix;
  } else {
    r.z = 4.0 / 3.0 - (2.0 * (double)i) / (3.0 * (double)n);
    r.s = sqrt((1.0 - r.z) * (1.0 + r.z));
    r.npix = (int)(4 * n);
    r.first = 2 * n * (n - 1) + ((int64_t)i - n) * 4 * n;
    r.phi0 = (((i - nside) & 1) == 0) ? kPi / (double)r.npix : 0.0;
  }
  return r;
}

// Ring (1-based) of a RING pixel index
__device__ __forceinline__ int pix2ring(int nside, int64_t p, int64_t* j) {
  const int64_t n = nside;
  const int64_t ncap = 2 * n * (n - 1), np = 12 * n * n;
  if (p < ncap) {
    int64_t i = (int64_t)((1.0 + sqrt(1.0 + 2.0 * (double)p)) * 0.5);
    while (2 * i * (i - 1) > p) --i;
    while (2 * (i + 1) * i <= p) ++i;
    *j = p - 2 * i * (i - 1);
    return (int)i;
  }
  if (p < np - ncap) {
    const int64_t q = p - ncap;
    *j = q % (4 * n);
    return (int)(q / (4 * n) + n);
  }
  const int64_t q = np - p;
  int64_t i = (int64_t)((1.0 + sqrt(2.0 * (double)q - 1.0)) * 0.5);
  while (i > 1 && 2 * i * (i - 1) >= q) --i;
  while (2 * i * (i + 1) < q) ++i;
  *j = p - (np - 2 * i * (i + 1));
  return (int)(4 * n - i);
}

// continuous ring coordinate of z (ring i at z_i gives i)
__device__ __forceinline__ double ring_coord(int nside, double z) {
  const double n = nside;
  if (z > 2.0 / 3.0) return n * sqrt(3.0 * (1.0 - z));
  if (z < -2.0 / 3.0) return 4.0 * n - n * sqrt(3.0 * (1.0 + z));
  return n * (2.0 - 1.5 * z);
}

// theta of ring i
__device__ __forceinline__ double ring_theta(int nside, int i) {
  const Ring r = ring_geom(nside, i);
  return atan2(r.s, r.z);
}

// Continuous ring coordinate of colatitude theta (cos z, sin s): ring centres
// sit at integers 1 .. 4 nside - 1; used to find the bracketing rings.
__device__ __forceinline__ int ring_above(int nside, double z, double s) {
  const double nd = (double)nside;
  double x;
  if (z > kTwoThirds) x = nd * sqrt(3.0 * (1.0 - z) ) ;
  else if (z < -kTwoThirds) x = 4.0 * nd - nd * sqrt(3.0 * (1.0 + z));
  else x = nd * (2.0 - 1.5 * z);
  (void)s;
  int i = (int)floor(x);
  if (i < 0) i = 0;
  if (i > 4 * nside - 1) i = 4 * nside - 1;
  return i;  // ring index with theta_i <= theta (0 = above the first ring)
}

// Two pixels of ring i bracketing phi and the weight of the second
__device__ __forceinline__ void ring_pair(int nside, int i, double phi, int64_t* p0, int64_t* p1, double* f) {
  const Ring r = ring_geom(nside, i);
  const double t = (phi - r.phi0) * (double)r.npix / (2.0 * kPi);
  const double j0 = floor(t);
  *f = t - j0;
  int64_t j = (int64_t)j0;
  j = imod(j, r.npix);
  *p0 = r.first + j;
  *p1 = r.first + (j + 1 == r.npix ? 0 : j + 1);
}

// HEALPix ring-bilinear interpolation weights at (theta, phi): up to 8 pixel
// indices / weights (linear in theta between bracketing rings, linear in
// phi on each ring; above the first / below the last ring the ring is
// blended with the mean of its four pixels at the pole).
struct Interp8 {
  int64_t p[8];
  double w[8];
};

__device__ __forceinline__ Interp8 interp_weights(int nside, double theta, double phi) {
  Interp8 o;
  const double z = cos(theta);
  int i1 = ring_above(nside, z, 0.0);
  const int nr = 4 * nside - 1;
  // ring_above is exact up to rounding; settle the bracket on ring colatitudes
  while (i1 >= 1 && ring_theta(nside, i1) > theta) --i1;
  while (i1 + 1 <= nr && ring_theta(nside, i1 + 1) <= theta) ++i1;
  for (int k = 0; k < 8; ++k) { o.p[k] = 0; o.w[k] = 0.0; }
  if (i1 == 0 || i1 == nr) {
    const int ir = (i1 == 0) ? 1 : nr;
    const double tr = ring_theta(nside, ir);
    const double w = (i1 == 0) ? theta / tr : (kPi - theta) / (kPi - tr);
    int64_t a0, a1;
    double fa;
    ring_pair(nside, ir, phi, &a0, &a1, &fa);
    o.p[0] = a0; o.w[0] = w * (1.0 - fa);
    o.p[1] = a1; o.w[1] = w * fa;
    const Ring r = ring_geom(nside, ir);
    for (int k = 0; k < 4; ++k) { o.p[4 + k] = r.first + k; o.w[4 + k] = (1.0 - w) * 0.25; }
    return o;
  }
  const double ta = ring_theta(nside, i1), tb = ring_theta(nside, i1 + 1);
  const double w = (theta - ta) / (tb - ta);
  int64_t a0, a1, b0, b1;
  double fa, fb;
  ring_pair(nside, i1, phi, &a0, &a1, &fa);
  ring_pair(nside, i1 + 1, phi, &b0, &b1, &fb);
  o.p[0] = a0; o.w[0] = (1.0 - w) * (1.0 - fa);
  o.p[1] = a1; o.w[1] = (1.0 - w) * fa;
  o.p[2] = b0; o.w[2] = w * (1.0 - fb);
  o.p[3] = b1; o.w[3] = w * fb;
  return o;
}

// Same interpolation with the ring colatitudes taken from a table
// (ring_th[i - 1] = theta of ring i).
__device__ __forceinline__ Interp8 interp_weights_tab(int nside, const double* __restrict__ ring_th, double theta,
                                                     double phi) {
  Interp8 o;
  const int nr = 4 * nside - 1;
  int i1 = ring_above(nside, cos(theta), 0.0);
  while (i1 >= 1 && ring_th[i1 - 1] > theta) --i1;
  while (i1 + 1 <= nr && ring_th[i1] <= theta) ++i1;
#pragma unroll
  for (int k = 0; k < 8; ++k) { o.p[k] = 0; o.w[k] = 0.0; }
  if (i1 == 0 || i1 == nr) {
    const int ir = (i1 == 0) ? 1 : nr;
    const double tr = ring_th[ir - 1];
    const double w = (i1 == 0) ? theta / tr : (kPi - theta) / (kPi - tr);
    int64_t a0, a1;
    double fa;
    ring_pair(nside, ir, phi, &a0, &a1, &fa);
    o.p[0] = a0; o.w[0] = w * (1.0 - fa);
    o.p[1] = a1; o.w[1] = w * fa;
    const Ring r = ring_geom(nside, ir);
#pragma unroll
    for (int k = 0; k < 4; ++k) { o.p[4 + k] = r.first + k; o.w[4 + k] = (1.0 - w) * 0.25; }
    return o;
  }
  const double ta = ring_th[i1 - 1], tb = ring_th[i1];
  const double w = (theta - ta) / (tb - ta);
  int64_t a0, a1, b0, b1;
  double fa, fb;
  ring_pair(nside, i1, phi, &a0, &a1, &fa);
  ring_pair(nside, i1 + 1, phi, &b0, &b1, &fb);
  o.p[0] = a0; o.w[0] = (1.0 - w) * (1.0 - fa);
  o.p[1] = a1; o.w[1] = (1.0 - w) * fa;
  o.p[2] = b0; o.w[2] = w * (1.0 - fb);
  o.p[3] = b1; o.w[3] = w * fb;
  return o;
}

__device__ __forceinline__ double interp_map_tab(const double* __restrict__ map, int nside,
                                                 const double* __restrict__ ring_th, double th, double ph) {
  const Interp8 w = interp_weights_tab(nside, ring_th, th, ph);
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (w.w[k] != 0.0) v += w.w[k] * map[w.p[k]];
  return v;
}

// FP32 <-> FP64 by moving bits on the integer pipe (the hardware conversions
// run on the FP64 pipe, 1/64 of the FP32 rate on this GPU).
// f2d_exact: exact for normal floats, infinities and NaN; zero and subnormal
// floats give (signless) zero.
__device__ __forceinline__ double f2d_exact(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((e == 0xFFu ? 0x7FFu : e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
// d2f_rn: round to nearest even, identical to (float)x; results that are
// zero, subnormal or out of the float range go through the hardware conversion.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FFu) - 1023 + 127;
  if (e <= 0 || e >= 255) return (float)x;
  const unsigned m = (unsigned)((b >> 29) & 0x7FFFFFu);
  const unsigned rem = (unsigned)(b & 0x1FFFFFFFu);
  unsigned f = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)e << 23) | m;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ++f;   // a mantissa carry steps the exponent
  return __uint_as_float(f);
}

__device__ __forceinline__ void record_error(int* d_err, int code) {
  atomicCAS(d_err, 0, code);
}

}  // namespace clc
