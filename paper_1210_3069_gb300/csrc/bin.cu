// Step 1 of the lens-plane path: particle deposit on HEALPix pixels and the
// plane source kappa^(m) (paper Sec. 3.2 source construction, Eq. lenspoisson;
// pixel indexing Sec. 3.1 / Gorski et al. 2005).
#include "common.cuh"

namespace clc {

// One thread per particle (grid-stride): 16 B read, one L2 atomic increment.
__global__ void k_bin(const double* __restrict__ z, const double* __restrict__ phi, int64_t n,
                      int nside, int nest, uint32_t* __restrict__ counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double zi = z[i], pi = phi[i];
    const int64_t p = nest ? ang2pix_nest(nside, zi, pi) : ang2pix_ring(nside, zi, pi);
    atomicAdd(counts + p, 1u);
  }
}

// kappa = scale * (counts / nbar - 1), each operation rounded separately
// kappa of a pixel with c particles: scale (c / nbar - 1), each operation
// correctly rounded
__device__ __forceinline__ double kappa_of(uint32_t c, double nbar, double scale) {
  return __dmul_rn(scale, __dsub_rn(__ddiv_rn((double)c, nbar), 1.0));
}

// Counts are small integers, so kappa takes few distinct values: a table of
// the first kKappaTable (the same correctly rounded operations, once per
// count) replaces the FP64 division per pixel, which would make this pass
// FP64-bound; larger counts divide.
constexpr int kKappaTable = 4096;

__global__ void k_kappa_table(double nbar, double scale, double* __restrict__ tab) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < kKappaTable) tab[c] = kappa_of((uint32_t)c, nbar, scale);
}

__global__ void k_counts_to_kappa(const uint32_t* __restrict__ counts, int64_t npix, double nbar,
                                  double scale, const double* __restrict__ tab, double* __restrict__ kappa) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) {
    const uint32_t c = counts[i];
    kappa[i] = c < (uint32_t)kKappaTable ? tab[c] : kappa_of(c, nbar, scale);
  }
}

// Partial-sky source (Sec. 3.4): particle count and pixel count of the
// covered region (exact integer sums), then nbar = their ratio and
// kappa = scale (counts / nbar - 1) on covered pixels, 0 (mean density)
// elsewhere.
__global__ void k_masked_sums(const uint32_t* __restrict__ counts, const uint8_t* __restrict__ covered, int64_t npix,
                              unsigned long long* __restrict__ sums) {
  unsigned long long c = 0, m = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
    if (covered[i]) {
      c += counts[i];
      ++m;
    }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  if ((threadIdx.x & 31) == 0 && (c || m)) {
    atomicAdd(sums, c);
    atomicAdd(sums + 1, m);
  }
}

__global__ void k_counts_to_kappa_masked(const uint32_t* __restrict__ counts, const uint8_t* __restrict__ covered,
                                         int64_t npix, const unsigned long long* __restrict__ sums, double scale,
                                         double* __restrict__ kappa) {
  const double nbar = __ddiv_rn((double)sums[0], (double)sums[1]);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
    kappa[i] = covered[i] ? __dmul_rn(scale, __dsub_rn(__ddiv_rn((double)counts[i], nbar), 1.0)) : 0.0;
}

// Coarse pixel P (RING) = mean of its NEST children at nside_fine.  The coarse
// pixel's NEST index comes from its centre (pix2ang followed by ang2pix_nest,
// which returns the pixel itself: centres lie far from pixel edges).
__global__ void k_degrade(const double* __restrict__ fine, int nf, double* __restrict__ coarse, int ns,
                          int shift) {
  const int64_t npc = 12ll * ns * ns;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int nchild = 1 << shift;
  const double inv = 1.0 / (double)nchild;
  for (int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; P < npc; P += stride) {
    int64_t j;
    const int i = pix2ring(ns, P, &j);
    const Ring r = ring_geom(ns, i);
    const double phi = r.phi0 + (2.0 * kPi) * (double)j / (double)r.npix;
    const int64_t pn = ang2pix_nest(ns, r.z, phi);
    double acc = 0.0;
    for (int c = 0; c < nchild; ++c) acc += fine[nest2ring(nf, (pn << shift) + c)];
    coarse[P] = acc * inv;
  }
}

// ---------------------------------------------------------------------------
// Adaptive Epanechnikov smoothing (Sec. 3.2): a particle's unit mass goes to
// the RING pixels whose centres lie within angular distance sigma, in
// proportion to 1 - (theta / sigma)^2 (the kernel's normalisation cancels),
// the weights divided by their sum so that the mass is conserved exactly;
// with no centre within sigma the mass goes to the particle's own pixel.
// One thread per particle: the rings that can reach the kernel, and on each
// the pixels within the longitude span that can, are visited; the distance
// test itself is exact (chord^2 < 4 sin^2(sigma / 2)), so the spans only have
// to be wide enough.

constexpr int kSmoothCache = 48;   // pixels of the first pass kept for the deposit

// theta^2 from the chord c^2 = |a - b|^2 of two unit vectors, 4 asin^2(c / 2):
// the Taylor series of asin^2 through the c^12 term for c^2 <= 1/400 (first
// omitted term below 1e-17 relative), else directly
__device__ __forceinline__ double theta2_of_chord2(double c2) {
  if (c2 <= 0.0025)
    return c2 * (1.0 + c2 * ((1.0 / 12.0) + c2 * ((1.0 / 90.0) + c2 * ((1.0 / 560.0) + c2 * ((1.0 / 3150.0) +
                                                                                           c2 * (1.0 / 16632.0))))));
  const double t = 2.0 * asin(0.5 * sqrt(c2));
  return t * t;
}

// Calls f(pixel, weight) for every RING pixel within the kernel of the
// particle at unit vector (xp, yp, zp) (sin of colatitude sp, longitude pp).
template <typename F>
__device__ __forceinline__ void kernel_pixels(int nside, double xp, double yp, double zp, double sp, double pp,
                                              double sg, double c2max, double inv_s2, F f) {
  const double thp = atan2(sp, zp);
  const double zhi = cos(fmax(0.0, thp - sg)), zlo = cos(fmin(kPi, thp + sg));
  const int i0 = max(1, (int)floor(ring_coord(nside, zhi)) - 1);
  const int i1 = min(4 * nside - 1, (int)ceil(ring_coord(nside, zlo)) + 1);
  for (int i = i0; i <= i1; ++i) {
    const Ring r = ring_geom(nside, i);
    const int np = r.npix;
    const int shift = r.phi0 != 0.0 ? 1 : 0;
    int jl = 0, jh = np - 1;
    const double den = 2.0 * sp * r.s;
    if (den > 1e-300) {
      // cos(dphi) > C on the pixels within the kernel
      const double C = (2.0 - c2max - 2.0 * zp * r.z) / den;
      if (C >= 1.0) continue;
      if (C > -1.0) {
        const double span = acos(C), dphi = 2.0 * kPi / (double)np;
        const double base = (pp - r.phi0) / dphi;
        jl = (int)floor(base - span / dphi) - 1;
        jh = (int)ceil(base + span / dphi) + 1;
        if (jh - jl + 1 >= np) {
          jl = 0;
          jh = np - 1;
        }
      }
    }
    // pixel longitudes pi (2 j + shift) / np by a rotation from the first
    double cs, sn, cd, sd;
    sincospi((double)(2 * jl + shift) / (double)np, &sn, &cs);
    sincospi(2.0 / (double)np, &sd, &cd);
    for (int j = jl; j <= jh; ++j) {
      const double dx = xp - r.s * cs, dy = yp - r.s * sn, dz = zp - r.z;
      const double c2 = dx * dx + dy * dy + dz * dz;
      if (c2 < c2max) {
        const double w = 1.0 - theta2_of_chord2(c2) * inv_s2;
        if (w > 0.0) f(r.first + (int64_t)(((j % np) + np) % np), w);
      }
      const double c0 = cs;
      cs = c0 * cd - sn * sd;
      sn = sn * cd + c0 * sd;
    }
  }
}

__global__ void k_smooth_particles(const double* __restrict__ z, const double* __restrict__ phi,
                                   const double* __restrict__ sig_each, int64_t n, int nside, double sigma,
                                   double* __restrict__ map) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double zp = z[i], pp = phi[i];
    const double sg = sig_each ? sig_each[i] : sigma;
    const double sp = sqrt((1.0 - zp) * (1.0 + zp));
    double sphi, cphi;
    sincos(pp, &sphi, &cphi);
    const double xp = sp * cphi, yp = sp * sphi;
    const double hs = sin(0.5 * sg);
    const double c2max = 4.0 * hs * hs, inv_s2 = 1.0 / (sg * sg);
    int64_t cp[kSmoothCache];
    double cw[kSmoothCache];
    int nc = 0;
    bool spill = false;
    double tot = 0.0;
    kernel_pixels(nside, xp, yp, zp, sp, pp, sg, c2max, inv_s2, [&](int64_t p, double w) {
      tot += w;
      if (nc < kSmoothCache) {
        cp[nc] = p;
        cw[nc] = w;
        ++nc;
      } else {
        spill = true;
      }
    });
    if (!(tot > 0.0)) {
      atomicAdd(map + ang2pix_ring(nside, zp, pp), 1.0);
      continue;
    }
    const double inv = 1.0 / tot;
    if (!spill) {
      for (int k = 0; k < nc; ++k) atomicAdd(map + cp[k], cw[k] * inv);
    } else {
      kernel_pixels(nside, xp, yp, zp, sp, pp, sg, c2max, inv_s2,
                    [&](int64_t p, double w) { atomicAdd(map + p, w * inv); });
    }
  }
}

// kappa = scale * (rho / nbar - 1), each operation rounded separately
__global__ void k_density_to_kappa(const double* __restrict__ rho, int64_t npix, double nbar, double scale,
                                   double* __restrict__ kappa) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
    kappa[i] = __dmul_rn(scale, __dsub_rn(__ddiv_rn(rho[i], nbar), 1.0));
}

static int grid_for(clc_ctx* ctx, int64_t n, int threads) {
  int64_t blocks = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms(ctx) * 16;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace clc

using namespace clc;

extern "C" int clc_bin_particles(clc_ctx* ctx, const double* z, const double* phi, int64_t n, int nside,
                                 int ordering, uint32_t* counts) {
  if (!ctx) return CLC_EINVAL;
  if (n < 0 || !valid_nside(nside) || (ordering != CLC_RING && ordering != CLC_NEST))
    return set_err(ctx, CLC_EINVAL, "clc_bin_particles: bad n, nside or ordering");
  if (n == 0) return CLC_OK;
  if (!z || !phi || !counts) return set_err(ctx, CLC_EINVAL, "clc_bin_particles: null pointer");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_bin", k_bin, grid_for(ctx, n, 256), 256, 0, z, phi, n, nside, ordering == CLC_NEST, counts);
  return launch_check(ctx, "k_bin");
}

extern "C" int clc_counts_to_kappa(clc_ctx* ctx, const uint32_t* counts, int nside, double nbar, double scale,
                                   double* kappa) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside) || !(nbar > 0)) return set_err(ctx, CLC_EINVAL, "clc_counts_to_kappa: bad nside or nbar");
  if (!counts || !kappa) return set_err(ctx, CLC_EINVAL, "clc_counts_to_kappa: null pointer");
  cudaSetDevice(ctx->device);
  const int64_t npix = 12ll * nside * nside;
  double* tab = (double*)scratch(ctx, 7, sizeof(double) * kKappaTable);
  if (!tab) return CLC_ENOMEM;
  CLC_LAUNCH(ctx, "k_counts_to_kappa", k_kappa_table, kKappaTable / 256, 256, 0, nbar, scale, tab);
  CLC_LAUNCH(ctx, "k_counts_to_kappa", k_counts_to_kappa, grid_for(ctx, npix, 256), 256, 0, counts, npix, nbar, scale,
             (const double*)tab, kappa);
  return launch_check(ctx, "k_counts_to_kappa");
}

extern "C" int clc_counts_to_kappa_masked(clc_ctx* ctx, const uint32_t* counts, const uint8_t* covered, int nside,
                                          double scale, double* kappa) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside)) return set_err(ctx, CLC_EINVAL, "clc_counts_to_kappa_masked: bad nside");
  if (!counts || !covered || !kappa) return set_err(ctx, CLC_EINVAL, "clc_counts_to_kappa_masked: null pointer");
  cudaSetDevice(ctx->device);
  const int64_t npix = 12ll * nside * nside;
  unsigned long long* sums = (unsigned long long*)scratch(ctx, 7, 2 * sizeof(unsigned long long));
  if (!sums) return CLC_ENOMEM;
  cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), ctx->stream);
  CLC_LAUNCH(ctx, "k_masked_sums", k_masked_sums, grid_for(ctx, npix, 256), 256, 0, counts, covered, npix, sums);
  CLC_LAUNCH(ctx, "k_counts_to_kappa", k_counts_to_kappa_masked, grid_for(ctx, npix, 256), 256, 0, counts, covered,
             npix, (const unsigned long long*)sums, scale, kappa);
  return launch_check(ctx, "k_counts_to_kappa_masked");
}

extern "C" int clc_degrade(clc_ctx* ctx, const double* fine, int nf, double* coarse, int ns) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nf) || !valid_nside(ns) || ns > nf) return set_err(ctx, CLC_EINVAL, "clc_degrade: bad nside");
  if (!fine || !coarse) return set_err(ctx, CLC_EINVAL, "clc_degrade: null pointer");
  cudaSetDevice(ctx->device);
  int shift = 0;
  while ((ns << (shift / 2)) < nf) shift += 2;
  const int64_t npc = 12ll * ns * ns;
  CLC_LAUNCH(ctx, "k_degrade", k_degrade, grid_for(ctx, npc, 256), 256, 0, fine, nf, coarse, ns, shift);
  return launch_check(ctx, "k_degrade");
}

extern "C" int clc_smooth_particles(clc_ctx* ctx, const double* z, const double* phi, int64_t n, int nside,
                                    double sigma, const double* sigma_each, double* map) {
  if (!ctx) return CLC_EINVAL;
  if (n < 0 || !valid_nside(nside) || nside > 8192 || (!sigma_each && !(sigma > 0.0 && sigma <= 0.5)))
    return set_err(ctx, CLC_EINVAL, "clc_smooth_particles: need n >= 0, nside <= 8192 and 0 < sigma <= 0.5");
  if (n == 0) return CLC_OK;
  if (!z || !phi || !map) return set_err(ctx, CLC_EINVAL, "clc_smooth_particles: null pointer");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_smooth_particles", k_smooth_particles, grid_for(ctx, n, 128), 128, 0, z, phi, sigma_each, n,
             nside, sigma, map);
  return launch_check(ctx, "k_smooth_particles");
}

extern "C" int clc_density_to_kappa(clc_ctx* ctx, const double* rho, int nside, double nbar, double scale,
                                    double* kappa) {
  if (!ctx) return CLC_EINVAL;
  if (!valid_nside(nside) || !(nbar > 0)) return set_err(ctx, CLC_EINVAL, "clc_density_to_kappa: bad nside or nbar");
  if (!rho || !kappa) return set_err(ctx, CLC_EINVAL, "clc_density_to_kappa: null pointer");
  cudaSetDevice(ctx->device);
  const int64_t npix = 12ll * nside * nside;
  CLC_LAUNCH(ctx, "k_density_to_kappa", k_density_to_kappa, grid_for(ctx, npix, 256), 256, 0, rho, npix, nbar, scale,
             kappa);
  return launch_check(ctx, "k_density_to_kappa");
}
