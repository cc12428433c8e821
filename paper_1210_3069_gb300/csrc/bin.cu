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
__global__ void k_counts_to_kappa(const uint32_t* __restrict__ counts, int64_t npix, double nbar,
                                  double scale, double* __restrict__ kappa) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) {
    kappa[i] = __dmul_rn(scale, __dsub_rn(__ddiv_rn((double)counts[i], nbar), 1.0));
  }
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
  CLC_LAUNCH(ctx, "k_counts_to_kappa", k_counts_to_kappa, grid_for(ctx, npix, 256), 256, 0, counts, npix, nbar, scale, kappa);
  return launch_check(ctx, "k_counts_to_kappa");
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
