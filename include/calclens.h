/*
 * calclens.h - C ABI of the GB300 lens-plane library (libcalclens_gb300.so).
 *
 * The library computes the hot path of curved-sky multiple-plane weak-lensing
 * ray tracing (Becker 2012, "CALCLENS"): particle binning to HEALPix pixels,
 * the spherical-harmonic (SHT) Poisson solve of a lens plane, the SHT+MG
 * multigrid refinement on bundle patches, the deflection / shear derivatives
 * and the multiple-plane ray recursion.  Every step runs in hand-written CUDA
 * kernels for sm_103a.
 *
 * Conventions shared by all calls
 * -------------------------------
 * - Pointers are DEVICE pointers (caller-owned, already allocated) unless the
 *   argument name ends in _host.  The library never frees caller memory.
 * - Maps are HEALPix RING-ordered FP64 arrays of 12 nside^2 values unless an
 *   `ordering` argument says otherwise; nside must be a power of two in
 *   [1, 8192].  Positions are (z = cos theta, phi) in FP64, phi in [0, 2 pi].
 * - Spherical-harmonic coefficients a_lm (m >= 0, l <= lmax) are complex FP64
 *   stored as interleaved (re, im) pairs, packed m-major:
 *   index(l, m) = m (2 lmax + 1 - m) / 2 + l, (lmax + 1)(lmax + 2) / 2 pairs.
 *   Y_lm are orthonormal with the Condon-Shortley phase.
 * - Calls are asynchronous on the context's stream and return a status
 *   code before completion; clc_sync() waits and reports device-side errors.
 *   Argument errors are reported as CLC_EINVAL before anything is launched.
 *   No exception crosses the ABI.  A context is not thread-safe.
 * - Lens fields are given in the orthonormal (theta-hat, phi-hat) basis with
 *   the conventions of the paper's Appendix A: alpha = -grad psi,
 *   U_ab = covariant Hessian of psi, kappa = U_tt + U_pp (twice the standard
 *   convergence, Eq. lenspoisson), gamma_1 = (U_tt - U_pp) / 2, gamma_2 = U_tp.
 */
#ifndef CALCLENS_H
#define CALCLENS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  CLC_OK = 0,
  CLC_EINVAL = 1,        /* invalid argument; nothing was launched            */
  CLC_ENOMEM = 2,        /* device allocation failed                          */
  CLC_ECUDA = 3,         /* a CUDA runtime call or kernel failed              */
  CLC_ENOTCONVERGED = 4, /* MG hit max_cycles above tol; outputs are written  */
  CLC_ETIMEOUT = 5       /* a bounded device-side wait gave up                */
};

enum { CLC_RING = 0, CLC_NEST = 1 };             /* HEALPix ordering        */
enum { CLC_FP64 = 0, CLC_FP32 = 1, CLC_MIXED = 2 }; /* arithmetic of a solve */
enum { CLC_SOLVER_SHT = 0, CLC_SOLVER_SHTMG = 1 }; /* plane Poisson solver    */

typedef struct clc_ctx clc_ctx;
typedef struct clc_plane_solution clc_plane_solution;

/* Output lens fields; any pointer may be NULL to skip that field.  Each is a
 * device FP64 array with one value per point (pixel or ray). */
typedef struct clc_derivs {
  double* a_th; /* alpha_theta */
  double* a_ph; /* alpha_phi   */
  double* u_tt; /* U_theta-theta */
  double* u_pp; /* U_phi-phi     */
  double* u_tp; /* U_theta-phi   */
} clc_derivs;

/* Parameters of the SHT+MG plane solver (paper Sec. 3.2). */
typedef struct clc_mg_params {
  int nside_sht;    /* HEALPix Nside of the global SHT step                  */
  int lmax;         /* SHT band limit, lmax <= 4 nside_sht                   */
  int nside_bundle; /* Nside of the bundle cells; one MG patch per bundle    */
  int ncell;        /* cells per patch side on the finest level (power of 2, >= 16) */
  int nu1, nu2;     /* red-black Gauss-Seidel sweeps before / after the coarse step, 0..8, sum >= 1 */
  int max_cycles;   /* V-cycle cap when iterating to tol                     */
  int fixed_cycles; /* > 0: run exactly this many V-cycles, ignore tol       */
  double tol;       /* CLC_STOP_RESIDUAL: stop when max over patches ||f - L u||_2 / ||f||_2 < tol */
  int precision;    /* CLC_FP64: all FP64; CLC_FP32: FP32 V-cycles and residual
                       (FP64 coarsest solve); CLC_MIXED: FP32 V-cycles refining a
                       residual of FP64 accuracy (float-float), converging to the
                       same tol as CLC_FP64 */
  int stop_rule;    /* CLC_STOP_RESIDUAL (0, the rule above) or CLC_STOP_TAU (1):
                       the paper's rule (Sec. 3.2), stop when max over patches of
                       rms(f - L u) / rms(tau) < eps, tau = L_c R u - R L_f u the
                       truncation-error estimate on the next coarser level (R the
                       area-weighted restriction, the coarse ghost ring holding
                       2 psi_SHT at the coarse edge faces), rms over the patch's
                       fine and coarse cells */
  double eps;       /* CLC_STOP_TAU: the fraction (the paper uses 0.1 and 0.01) */
  int refine_cycles;/* CLC_MIXED: FP32 V-cycles between two float-float residual
                       refinements (0 = 2); with CLC_STOP_* checked after each */
} clc_mg_params;

enum { CLC_STOP_RESIDUAL = 0, CLC_STOP_TAU = 1 };

/* Ray state, structure of arrays of n rays (device FP64):
 * x[3][n] Cartesian position, beta[3][n] propagation direction,
 * A[4][n] and Ap[4][n] the inverse magnification matrices A^(n) and A^(n-1)
 * (row-major 2x2: A_tt, A_tp, A_pt, A_pp) in the (theta-hat, phi-hat) basis at
 * x, and bundle[n] the NEST index of each ray's home bundle (only read by the
 * SHT+MG solver; may be NULL for the pure-SHT solver). */
typedef struct clc_rays {
  int64_t n;
  double* x;
  double* beta;
  double* A;
  double* Ap;
  int32_t* bundle;
} clc_rays;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */

/* Create a context on CUDA device `device` that enqueues all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * The context owns scratch memory, SHT plans and Legendre tables. */
int clc_create(clc_ctx** ctx, int device, void* cuda_stream);
int clc_destroy(clc_ctx* ctx);
/* Wait for all enqueued work; returns CLC_ECUDA / CLC_ETIMEOUT if a kernel
 * failed or recorded a device-side error since the last sync. */
int clc_sync(clc_ctx* ctx);
/* Message describing the last non-OK status of this context ("" if none). */
const char* clc_last_error(const clc_ctx* ctx);
/* Release cached plans and Legendre tables (they are rebuilt on demand). */
int clc_release_caches(clc_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Step 1: binning (paper Sec. 3.2 source construction; Sec. 3.1 indexing)   */

/* counts[ang2pix(nside, z[i], phi[i])] += 1 for i < n, RING or NEST ordering.
 * The pixel index follows the HEALPix formulas of Gorski et al. (2005) with
 * every FP64 operation correctly rounded and unfused, so indices are
 * reproducible bit for bit.  counts (uint32[12 nside^2]) is accumulated, not
 * cleared.  n == 0 is a no-op. */
int clc_bin_particles(clc_ctx* ctx, const double* z, const double* phi, int64_t n,
                      int nside, int ordering, uint32_t* counts);

/* kappa[p] = scale * (counts[p] / nbar - 1) (Eq. lenspoisson for equal-mass
 * particles, nbar = particles per pixel), each operation rounded separately. */
int clc_counts_to_kappa(clc_ctx* ctx, const uint32_t* counts, int nside, double nbar,
                        double scale, double* kappa);

/* Adaptive Epanechnikov smoothing of unit-mass particles (Sec. 3.2): each
 * particle's mass is spread over the RING pixels whose centres lie at angular
 * distance theta < sigma from it, in proportion to the kernel
 * K(theta; sigma) ~ 1 - (theta / sigma)^2, the weights divided by their sum so
 * that the mass is conserved exactly; a particle with no pixel centre within
 * sigma puts its mass on its own pixel.  nside <= 8192.  sigma (radians, 0 < sigma <= 0.5) is
 * one smoothing length for all particles, or sigma_each[n] (device, may be
 * NULL) one per particle.  map (FP64[12 nside^2], particle number per pixel)
 * is accumulated, not cleared; sums of FP64 atomic adds, so the last bits
 * depend on their order.  n == 0 is a no-op. */
int clc_smooth_particles(clc_ctx* ctx, const double* z, const double* phi, int64_t n, int nside,
                         double sigma, const double* sigma_each, double* map);

/* kappa[p] = scale * (rho[p] / nbar - 1) (Eq. lenspoisson) for a smoothed
 * particle-number map rho, each operation rounded separately. */
int clc_density_to_kappa(clc_ctx* ctx, const double* rho, int nside, double nbar, double scale,
                         double* kappa);

/* Partial-sky source (Sec. 3.4): for a light cone that covers only the RING
 * pixels with covered[p] != 0 (uint8 mask), kappa[p] = scale * (counts[p] /
 * nbar - 1) on covered pixels with nbar = (particles in covered pixels) /
 * (number of covered pixels), the light cone's own mean density, and 0 (matter
 * at the mean density) elsewhere, so that kappa has no monopole.  Integer
 * sums, then the operations of clc_counts_to_kappa: reproducible bit for bit. */
int clc_counts_to_kappa_masked(clc_ctx* ctx, const uint32_t* counts, const uint8_t* covered, int nside,
                               double scale, double* kappa);

/* Coarse RING map = mean of the (nside_fine / nside_coarse)^2 NEST children of
 * every coarse pixel (children summed in NEST order): equal to binning the
 * same particles at nside_coarse. */
int clc_degrade(clc_ctx* ctx, const double* map_fine, int nside_fine, double* map_coarse,
                int nside_coarse);

/* ------------------------------------------------------------------------ */
/* Step 2: spherical-harmonic transforms and the SHT Poisson solve (Sec. 3.2) */

/* Limit the FP64 Legendre table (sum over m of (lmax + 2 - m) * 2 nside
 * doubles; 262 GB at nside 2048, lmax 4096) to `bytes` (0 = the free device
 * memory decides).  Larger tables are built and used one order range m0..m1
 * at a time inside each FP64 SHT call (same results; the recurrence is then
 * recomputed per call). */
int clc_set_table_budget(clc_ctx* ctx, size_t bytes);

/* a_lm = (4 pi / Npix) sum_p map[p] Y*_lm(p) (uniform quadrature). */
int clc_sht_analysis(clc_ctx* ctx, const double* map, int nside, int lmax, double* alm);
/* map[p] = sum_lm a_lm Y_lm(p) for a real field (m < 0 implied). */
int clc_sht_synthesis(clc_ctx* ctx, const double* alm, int nside, int lmax, double* map);

/* Pure-SHT plane solve (Sec. 3.2): analysis of kappa, psi_lm = -kappa_lm /
 * (l (l + 1)) with psi_00 = 0, synthesis of psi (if psi != NULL) and, for the
 * non-NULL fields of `out` (out may be NULL), the deflection and Hessian at
 * every pixel centre synthesised directly from psi_lm.
 * precision: CLC_FP64 (FP64 Legendre contraction) or CLC_MIXED (split
 * hi + lo FP16 tensor-core contraction with FP32 accumulation; needs
 * nside >= 64, relative L2 error of the outputs about 1e-6).
 * All maps are device pointers of 12 nside^2 doubles (RING order). */
int clc_poisson_sht(clc_ctx* ctx, const double* kappa, int nside, int lmax, int precision,
                    double* psi, const clc_derivs* out);

/* The pure-SHT plane solve of clc_poisson_sht for nplanes planes of the same
 * (nside, lmax) (the lens planes of one light cone, Sec. 3.2).  kappa and psi
 * are HOST arrays of nplanes DEVICE map pointers (psi may be NULL, entries
 * may not); out is NULL or a host array of nplanes clc_derivs.  With CLC_MIXED
 * up to 64 planes (21 with derivatives) share one pass over the FP16 lambda
 * table on the tensor cores; CLC_FP64 solves the planes one by one.  Errors:
 * CLC_EINVAL for bad sizes, a NULL kappa entry or nside < 64 with CLC_MIXED;
 * CLC_ENOMEM if the FP16 table (4 bytes per lambda_lm value and ring) does
 * not fit. */
int clc_poisson_sht_batch(clc_ctx* ctx, const double* const* kappa, int nplanes, int nside, int lmax,
                          int precision, double* const* psi, const clc_derivs* out);

/* A reusable plan for a fixed batch of pure-SHT plane solves of mixed sizes
 * (paper Sec. 3.2; mixed precision only): nplanes planes, plane i of
 * (nside[i], lmax[i]) with 64 <= nside <= 4096 and lmax <= 4 nside, grouped
 * into at most 8 classes of equal (nside, lmax) holding at most 64 planes
 * (21 with derivatives) each.
 * Every plane of the batch goes through six persistent launches (ring FFTs,
 * operand packing, tensor-core analysis, packing, tensor-core synthesis, ring
 * FFTs) whose work lists span all sizes.  flags: CLC_PLAN_GRAPH captures the
 * six launches in a CUDA graph on the first execution and replays it;
 * CLC_PLAN_TUNE times candidate launch shapes (pipeline depth, resident CTAs
 * per SM) on the first execution and keeps the fastest.  The plan owns its
 * intermediate buffers (device memory, freed by clc_sht_plan_destroy) and the
 * shared FP16 tables stay cached in the context.  Errors: CLC_EINVAL for
 * sizes outside the limits, CLC_ENOMEM if the tables or buffers do not fit. */
typedef struct clc_sht_plan clc_sht_plan;
#define CLC_PLAN_GRAPH 1
#define CLC_PLAN_TUNE 2
int clc_sht_plan_create(clc_ctx* ctx, int nplanes, const int* nside_host, const int* lmax_host, int derivatives,
                        int flags, clc_sht_plan** plan);
/* Solve every plane: kappa, psi are host arrays of nplanes device maps (psi
 * NULL or entries NULL to skip), out a host array of nplanes clc_derivs (used
 * when the plan was created with derivatives).  Asynchronous on the context's
 * stream; the host arrays may be reused as soon as the call returns. */
int clc_sht_plan_execute(clc_sht_plan* plan, const double* const* kappa, double* const* psi,
                         const clc_derivs* out);
/* Launch shapes in use (5 ints: analysis stages, analysis CTAs/SM, synthesis
 * stages, synthesis CTAs/SM, FFT CTAs/SM), the tuned time of each of the six
 * launches in ms (0 before tuning), and the device bytes the plan uses
 * (buffers plus its share of cached tables).  Any output may be NULL. */
int clc_sht_plan_info(const clc_sht_plan* plan, int* shape5, double* stage_ms6, size_t* device_bytes);
int clc_sht_plan_destroy(clc_sht_plan* plan);

/* ------------------------------------------------------------------------ */
/* Step 3: SHT+MG plane solve (Sec. 3.2)                                      */

/* Allocate the multigrid state of one plane (patches of all 12 nside_bundle^2
 * bundles) for maps of nside_fine.  The handle is owned by the caller and
 * freed with clc_solution_destroy. */
int clc_solution_create(clc_ctx* ctx, int nside_fine, const clc_mg_params* params,
                        clc_plane_solution** sol);
int clc_solution_destroy(clc_plane_solution* sol);
/* Partial sky (Sec. 3.4): the SHT still runs over the full sky, but MG
 * patches exist only for the nbundles distinct NEST bundles listed in
 * bundles_host (each < 12 nside_bundle^2), so memory and time scale with the
 * domain.  Lookups (clc_poisson_shtmg outputs, clc_lens_derivs, clc_ray_step,
 * galaxy traces) of points whose bundle has no patch return zero lens fields
 * (matter at the mean density does not deflect) and are counted. */
int clc_solution_create_domain(clc_ctx* ctx, int nside_fine, const clc_mg_params* params, const int32_t* bundles_host,
                               int nbundles, clc_plane_solution** sol);
/* Number of patches of the solution and the lookups outside its domain since
 * its last solve (0 on the full sky); waits for the context's stream. */
int clc_solution_domain(const clc_plane_solution* sol, int* npatch_host, int64_t* outside_host);
/* V-cycles run and final max residual ratio of the last solve into sol. */
int clc_solution_info(const clc_plane_solution* sol, int* cycles_host, double* residual_host);

/* SHT step at (nside_sht, lmax) on kappa_fine degraded to nside_sht, then
 * FAS multigrid V-cycles on every bundle patch (Dirichlet values and starting
 * guess from the SHT potential, source = kappa_fine, both by HEALPix
 * ring-bilinear interpolation), leaving the finest-level potential in `sol`.
 * If `out` is non-NULL, the fourth-order finite-difference lens fields are
 * evaluated at every pixel centre of nside_fine (each pixel in its own
 * bundle's patch).  Returns CLC_ENOTCONVERGED if max_cycles were used without
 * reaching tol (the solution and outputs are still written). */
int clc_poisson_shtmg(clc_ctx* ctx, const double* kappa_fine, int nside_fine,
                      const clc_mg_params* params, clc_plane_solution* sol,
                      const clc_derivs* out);

/* ------------------------------------------------------------------------ */
/* Step 4: lens fields at arbitrary points (Sec. 3.2 derivatives)            */

/* alpha and U at n points (z, phi), each evaluated in the patch of bundle[i]
 * (NEST index at nside_bundle; NULL = the bundle containing the point):
 * fourth-order finite differences on the finest patch level, bilinear
 * interpolation to the point, Appendix A formulas, rotation to the global
 * (theta-hat, phi-hat) basis. */
int clc_lens_derivs(clc_ctx* ctx, const clc_plane_solution* sol, const double* z,
                    const double* phi, const int32_t* bundle, int64_t n, const clc_derivs* out);

/* ------------------------------------------------------------------------ */
/* Step 5: multiple-plane ray recursion (Sec. 2.2, Appendix B)               */

/* Initialise rays at unit vectors of (z, phi) on the sphere of radius chi0:
 * x = chi0 n, beta = n, A = Ap = identity (Eq. betaprop, posprop, Atraj).
 * If bundle is non-NULL and nside_bundle > 0, bundle[i] = NEST pixel of the
 * ray's start at nside_bundle. */
int clc_rays_init(clc_ctx* ctx, const double* z, const double* phi, double chi0,
                  int nside_bundle, clc_rays* rays);

/* Rays on every RING pixel centre of nside (the paper's ray layout, Sec. 3.1):
 * ray k starts at pixel k; rays->n must equal 12 nside^2.  bundle[k] (if
 * nside_bundle > 0) = the pixel's NEST index shifted right by
 * 2 log2(nside / nside_bundle). */
int clc_rays_init_pixels(clc_ctx* ctx, int nside, double chi0, int nside_bundle, clc_rays* rays);

/* Advance all rays from the plane at chi_n to the sphere at chi_next using
 * the lens fields of that plane: either the SHT+MG solution `sol` (sol !=
 * NULL; rays looked up in their home bundle's patch) or RING maps `maps` of
 * nside_maps (sol == NULL; ring-bilinear interpolation of alpha as a tangent
 * 3-vector and U as a tangent 3x3 tensor).  chi_prev is the previous plane
 * (0 for the first plane).  Eq. Atraj, Eq. betaprop, Eq. posprop and the
 * parallel transport of Appendix B.  The rays must lie on the sphere of
 * radius chi_n, as clc_rays_init / clc_rays_init_pixels at chi_n and the
 * previous clc_ray_step to chi_n leave them: a ray's direction is taken as
 * x / chi_n. */
int clc_ray_step(clc_ctx* ctx, const clc_plane_solution* sol, const clc_derivs* maps,
                 int nside_maps, double chi_prev, double chi_n, double chi_next, clc_rays* rays);

/* Full driver of the paper's Sec. 3 steps 2-5 over nplanes planes: for plane m
 * solve for its potential from kappa_planes[m] (device RING maps of nside)
 * with the chosen solver, then advance the rays from chi_host[m] to
 * chi_host[m + 1] (chi_host has nplanes + 1 entries; the last is the source
 * sphere).  For CLC_SOLVER_SHT, `mg` supplies only nside_sht = nside of the
 * maps and lmax.  The rays must have been initialised at chi_host[0]. */
int clc_raytrace_planes(clc_ctx* ctx, int solver, const clc_mg_params* mg,
                        const double* const* kappa_planes_host, int nplanes, int nside,
                        const double* chi_host, clc_rays* rays);

/* ------------------------------------------------------------------------ */
/* Galaxy images by grid search (Sec. 2.3; grid-search implementation, Sec. 3) */

/* Images of ngal galaxies on one source sphere.  The rays must have been
 * started at the RING pixel centres of nside (clc_rays_init_pixels, n =
 * 12 nside^2) and traced to the galaxies' source sphere: x[3][n] their
 * positions there (any common positive length) and A[4][n] their inverse
 * magnification matrices in the (theta-hat, phi-hat) basis at x (device,
 * the layout of clc_rays).  g[3][ngal] (device) are the galaxies' source
 * positions as Cartesian vectors of any positive length.
 *
 * Triangles: between consecutive rings every pixel centre closes one
 * triangle with its predecessor on its ring and the last centre of the
 * neighbouring ring before it in longitude; ring 1 and the last ring close
 * the caps with two triangles each (2 npix - 4 triangles, counter-clockwise
 * seen from outside).  Triangle id 2 p + s belongs to centre p (s = 0: strip
 * below p's ring, s = 1: strip above; the caps are ids 3, 7, 2 (npix - 3),
 * 2 (npix - 1)).  A galaxy has one image per triangle whose rays' source
 * positions contain it in the gnomonic projection at the galaxy (triple
 * products det(g, x_i, x_j) of one sign, each edge's product evaluated once
 * on its endpoints in increasing pixel order, all vertices in g's
 * hemisphere); the image is the unit vector along sum_i lambda_i c_i, c_i
 * the vertices' pixel centres and lambda the barycentric coordinates in
 * that projection.  The matrix at the image is the ring-bilinear
 * interpolation (clc_ray_step's map interpolation) of the rays' A, each
 * parallel transported from the basis at its source position to the image.
 *
 * Outputs (device): nimg[ngal] the number of images found; for slot
 * q < max_images (1..8) in increasing triangle id: tri[q][ngal] the
 * triangle id (-1 if unused), img[3][q][ngal] (index (c * max_images + q) *
 * ngal + m) the image's unit vector (0 if unused), and A_img[4][q][ngal]
 * (same indexing) the matrix at the image in the basis there (0 if unused).  A and A_img are both NULL to skip
 * the matrices.  A galaxy vector of zero length or with a non-finite
 * component has no image.  The search visits only pixels near each galaxy, with a
 * radius taken from the largest displacement of a ray from its pixel centre
 * and the largest triangle on the source sphere, and finds every triangle
 * that contains the galaxy.  CLC_EINVAL before any search launch for bad
 * arguments, non-finite ray positions, or rays so far from their pixels
 * that the search would cover most of the sphere for many galaxies.  The
 * call waits for a small device-to-host copy of that radius. */
int clc_find_images(clc_ctx* ctx, int nside, const double* x, const double* A, int64_t ngal, const double* g,
                    int max_images, int32_t* nimg, int64_t* tri, double* img, double* A_img);

/* ------------------------------------------------------------------------ */
/* Differentiation: galaxy shears and their adjoint (Sec. 2.2, 3.2, App. D)   */

/* Shears of ngal galaxies through nplanes pure-SHT planes: one ray per
 * galaxy starts at its direction (gz = cos theta, gphi) on the sphere of
 * chi_host[0]; plane m's lens fields come from clc_poisson_sht of
 * kappa[m] (device RING map of nside, band limit lmax, CLC_FP64 or
 * CLC_MIXED) and the rays follow the plane recursion of clc_ray_step.  A
 * galaxy at comoving distance gchi with chi[n] <= gchi < chi[n + 1] takes
 * A_g = (1 - t) A^(n) + t A^(n+1), t = (chi[n+1] / gchi)(gchi - chi[n]) /
 * (chi[n+1] - chi[n]) (Appendix D); gamma (device, [2][ngal]) receives
 * gamma_1 = -(A_g00 - A_g11) / 2, gamma_2 = -(A_g01 + A_g10) / 2 (zero for
 * galaxies in front of chi[0]).  With tape != NULL the ray states entering
 * every plane (14 doubles per galaxy and plane) are kept in a new tape for
 * clc_gal_trace_adjoint; the kappa maps must stay alive until then. */
typedef struct clc_gal_tape clc_gal_tape;
int clc_gal_trace(clc_ctx* ctx, int nplanes, const double* const* kappa_host, int nside, int lmax, int precision,
                  const double* chi_host, int64_t ngal, const double* gz, const double* gphi, const double* gchi,
                  double* gamma, clc_gal_tape** tape);
/* Gradient of a loss with respect to every kappa map, given
 * gamma_bar = dLoss / dgamma (device, [2][ngal]): the planes are revisited
 * last to first, each plane's lens maps recomputed, each ray step
 * differentiated from its checkpoint and the adjoint of the SHT Poisson solve
 * applied.  kappa_bar is a host array of nplanes device maps (written). */
int clc_gal_trace_adjoint(clc_gal_tape* tape, const double* gamma_bar, double* const* kappa_bar_host);
/* clc_gal_trace with the SHT+MG solver of Sec. 3.2 on every plane (params:
 * as for clc_poisson_shtmg, precision CLC_FP64 only; kappa maps of nside =
 * the fine Nside): each galaxy's ray is looked up in the patch of the bundle
 * that contains its starting direction (rays keep their bundle, Sec. 3.1).
 * The tape's adjoint (clc_gal_trace_adjoint) recomputes each plane's patch
 * solution and differentiates the converged solve: the adjoint patch
 * problem L^T lambda = ubar is solved with the same V-cycles (W L is
 * symmetric for W = diag(sin theta'), so lambda = W L^-1 W^-1 ubar), to a
 * relative residual of min(tol / 100, 1e-12); lambda then goes back through
 * the transposed interpolations of the source and of the boundary values,
 * the (symmetric) SHT Poisson solve and the transposed degrade.  The
 * gradient is that of the converged solve, so the forward should converge
 * (tol or enough fixed_cycles).  Returns CLC_ENOTCONVERGED (tape and outputs
 * written) if a plane stopped at max_cycles above tol. */
int clc_gal_trace_mg(clc_ctx* ctx, int nplanes, const double* const* kappa_host, int nside,
                     const clc_mg_params* params, const double* chi_host, int64_t ngal, const double* gz,
                     const double* gphi, const double* gchi, double* gamma, clc_gal_tape** tape);
int clc_gal_tape_destroy(clc_gal_tape* tape);

/* ------------------------------------------------------------------------ */
/* Split-precision tensor-core contraction (the building block of the        */
/* mixed-precision Legendre transforms; the paper is all FP64)               */

/* d[b] = a_hi[b] b_hi[b]^T + a_hi[b] b_lo[b]^T + a_lo[b] b_hi[b]^T for b < batch,
 * on the tcgen05 tensor cores with FP32 accumulation.  a_* are FP16
 * [batch][M][K], b_* FP16 [batch][N][K] (row-major, K contiguous), d FP32
 * [batch][M][N].  Splitting x = x_hi + x_lo (x_hi = fp16(x), x_lo =
 * fp16(x - x_hi)) gives products of ~22-bit operands.  Needs M >= 1,
 * N in [16, 256] a multiple of 16, K a multiple of 64, batch <= 65535. */
int clc_gemm_f16x3(clc_ctx* ctx, const void* a_hi, const void* a_lo, const void* b_hi, const void* b_lo, int M,
                   int N, int K, int batch, float* d);

/* ------------------------------------------------------------------------ */
/* Spectra of the final lensing fields (paper Sec. 5)                        */

/* E and B coefficients (packed like clc_sht_analysis, l < 2 zero) of the
 * spin-2 shear gamma_1 + i gamma_2 given as RING maps in the (theta-hat,
 * phi-hat) basis.  Convention: a potential's shear gamma = eth^2 psi / 2
 * (gamma_1 = (U_tt - U_pp)/2, gamma_2 = U_tp) has E_lm = N_l psi_lm / 2,
 * N_l = sqrt((l+2)!/(l-2)!), and B_lm = 0; uniform quadrature as in
 * clc_sht_analysis. */
int clc_eb_analysis(clc_ctx* ctx, const double* gamma1, const double* gamma2, int nside, int lmax,
                    double* E_alm, double* B_alm);
/* cl[l] = (a_l0 b_l0* + 2 sum_{m>0} Re a_lm b_lm*) / (2l+1), l <= lmax
 * (b = a if alm2 is NULL). */
int clc_power_spectrum(clc_ctx* ctx, const double* alm, const double* alm2, int lmax, double* cl);
/* From inverse magnification matrices A (SoA A[4][12 nside^2]: A_tt, A_tp,
 * A_pt, A_pp of the rays started at the RING pixel centres, ray k at pixel
 * k), the spectra of kappa = 1 - (A_tt + A_pp)/2, of the E and B modes of
 * gamma = (-(A_tt - A_pp)/2, -(A_tp + A_pt)/2) and of omega = (A_tp - A_pt)/2
 * (Eq. invmagmat, Sec. 5): cl_out[4][lmax + 1] in the order kappa, E, B,
 * omega.  The maps are taken in the basis at each ray's image position (its
 * pixel centre).  x (device, SoA x[3][12 nside^2], nullable): the rays'
 * positions on the source sphere, in whose tangent basis the ray recursion
 * leaves A (clc_rays.x); each A is then first carried to its pixel centre by
 * the transport of Appendix B.  x == NULL: A is already in the pixel basis.
 * In the image basis C_l^E = s_l C_l^kappa and, at second order, C_l^B =
 * s_l C_l^omega, s_l = (l+2)(l-1)/(l(l+1)). */
int clc_lensing_spectra(clc_ctx* ctx, const double* x, const double* A, int nside, int lmax, double* cl_out);

/* ------------------------------------------------------------------------ */
/* Diagnostics (no counterpart in the paper beyond its per-step wall timers) */

/* enable != 0: start recording a CUDA-event pair around every kernel launch
 * of this context (previous records are dropped); 0: stop recording. */
int clc_profile(clc_ctx* ctx, int enable);
/* Launches recorded for the kernel `name` (e.g. "k_smooth") since profiling
 * was enabled and their summed device time in milliseconds (waits for the
 * stream). */
int clc_profile_query(clc_ctx* ctx, const char* name, int64_t* launches_host, double* total_ms_host);
/* Number of kernels this context has launched since it was created. */
int64_t clc_launch_count(const clc_ctx* ctx);
/* Exercise the bounded-wait error path of the pipelined kernels: one CTA
 * waits on an mbarrier that nothing completes and gives up after `polls`
 * polls (1 .. 2^20), recording a timeout in the context's device error word
 * exactly as the tensor-core and MG kernels do when a copy never lands.  The
 * next clc_sync returns CLC_ETIMEOUT and clears the word; the context stays
 * usable.  No copy or MMA is left in flight. */
int clc_diag_bounded_wait(clc_ctx* ctx, int64_t polls);

/* ------------------------------------------------------------------------ */
/* Allocation-free SHT analysis.  The paper has no counterpart: this entry   */
/* exists for callers of this library that cannot allocate device memory.    */
/*                                                                          */
/* clc_sht_analysis allocates on first use (context scratch, FFT plans,      */
/* Legendre tables).  Some callers cannot: code recording work into a CUDA   */
/* graph (allocation is not allowed while a stream is being captured), code  */
/* running inside a framework whose caching allocator owns all device memory,*/
/* or long-running services that must not grow their footprint after start. */
/* This variant computes the same a_lm (same conventions, same result within */
/* 1e-10 relative) with a direct DFT per ring and the Legendre recurrence on */
/* the fly; its only scratch, the ring Fourier coefficients, is a fixed      */
/* 2.1 MB file-scope device array that every GPU loading the library keeps   */
/* until the process exits.  It never calls cudaMalloc or cudaFree and needs */
/* no context: it runs on the calling thread's current device, on            */
/* `cuda_stream` (a cudaStream_t; NULL = legacy default stream).             */
/* Limits: nside a power of two <= 128, 0 <= lmax <= min(256, 4 nside);      */
/* anything else (or a NULL pointer) returns CLC_EINVAL without launching.   */
/* The first call on each device looks up the array's device address; make */
/* that first call before any stream capture.  All calls share the array:    */
/* calls whose work overlaps on the GPU (different streams, no ordering)     */
/* race and must not be issued.  Returns CLC_ECUDA if a launch fails.        */
int clc_sht_analysis_noalloc(const double* map, int nside, int lmax, double* alm, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CALCLENS_H */
