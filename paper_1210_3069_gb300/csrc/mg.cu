// SHT+MG plane solver (paper Sec. 3.2): the SHT potential at (nside_sht,
// lmax) supplies Dirichlet values and the starting guess on one patch per
// bundle cell; FAS multigrid V-cycles with red-black Gauss-Seidel relaxation
// refine it to the fine resolution.
//
// Discretisation (the paper defers to Barros 1992; readings documented with
// the oracle): patch centred on the bundle centre rotated to (pi/2, 0), side
// 4 sqrt(pi/3) / nside_bundle, n x n cell-centred cells of spacing h,
// (Lu)_ij = aS_i (u_{i+1,j} - u_ij) + aN_i (u_{i-1,j} - u_ij) + b_i (u_{i,j+1} + u_{i,j-1} - 2 u_ij)
// with aS = sin t'_{i+1/2} / (h^2 sin t'_i), aN = sin t'_{i-1/2} / (h^2 sin t'_i),
// b = 1 / (h^2 sin^2 t'_i); Dirichlet values g on the patch edge through
// ghost cells holding 2 g - u_adjacent (the -u part folded into the
// diagonal); area-weighted restriction; bilinear prolongation with injection
// next to the edge; exact solve on the coarsest level.
//
// All patches of all levels are processed by one launch per operation; every
// patch is an independent problem (the paper's "embarrassingly parallel"
// MG step, Sec. 3.1), so the launches shard naturally over the SMs.
#include <cmath>

#include "mg.cuh"
#include "patch_fd.cuh"
#include "umma.cuh"


namespace clc {

MGView mg_view(const clc_plane_solution* sol) {
  MGView v;
  v.npatch = sol->npatch;
  v.n = sol->sizes[0];
  v.h = sol->h;
  v.inv_h = 1.0 / sol->h;
  v.rot = (const double*)sol->rot.p;
  v.u = (const double*)sol->base.p;
  v.slot = sol->partial ? (const int32_t*)sol->bundle_slot.p : nullptr;
  v.outside = sol->partial ? (unsigned long long*)sol->outside.p : nullptr;
  return v;
}

// Launch shape of the MG kernels: blocks of 32 x 8 threads over the cells of
// one patch, blockIdx.z = patch (no 64-bit index division anywhere).
constexpr int kBX = 32, kBY = 8;

// Float-float ("double-float") arithmetic: a value is hi + lo with two FP32
// words, |lo| <= ulp(hi) / 2 (about 48 significant bits).  Sums by Knuth's
// two-sum, products by the FMA-based exact product (Dekker's splitting made
// unnecessary by fmaf), each renormalised with Dekker's fast two-sum.  Used
// for the FP64-accurate residual of the mixed MG path, which would otherwise
// run on the FP64 pipe (1/58 of the FP32 rate on this GPU).
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 ff_fast_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float2 s = ff_two_sum(a.x, b.x);
  const float2 t = ff_two_sum(a.y, b.y);
  s.y += t.x;
  s = ff_fast_sum(s.x, s.y);
  s.y += t.y;
  return ff_fast_sum(s.x, s.y);
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_add_f(float2 a, float b) {
  float2 s = ff_two_sum(a.x, b);
  s.y += a.y;
  return ff_fast_sum(s.x, s.y);
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
  return ff_fast_sum(p, e);
}

// Float-float sum with one two-sum (the low words added directly): its error
// stays below about 2^-47 (|a| + |b|), the precision the residual needs,
// whose terms it sums (a residual is accurate only relative to its terms).
__device__ __forceinline__ float2 ff_add_lite(float2 a, float2 b) {
  const float2 s = ff_two_sum(a.x, b.x);
  return ff_fast_sum(s.x, s.y + (a.y + b.y));
}

// Position of cell (i, j) in a patch's source array (n x n cells, n even):
// the red cells ((i + j) even) first, then the black ones, each colour row by
// row, so that a colour's sweep reads its sources contiguously.
__host__ __device__ __forceinline__ size_t fidx(int n, int i, int j) {
  return ((size_t)((i + j) & 1) * n + i) * (size_t)(n >> 1) + (size_t)(j >> 1);
}

// Layout of a correction array (one patch of n x n cells): the two colours
// apart, each as rows i = -1 - kUHalo .. n + kUHalo of upitch(n) entries;
// cell (i, j), -1 <= j <= n, at entry j / 2 + 1 of row i of colour
// (i + j) & 1.  Entries outside the patch and its ghost ring are zero.  The
// rows of one colour are contiguous, so a band of rows (with the halo of up
// to kUHalo rows that the fused smoothing kernels read) moves in one bulk
// copy per colour, and the row pitch keeps every row 16-byte aligned.
constexpr int kUHalo = 17;   // 2 nu + 1 for the largest sweep count (8)
__host__ __device__ constexpr int upitch(int n) { return n / 2 + 4; }
__host__ __device__ __forceinline__ size_t uplane_of(int n) { return (size_t)(n + 2 + 2 * kUHalo) * upitch(n); }
__host__ __device__ __forceinline__ size_t upatch(int n) { return 2 * uplane_of(n); }
__host__ __device__ __forceinline__ size_t uidx(int n, int i, int j) {
  return (size_t)((i + j) & 1) * uplane_of(n) + (size_t)(i + 1 + kUHalo) * upitch(n) + (size_t)((j >> 1) + 1);
}

// store a value computed in FP64 in the solver's storage type
template <typename T>
__device__ __forceinline__ T from_double(double v) { return (T)v; }
template <>
__device__ __forceinline__ float2 from_double<float2>(double v) {
  const float h = d2f_rn(v);
  return make_float2(h, d2f_rn(v - f2d_exact(h)));
}

__global__ void k_mg_rotations(int nb, int npatch, const int32_t* __restrict__ slot_bundle, double* rot) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= npatch) return;
  const int b = slot_bundle ? slot_bundle[slot] : slot;
  const int64_t rp = nest2ring(nb, b);
  int64_t j;
  const int i = pix2ring(nb, rp, &j);
  const Ring r = ring_geom(nb, i);
  const double phi = r.phi0 + (2.0 * kPi) * (double)j / (double)r.npix;
  const double z = r.z, s = sqrt((1.0 - z) * (1.0 + z));
  const double cp = cos(phi), sp = sin(phi);
  double* R = rot + 9 * (size_t)slot;
  R[0] = s * cp; R[1] = s * sp; R[2] = z;
  R[3] = -sp;    R[4] = cp;     R[5] = 0.0;
  R[6] = -z * cp; R[7] = -z * sp; R[8] = s;
}

// global colatitude / longitude of patch-frame vector v in patch b
__device__ __forceinline__ void cell_angles(const double* R, const double* v, double* th, double* ph) {
  double g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = R[k] * v[0] + R[3 + k] * v[1] + R[6 + k] * v[2];
  *th = atan2(sqrt(g[0] * g[0] + g[1] * g[1]), g[2]);
  double p = atan2(g[1], g[0]);
  if (p < 0) p += 2.0 * kPi;
  *ph = p;
}

// base = psi_SHT at the cell centres, 2 psi_SHT at the edge faces (ghost ring)
__global__ void k_mg_setup_base(int n, const double* __restrict__ rot, const double* __restrict__ pvec,
                                const double* __restrict__ psi, int ns, const double* __restrict__ ring_th,
                                double* __restrict__ base) {
  const int b = blockIdx.z;
  const int k1 = blockIdx.y * kBY + threadIdx.y, k2 = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  if (k1 >= side || k2 >= side) return;
  const int cell = k1 * side + k2;
  double th, ph;
  cell_angles(rot + 9 * (size_t)b, pvec + 3 * (size_t)cell, &th, &ph);
  const double v = interp_map_tab(psi, ns, ring_th, th, ph);
  const bool ring = k1 == 0 || k2 == 0 || k1 == n + 1 || k2 == n + 1;
  base[(size_t)b * side * side + cell] = ring ? 2.0 * v : v;
}

// defect f' = kappa(cell) - L(base) and ||kappa||^2 per patch
template <typename T>
__global__ void k_mg_setup_defect(int n, const double* __restrict__ rot, const double* __restrict__ pvec,
                                  const double* __restrict__ kappa, int nf, const double* __restrict__ ring_th,
                                  const double* __restrict__ base, const double* __restrict__ coef,
                                  const double* __restrict__ diag, T* __restrict__ f, double* __restrict__ fnorm) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  double ff = 0.0;
  if (i < n && j < n) {
    const int cell = (i + 1) * side + (j + 1);
    double th, ph;
    cell_angles(rot + 9 * (size_t)b, pvec + 3 * (size_t)cell, &th, &ph);
    const double src = interp_map_tab(kappa, nf, ring_th, th, ph);
    const double* U = base + (size_t)b * side * side;
    const double nb = coef[i] * U[cell + side] + coef[n + i] * U[cell - side] + coef[2 * n + i] * (U[cell + 1] + U[cell - 1]);
    f[(size_t)b * n * n + fidx(n, i, j)] = from_double<T>(src - (nb - diag[i * n + j] * U[cell]));
    ff = src * src;
  }
  for (int o = 16; o > 0; o >>= 1) ff += __shfl_xor_sync(0xffffffffu, ff, o);
  if (threadIdx.x == 0 && ff != 0.0) atomicAdd(fnorm + b, ff);
}

// Float-float form of the four weights of a plan entry (same 32 bytes as
// the FP64 form), for the mixed-precision set-up.
struct alignas(32) FF4 {
  float2 w[4];
};

// Interpolation plan of one map for the positions of a patch level: either
// all (n+2)^2 positions (ring = 1) or the n^2 interior cells (ring = 0).
// ffw: weights stored as float-float pairs.  Entries that need the 8-pixel
// polar stencil keep (theta, phi) in FP64 with index -1.
__global__ void k_mg_plan(int n, int ring, const double* __restrict__ rot, const double* __restrict__ pvec, int nside,
                          const double* __restrict__ ring_th, int ffw, int4* __restrict__ idx,
                          double4_32a* __restrict__ w) {
  const int b = blockIdx.z;
  const int side = n + 2;
  const int m = ring ? side : n;
  const int k1 = blockIdx.y * kBY + threadIdx.y, k2 = blockIdx.x * kBX + threadIdx.x;
  if (k1 >= m || k2 >= m) return;
  const int cell = ring ? k1 * side + k2 : (k1 + 1) * side + (k2 + 1);
  double th, ph;
  cell_angles(rot + 9 * (size_t)b, pvec + 3 * (size_t)cell, &th, &ph);
  const Interp8 o = interp_weights_tab(nside, ring_th, th, ph);
  const size_t pos = (size_t)b * m * m + (size_t)k1 * m + k2;
  if (o.w[4] != 0.0 || o.w[5] != 0.0) {
    idx[pos] = make_int4(-1, 0, 0, 0);
    w[pos] = double4_32a{th, ph, 0.0, 0.0};
    return;
  }
  idx[pos] = make_int4((int)o.p[0], (int)o.p[1], (int)o.p[2], (int)o.p[3]);
  if (ffw) {
    FF4 q;
#pragma unroll
    for (int k = 0; k < 4; ++k) q.w[k] = from_double<float2>(o.w[k]);
    reinterpret_cast<FF4*>(w)[pos] = q;
  } else {
    w[pos] = double4_32a{o.w[0], o.w[1], o.w[2], o.w[3]};
  }
}

// FP64 map -> float-float pairs
__global__ void k_split_ff(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = from_double<float2>(src[k]);
}

// plan interpolation in float-float arithmetic (FP32 pipe); polar entries in FP64
__device__ __forceinline__ float2 apply_plan_ff(const float2* __restrict__ map_ff, const double* __restrict__ map,
                                                int nside, const double* __restrict__ ring_th, int4 ix,
                                                const double4_32a* __restrict__ wp, size_t pos) {
  if (ix.x < 0) {
    const double4_32a w = wp[pos];
    return from_double<float2>(interp_map_tab(map, nside, ring_th, w.x, w.y));
  }
  const FF4 q = reinterpret_cast<const FF4*>(wp)[pos];
  float2 v = ff_mul(q.w[0], map_ff[ix.x]);
  v = ff_add(v, ff_mul(q.w[1], map_ff[ix.y]));
  v = ff_add(v, ff_mul(q.w[2], map_ff[ix.z]));
  return ff_add(v, ff_mul(q.w[3], map_ff[ix.w]));
}

// Mixed set-up, float-float: base = psi_SHT interpolated (2 psi_SHT on the
// ghost ring), kept both as float-float pairs and as their FP64 sum.
// Rows per thread of the defect set-up (independent kappa gathers in flight).
constexpr int kSetupRows = 8;

__global__ void k_mg_setup_base_ff(int n, const int4* __restrict__ idx, const double4_32a* __restrict__ w,
                                   const float2* __restrict__ psi_ff, const double* __restrict__ psi, int ns,
                                   const double* __restrict__ ring_th, float2* __restrict__ base_ff,
                                   double* __restrict__ base) {
  const int b = blockIdx.z;
  const int k1 = blockIdx.y * kBY + threadIdx.y, k2 = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  if (k1 >= side || k2 >= side) return;
  const size_t pos = (size_t)b * side * side + (size_t)k1 * side + k2;
  float2 v = apply_plan_ff(psi_ff, psi, ns, ring_th, idx[pos], w, pos);
  if (k1 == 0 || k2 == 0 || k1 == n + 1 || k2 == n + 1) v = make_float2(2.f * v.x, 2.f * v.y);
  base_ff[pos] = v;
  base[pos] = f2d_exact(v.x) + f2d_exact(v.y);
}

// Mixed set-up, float-float: defect source f' = kappa - L base at the cells,
// ||kappa||^2 per patch.
__global__ void k_mg_setup_defect_ff(int n, const int4* __restrict__ idx, const double4_32a* __restrict__ w,
                                     const float2* __restrict__ kap_ff, const double* __restrict__ kappa, int nf,
                                     const double* __restrict__ ring_th, const float2* __restrict__ base_ff,
                                     const float2* __restrict__ coef, const float2* __restrict__ diag,
                                     float2* __restrict__ f, double* __restrict__ fnorm) {
  const int b = blockIdx.z;
  const int j = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  float ff = 0.f;
#pragma unroll
  for (int kr = 0; kr < kSetupRows; ++kr) {
    const int i = (blockIdx.y * kSetupRows + kr) * kBY + threadIdx.y;
    if (i >= n || j >= n) continue;
    const size_t pos = (size_t)b * n * n + (size_t)i * n + j;
    const float2 src = apply_plan_ff(kap_ff, kappa, nf, ring_th, idx[pos], w, pos);
    const float2* U = base_ff + (size_t)b * side * side + (size_t)(i + 1) * side + (j + 1);
    // L base = aS uS + aN uN + b (uE + uW) - diag uC
    const float2 nb = ff_add(ff_add(ff_mul(coef[i], U[side]), ff_mul(coef[n + i], U[-side])),
                             ff_add(ff_mul(coef[2 * n + i], ff_add(U[1], U[-1])), ff_neg(ff_mul(diag[i * n + j], U[0]))));
    f[(size_t)b * n * n + fidx(n, i, j)] = ff_add(src, ff_neg(nb));
    ff = fmaf(src.x, src.x, ff);
  }
  for (int o = 16; o > 0; o >>= 1) ff += __shfl_xor_sync(0xffffffffu, ff, o);
  if (threadIdx.x == 0 && ff != 0.f) atomicAdd(fnorm + b, (double)ff);
}

__device__ __forceinline__ double apply_plan(const double* __restrict__ map, int nside, const double* __restrict__ ring_th,
                                             int4 ix, double4_32a w) {
  if (ix.x < 0) return interp_map_tab(map, nside, ring_th, w.x, w.y);
  return w.x * map[ix.x] + w.y * map[ix.y] + w.z * map[ix.z] + w.w * map[ix.w];
}

__global__ void k_mg_setup_base_plan(int n, const int4* __restrict__ idx, const double4_32a* __restrict__ w,
                                     const double* __restrict__ psi, int ns, const double* __restrict__ ring_th,
                                     double* __restrict__ base) {
  const int b = blockIdx.z;
  const int k1 = blockIdx.y * kBY + threadIdx.y, k2 = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  if (k1 >= side || k2 >= side) return;
  const size_t pos = (size_t)b * side * side + (size_t)k1 * side + k2;
  const double v = apply_plan(psi, ns, ring_th, idx[pos], w[pos]);
  const bool ring = k1 == 0 || k2 == 0 || k1 == n + 1 || k2 == n + 1;
  base[pos] = ring ? 2.0 * v : v;
}

template <typename T>
__global__ void k_mg_setup_defect_plan(int n, const int4* __restrict__ idx, const double4_32a* __restrict__ w,
                                       const double* __restrict__ kappa, int nf, const double* __restrict__ ring_th,
                                       const double* __restrict__ base, const double* __restrict__ coef,
                                       const double* __restrict__ diag, T* __restrict__ f, double* __restrict__ fnorm) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  const int side = n + 2;
  double ff = 0.0;
  if (i < n && j < n) {
    const size_t pos = (size_t)b * n * n + (size_t)i * n + j;
    const double src = apply_plan(kappa, nf, ring_th, idx[pos], w[pos]);
    const int cell = (i + 1) * side + (j + 1);
    const double* U = base + (size_t)b * side * side;
    const double nb = coef[i] * U[cell + side] + coef[n + i] * U[cell - side] + coef[2 * n + i] * (U[cell + 1] + U[cell - 1]);
    f[(size_t)b * n * n + fidx(n, i, j)] = from_double<T>(src - (nb - diag[i * n + j] * U[cell]));
    ff = src * src;
  }
  for (int o = 16; o > 0; o >>= 1) ff += __shfl_xor_sync(0xffffffffu, ff, o);
  if (threadIdx.x == 0 && ff != 0.0) atomicAdd(fnorm + b, ff);
}

// ---------------------------------------------------------------------------
// Fused tile kernels of the V-cycle (red-black Gauss-Seidel, FAS restriction
// and prolongation of Sec. 3.2).  A CTA owns a kTile x kTile block of one
// patch (the whole patch when n < kTile) and stages the block with a halo of
// cells in shared memory, the two colours in separate arrays (region cell
// (r, c) at [(r + c) & 1][r][c / 2]).  Half-sweep h of a kernel updates the
// colour's cells of the region shrunk to halo - 1 - h cells around the block,
// so every value it reads is exact for that half-sweep: after the last one
// the block (and in the pre-smoothing kernel one more ring of cells) holds
// the values that the same half-sweeps over the whole patch give.  The
// arithmetic per cell is that of a plain sweep.  The kernels read the
// correction from one buffer and write their block to the other (the halo
// belongs to neighbouring CTAs, which may already have finished).

constexpr int kTile = 64;       // cells per block side
constexpr int kMaxSweeps = 8;   // nu1, nu2 limit (halo 2 nu + 1 <= 17 cells)

template <typename T>
struct alignas(4 * sizeof(T)) Quad {
  T x, y, z, w;
};

template <typename T>
struct Tile {
  Quad<T>* ra;   // per region row: aS, aN, b, 1 / diagonal (interior columns)
  Quad<T>* rb;   // per region row: 1 / diagonal (edge columns), diagonal (interior), diagonal (edge), area
  T* u;          // [2][W][W / 2]
  T* f;          // [2][W][W / 2]
  int n, W, hw, gi0, gj0;
  __device__ __forceinline__ int at(int r, int c) const { return (((r + c) & 1) * W + r) * hw + (c >> 1); }
};

__host__ __device__ constexpr int tile_side(int n) { return n < kTile ? n : kTile; }

template <typename T>
__host__ __device__ constexpr size_t tile_smem(int n, int halo) {
  return 2 * (size_t)(tile_side(n) + 2 * halo) * sizeof(Quad<T>) +
         2 * (size_t)(tile_side(n) + 2 * halo) * (tile_side(n) + 2 * halo) * sizeof(T);
}

template <typename T>
__device__ __forceinline__ Tile<T> tile_carve(unsigned char* sm, int n, int halo) {
  Tile<T> t;
  const int ts = tile_side(n), tiles = n / ts;
  t.n = n;
  t.W = ts + 2 * halo;
  t.hw = t.W >> 1;
  t.gi0 = (int)(blockIdx.x / tiles) * ts - halo;
  t.gj0 = (int)(blockIdx.x % tiles) * ts - halo;
  t.ra = reinterpret_cast<Quad<T>*>(sm);
  t.rb = t.ra + t.W;
  t.u = reinterpret_cast<T*>(t.rb + t.W);
  t.f = t.u + (size_t)t.W * t.W;
  return t;
}

// Stage the row coefficients, u over the region (zero beyond the ghost ring)
// and f over the region shrunk by fh cells.  The diagonal of a row takes one
// value in the interior columns and another in the two edge columns.
template <typename T>
__device__ __forceinline__ void tile_load(const Tile<T>& t, const T* __restrict__ U, const T* __restrict__ Fb,
                                          const T* __restrict__ coef, const T* __restrict__ invd,
                                          const T* __restrict__ diag, int fh) {
  const int n = t.n, tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  for (int r = tid; r < t.W; r += nt) {
    const int gi = t.gi0 + r;
    Quad<T> a{0, 0, 0, 0}, b{0, 0, 0, 0};
    if (gi >= 0 && gi < n) {
      const size_t row = (size_t)gi * n;
      a = Quad<T>{coef[gi], coef[n + gi], coef[2 * n + gi], invd[row + 1]};
      b = Quad<T>{invd[row], diag[row + 1], diag[row], coef[3 * n + gi]};
    }
    t.ra[r] = a;
    t.rb[r] = b;
  }
  for (int r = threadIdx.y; r < t.W; r += blockDim.y) {
    const int gi = t.gi0 + r;
    const bool urow = gi >= -1 && gi <= n;
    const bool frow = gi >= 0 && gi < n && r >= fh && r < t.W - fh;
    for (int c = threadIdx.x; c < t.W; c += blockDim.x) {
      const int gj = t.gj0 + c;
      T v = 0, w = 0;
      if (U && urow && gj >= -1 && gj <= n) v = U[uidx(n, gi, gj)];
      if (frow && gj >= 0 && gj < n && c >= fh && c < t.W - fh) w = Fb[fidx(n, gi, gj)];
      const int o = t.at(r, c);
      t.u[o] = v;
      t.f[o] = w;
    }
  }
}

// One colour of a red-black sweep over the region cells lo <= r, c < hi that
// lie inside the patch: u = (aS uS + aN uN + b (uE + uW) - f) / diagonal.
// Cells are dealt out flat over the CTA (row, colour index), so no lane idles
// on the short rows.
template <typename T>
__device__ __forceinline__ void tile_half_sweep(const Tile<T>& t, int colour, int lo, int hi) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int kc = (hi - lo) >> 1, total = (hi - lo) * kc;
  const int dq = nt / kc, dr = nt - dq * kc;
  int rr = tid / kc, kk = tid - rr * kc;
  const size_t plane = (size_t)t.W * t.hw;
  T* uc = t.u + colour * plane;
  const T* uo = t.u + (colour ^ 1) * plane;
  const T* fc = t.f + colour * plane;
  for (int idx = tid; idx < total; idx += nt) {
    const int r = lo + rr;
    const int p = (colour + r) & 1;          // column parity of the colour in row r
    const int k = ((lo - p + 1) >> 1) + kk;  // colour index of the cell in its row
    const int c = 2 * k + p;
    const int gi = t.gi0 + r, gj = t.gj0 + c;
    if (gi >= 0 && gi < t.n && gj >= 0 && gj < t.n) {
      const Quad<T> q = t.ra[r];
      const int row = r * t.hw;
      const T uE = uo[row + k + p], uW = uo[row + k + p - 1];
      const T uS = uo[row + t.hw + k], uN = uo[row - t.hw + k];
      const T v = fma(q.z, uE + uW, fma(q.y, uN, fma(q.x, uS, -fc[row + k])));
      uc[row + k] = v * ((gj == 0 || gj == t.n - 1) ? t.rb[r].x : q.w);
    }
    rr += dq;
    kk += dr;
    if (kk >= kc) {
      kk -= kc;
      ++rr;
    }
  }
}

// nu red-black sweeps; the region of half-sweep h is the block plus e0 - h cells
template <typename T>
__device__ __forceinline__ void tile_sweeps(const Tile<T>& t, int halo, int nu, int e0) {
  const int ts = t.W - 2 * halo;
  for (int h = 0; h < 2 * nu; ++h) {
    const int e = e0 - h;
    tile_half_sweep(t, h & 1, halo - e, halo + ts + e);
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void tile_store(const Tile<T>& t, int halo, T* __restrict__ U) {
  const int ts = t.W - 2 * halo;
  for (int r = halo + threadIdx.y; r < halo + ts; r += blockDim.y)
    for (int c = halo + threadIdx.x; c < halo + ts; c += blockDim.x) U[uidx(t.n, t.gi0 + r, t.gj0 + c)] = t.u[t.at(r, c)];
}

// Pre-smoothing and restriction: nu red-black sweeps on u_in (zero when
// u_in is NULL; written to u_out), then coarse cell (I, J) of the block gets
// the area-weighted average of the fine residual over its 2 x 2 children,
// fc = R (f - L u), the source of the coarse correction equation.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY) k_smooth_restrict(
    const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ f, const T* __restrict__ coef,
    const T* __restrict__ invd, const T* __restrict__ diag, const T* __restrict__ rden, int n, int nu,
    T* __restrict__ fc) {
  extern __shared__ __align__(16) unsigned char smem_sr[];
  const int halo = 2 * nu + 1;
  const Tile<T> t = tile_carve<T>(smem_sr, n, halo);
  const size_t b = blockIdx.z;
  tile_load(t, u_in ? u_in + b * upatch(n) : nullptr, f + b * n * n, coef, invd, diag, 1);
  __syncthreads();
  tile_sweeps(t, halo, nu, halo - 1);
  tile_store(t, halo, u_out + b * upatch(n));
  const int ts = t.W - 2 * halo, tc = ts >> 1, nc = n >> 1;
  const int I0 = (t.gi0 + halo) >> 1, J0 = (t.gj0 + halo) >> 1;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const size_t plane = (size_t)t.W * t.hw;
  for (int idx = tid; idx < tc * tc; idx += nt) {
    const int a = idx / tc, bb = idx - a * tc;
    T nr = 0;
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      const int r = halo + 2 * a + di;
      const Quad<T> q = t.ra[r], q2 = t.rb[r];
      T rs = 0;
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const int c = halo + 2 * bb + dj, gj = t.gj0 + c;
        const int col = (r + c) & 1, k = c >> 1, row = r * t.hw;
        const T* uo = t.u + (col ^ 1) * plane;
        const T ucv = t.u[col * plane + row + k];
        const T uE = uo[row + ((c + 1) >> 1)], uW = uo[row + ((c - 1) >> 1)];
        const T uS = uo[row + t.hw + k], uN = uo[row - t.hw + k];
        const T dg = (gj == 0 || gj == n - 1) ? q2.z : q2.y;
        // r = f - (aS uS + aN uN + b (uE + uW) - diag u)
        const T nb = fma(q.z, uE + uW, fma(q.y, uN, fma(q.x, uS, -dg * ucv)));
        rs += t.f[col * plane + row + k] - nb;
      }
      nr = fma(q2.w, rs, nr);
    }
    const int I = I0 + a, J = J0 + bb;
    fc[b * nc * nc + fidx(nc, I, J)] = nr * rden[I];   // rden = 1 / (2 (area_2I + area_2I+1))
  }
}

// Prolongation and post-smoothing: u_out = u_in + P(e_c) (cell-centred
// bilinear, injection next to the patch edge), then nu red-black sweeps.
// The coarse correction of the region (clamped to the coarse patch) is
// staged in shared memory after the fine arrays.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY) k_prolong_smooth(
    const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ f, const T* __restrict__ coef,
    const T* __restrict__ invd, const T* __restrict__ diag, const T* __restrict__ uc, int n, int nu) {
  extern __shared__ __align__(16) unsigned char smem_ps[];
  const int halo = 2 * nu;
  const Tile<T> t = tile_carve<T>(smem_ps, n, halo);
  const size_t b = blockIdx.z;
  const int nc = n >> 1;
  tile_load(t, u_in + b * upatch(n), f + b * n * n, coef, invd, diag, halo > 0 ? 1 : t.W);
  // coarse correction: rows / columns (gi0 / 2 - 1) .. (gi0 / 2 - 1 + Wc - 1)
  T* E = t.f + (size_t)t.W * t.W;
  const int Wc = t.hw + 2, Ic0 = (t.gi0 >> 1) - 1, Jc0 = (t.gj0 >> 1) - 1;
  const T* C = uc + b * upatch(nc);
  for (int a = threadIdx.y; a < Wc; a += blockDim.y) {
    const int I = min(max(Ic0 + a, 0), nc - 1);
    for (int c = threadIdx.x; c < Wc; c += blockDim.x) {
      const int J = min(max(Jc0 + c, 0), nc - 1);
      E[a * Wc + c] = C[uidx(nc, I, J)];
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < t.W; r += blockDim.y) {
    const int i = t.gi0 + r;
    if (i < 0 || i >= n) continue;
    const int a = (i >> 1) - Ic0, da = (i & 1) ? a + 1 : a - 1;
    for (int c = threadIdx.x; c < t.W; c += blockDim.x) {
      const int j = t.gj0 + c;
      if (j < 0 || j >= n) continue;
      const int bc = (j >> 1) - Jc0, db = (j & 1) ? bc + 1 : bc - 1;
      const T e11 = E[a * Wc + bc];
      T corr;
      if (i == 0 || j == 0 || i == n - 1 || j == n - 1)
        corr = e11;
      else
        corr = fma((T)9, e11, fma((T)3, E[da * Wc + bc] + E[a * Wc + db], E[da * Wc + db])) * (T)0.0625;
      t.u[t.at(r, c)] += corr;
    }
  }
  __syncthreads();
  tile_sweeps(t, halo, nu, halo - 1);
  tile_store(t, halo, u_out + b * upatch(n));
}

// ---------------------------------------------------------------------------
// Band form of the two fused kernels for patches of at most kBandMaxN cells a
// side: a CTA owns kBandRows whole rows of a patch, so the halo is needed
// only above and below (the patch's own edges are the Dirichlet ghost ring).
// Shared memory holds the region rows in the global layout of a correction
// array, so the region arrives by two bulk copies (one per colour, TMA
// engine, completion on an mbarrier) and the band's rows leave the same way;
// f arrives by two more.  In a half-sweep each warp owns 32 colour columns
// and walks a run of consecutive rows, keeping the other colour's values of
// rows i - 1, i, i + 1 of its column in registers.  The patch size is a
// template parameter, so every pitch is an immediate.

constexpr int kBandRows = 32;
constexpr int kBandMaxN = 256;
constexpr int kBandThreads = 512;
constexpr long long kMgWaitPolls = 1ll << 24;

template <int N>
struct BandGeo {
  static constexpr int nh = N / 2;                          // colour cells per row
  static constexpr int P = N / 2 + 4;                       // row pitch (upitch)
  static constexpr int br = N < kBandRows ? N : kBandRows;  // band rows
  static constexpr int kc = nh >= 64 ? 2 : 1;               // columns per thread in a half-sweep (32 apart)
  static constexpr int cg = nh >= 32 * kc ? nh / (32 * kc) : 1;   // warps across a row
  static constexpr int rg = (kBandThreads / 32) / cg;       // runs of rows per half-sweep
};

template <typename T>
__host__ __device__ constexpr size_t band_smem(int n, int halo) {
  return 2 * (size_t)((n < kBandRows ? n : kBandRows) + 2 * halo) *
         (sizeof(Quad<T>) + (size_t)(n / 2 + 4) * sizeof(T) + (size_t)(n / 2) * sizeof(T));
}

template <typename T, int N>
struct Band {
  using G = BandGeo<N>;
  Quad<T>* ra;   // per region row: aS, aN, b, 1 / diagonal (interior columns)
  Quad<T>* rb;   // per region row: 1 / diagonal (edge columns), diagonal (interior), diagonal (edge), area
  T* u;          // [2][W][P]: region rows gi0 .. gi0 + W - 1 of the two colours
  T* f;          // [2][W][nh]
  int W, gi0, bi0, uplane, fplane;
};

template <typename T, int N>
__device__ __forceinline__ Band<T, N> band_carve(unsigned char* sm, int halo) {
  using G = BandGeo<N>;
  Band<T, N> B;
  B.W = G::br + 2 * halo;
  B.bi0 = (int)blockIdx.x * G::br;
  B.gi0 = B.bi0 - halo;
  B.ra = reinterpret_cast<Quad<T>*>(sm);
  B.rb = B.ra + B.W;
  B.u = reinterpret_cast<T*>(B.rb + B.W);
  B.uplane = B.W * G::P;
  B.f = B.u + 2 * B.uplane;
  B.fplane = B.W * G::nh;
  return B;
}

// Start the bulk copies of the region (u of rows gi0 .. gi0 + W - 1, or zeros
// when Ub is NULL; f of the patch rows among gi0 + fh .. gi0 + W - fh - 1)
// and stage the row coefficients; band_wait completes the load.
template <typename T, int N>
__device__ __forceinline__ void band_issue(const Band<T, N>& B, uint64_t* bar, const T* __restrict__ Ub,
                                           const T* __restrict__ Fb, const T* __restrict__ coef,
                                           const T* __restrict__ invd, const T* __restrict__ diag, int fh) {
  using G = BandGeo<N>;
  if (threadIdx.x == 0) {
    umma::mbar_init(bar, 1);
    umma::fence_mbar_init();
    const int fa = max(B.gi0 + fh, 0), fb = min(B.gi0 + B.W - fh, N);
    const uint32_t ubytes = Ub ? (uint32_t)(B.uplane * sizeof(T)) : 0u;
    const uint32_t fbytes = fb > fa ? (uint32_t)((fb - fa) * G::nh * sizeof(T)) : 0u;
    umma::mbar_arrive_expect_tx(bar, 2 * ubytes + 2 * fbytes);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (ubytes)
        umma::bulk_g2s(B.u + c * B.uplane, Ub + c * uplane_of(N) + (size_t)(B.gi0 + 1 + kUHalo) * G::P, ubytes, bar);
      if (fbytes)
        umma::bulk_g2s(B.f + c * B.fplane + (fa - B.gi0) * G::nh, Fb + ((size_t)c * N + fa) * G::nh, fbytes, bar);
    }
  }
  for (int r = threadIdx.x; r < B.W; r += blockDim.x) {
    const int gi = B.gi0 + r;
    Quad<T> a{0, 0, 0, 0}, b{0, 0, 0, 0};
    if (gi >= 0 && gi < N) {
      const size_t row = (size_t)gi * N;
      a = Quad<T>{coef[gi], coef[N + gi], coef[2 * N + gi], invd[row + 1]};
      b = Quad<T>{invd[row], diag[row + 1], diag[row], coef[3 * N + gi]};
    }
    B.ra[r] = a;
    B.rb[r] = b;
  }
  if (!Ub)
    for (int e = threadIdx.x; e < 2 * B.uplane; e += blockDim.x) B.u[e] = 0;
}

// Wait (bounded) for the region; false on every thread if it did not arrive.
__device__ __forceinline__ bool band_wait(uint64_t* bar, int* d_err) {
  __syncthreads();   // also publishes the coefficient rows and the barrier initialisation
  const bool ok = __syncthreads_and(umma::mbar_wait(bar, 0, kMgWaitPolls));
  if (!ok && threadIdx.x == 0) {
    record_error(d_err, kDevTimeout);
    umma::mbar_wait(bar, 0, kMgWaitPolls);   // the copies in flight still target this CTA's memory
  }
  return ok;
}

template <int V>
struct IntC {
  static constexpr int value = V;
};

// One colour of a red-black sweep over the patch rows ga .. gb - 1 (all
// inside the patch, all columns).  A thread owns kc columns 32 apart and
// walks a run of rows; the column parity of the colour flips from row to
// row, so rows are taken in pairs with the parity fixed at compile time.
template <typename T, int N>
__device__ __forceinline__ void band_half_sweep(const Band<T, N>& B, int colour, int ga, int gb) {
  using G = BandGeo<N>;
  constexpr int KC = G::kc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunk = (gb - ga + G::rg - 1) / G::rg;
  const int r0 = ga + (warp / G::cg) * chunk, r1 = min(gb, r0 + chunk);
  const int k = 32 * KC * (warp % G::cg) + lane;
  if (r0 >= r1 || k >= G::nh) return;
  const int lr = r0 - B.gi0;
  const T* O = B.u + (colour ^ 1) * B.uplane + lr * G::P + k + 1;   // the other colour, row r0, column k
  T* C = B.u + colour * B.uplane + lr * G::P + k + 1;
  const T* F = B.f + colour * B.fplane + lr * G::nh + k;
  const Quad<T>* Q = B.ra + lr;
  const Quad<T>* R = B.rb + lr;
  const bool left = k == 0, right = k + 32 * (KC - 1) == G::nh - 1;
  T on[KC], oc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    on[c] = O[32 * c - G::P];
    oc[c] = O[32 * c];
  }
  auto step = [&](auto pc) {
    constexpr int p = decltype(pc)::value;   // column parity of the colour in this row
    const Quad<T> q = *Q;
    const bool edge = p ? right : left;
    const T ide = edge ? R->x : q.w;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const T os = O[32 * c + G::P];
      const T x = O[32 * c + 2 * p - 1];
      const T uE = p ? x : oc[c], uW = p ? oc[c] : x;
      const T id = (p ? c == KC - 1 : c == 0) ? ide : q.w;
      const T v = fma(q.z, uE + uW, fma(q.y, on[c], fma(q.x, os, -F[32 * c])));
      C[32 * c] = v * id;
      on[c] = oc[c];
      oc[c] = os;
    }
    O += G::P;
    C += G::P;
    F += G::nh;
    ++Q;
    ++R;
  };
  int cnt = r1 - r0;
  if (((colour + r0) & 1) == 0) {
    for (; cnt >= 2; cnt -= 2) {
      step(IntC<0>{});
      step(IntC<1>{});
    }
    if (cnt) step(IntC<0>{});
  } else {
    for (; cnt >= 2; cnt -= 2) {
      step(IntC<1>{});
      step(IntC<0>{});
    }
    if (cnt) step(IntC<1>{});
  }
}

template <typename T, int N>
__device__ __forceinline__ void band_sweeps(const Band<T, N>& B, int nu, int e0) {
  using G = BandGeo<N>;
  for (int h = 0; h < 2 * nu; ++h) {
    const int e = e0 - h;
    band_half_sweep(B, h & 1, max(0, B.bi0 - e), min(N, B.bi0 + G::br + e));
    __syncthreads();
  }
}

// Start the bulk copy of the band's own rows to global memory (thread 0
// waits for it at the end of the kernel).
template <typename T, int N>
__device__ __forceinline__ void band_store(const Band<T, N>& B, T* __restrict__ Ub) {
  using G = BandGeo<N>;
  umma::fence_proxy_async();   // this thread's shared-memory writes, visible to the bulk copy
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      umma::bulk_s2g(Ub + c * uplane_of(N) + (size_t)(B.bi0 + 1 + kUHalo) * G::P,
                     B.u + c * B.uplane + (B.bi0 - B.gi0) * G::P, (uint32_t)(G::br * G::P * sizeof(T)));
    umma::bulk_commit();
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(kBandThreads) k_band_smooth_restrict(
    const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ f, const T* __restrict__ coef,
    const T* __restrict__ invd, const T* __restrict__ diag, const T* __restrict__ rden, int nu,
    T* __restrict__ fc, int* d_err) {
  using G = BandGeo<N>;
  constexpr int NC = N / 2;
  extern __shared__ __align__(128) unsigned char smem_bsr[];
  __shared__ uint64_t bar;
  const int halo = 2 * nu + 1;
  const Band<T, N> B = band_carve<T, N>(smem_bsr, halo);
  const size_t b = blockIdx.z;
  band_issue(B, &bar, u_in ? u_in + b * upatch(N) : nullptr, f + b * N * N, coef, invd, diag, 1);
  if (!band_wait(&bar, d_err)) return;
  band_sweeps(B, nu, halo - 1);
  band_store(B, u_out + b * upatch(N));
  // Restriction of the band's rows.  Thread (J, run) walks coarse rows of
  // its run; fine columns 2J, 2J + 1 of fine row i are entry J + 1 of the
  // colour arrays i & 1 and (i + 1) & 1, their outer neighbours 2J - 1 and
  // 2J + 2 entries J and J + 2 of the other array.  After a black half-sweep
  // the residual of every black cell is zero (up to rounding: the cell was
  // just relaxed against its current neighbours), so with nu >= 1 only the
  // red children (2I, 2J) and (2I + 1, 2J + 1) contribute.
  constexpr int ncr = G::br / 2;
  constexpr int runs = kBandThreads / NC > 0 ? kBandThreads / NC : 1;
  constexpr int per = (ncr + runs - 1) / runs;
  const int J = threadIdx.x % NC, run = threadIdx.x / NC;
  const int Ia = (B.bi0 >> 1) + run * per, Ib = min((B.bi0 >> 1) + ncr, Ia + per);
  if (Ia < Ib) {
    auto at = [&](int i, int col, int e) -> T { return B.u[col * B.uplane + (i - B.gi0) * G::P + e]; };
    T n0 = at(2 * Ia - 1, (2 * Ia - 1) & 1, J + 1), n1 = at(2 * Ia - 1, (2 * Ia) & 1, J + 1);
    T a0 = at(2 * Ia, 0, J + 1), a1 = at(2 * Ia, 1, J + 1);
    const bool eL = J == 0, eR = J == NC - 1;
    for (int I = Ia; I < Ib; ++I) {
      // rows 2I - 1 (n), 2I (a), 2I + 1 (b), 2I + 2 (s): u(i, 2J), u(i, 2J + 1)
      const T b0 = at(2 * I + 1, 1, J + 1), b1 = at(2 * I + 1, 0, J + 1);
      const T s0 = at(2 * I + 2, 0, J + 1), s1 = at(2 * I + 2, 1, J + 1);
      T nr = 0;
      if (nu > 0) {
        // red child of row 2I: column 2J; red child of row 2I + 1: column 2J + 1
        const int r0 = 2 * I - B.gi0, r1 = r0 + 1;
        const T w = at(2 * I, 1, J);          // u(2I, 2J - 1)
        const T e = at(2 * I + 1, 1, J + 2);  // u(2I + 1, 2J + 2)
        const Quad<T> q0 = B.ra[r0], p0 = B.rb[r0], q1 = B.ra[r1], p1 = B.rb[r1];
        // r = f - (aS uS + aN uN + b (uE + uW) - diag u)
        const T nb0 = fma(q0.z, a1 + w, fma(q0.y, n0, fma(q0.x, b0, -(eL ? p0.z : p0.y) * a0)));
        const T nb1 = fma(q1.z, e + b0, fma(q1.y, a1, fma(q1.x, s1, -(eR ? p1.z : p1.y) * b1)));
        T rs0 = 0, rs1 = 0;
        rs0 += B.f[r0 * G::nh + J] - nb0;
        rs1 += B.f[r1 * G::nh + J] - nb1;
        nr = fma(p0.w, rs0, nr);
        nr = fma(p1.w, rs1, nr);
      } else {
#pragma unroll
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, r = i - B.gi0;
          const T c0 = di ? b0 : a0, c1 = di ? b1 : a1;   // this row
          const T N0 = di ? a0 : n0, N1 = di ? a1 : n1;   // row i - 1
          const T S0 = di ? s0 : b0, S1 = di ? s1 : b1;   // row i + 1
          const T w = at(i, di ^ 1, J);                   // u(i, 2J - 1)
          const T e = at(i, di, J + 2);                   // u(i, 2J + 2)
          const T f0 = B.f[di * B.fplane + r * G::nh + J];
          const T f1 = B.f[(di ^ 1) * B.fplane + r * G::nh + J];
          const Quad<T> q = B.ra[r], q2 = B.rb[r];
          const T nb0 = fma(q.z, c1 + w, fma(q.y, N0, fma(q.x, S0, -(eL ? q2.z : q2.y) * c0)));
          const T nb1 = fma(q.z, e + c0, fma(q.y, N1, fma(q.x, S1, -(eR ? q2.z : q2.y) * c1)));
          T rs = 0;
          rs += f0 - nb0;
          rs += f1 - nb1;
          nr = fma(q2.w, rs, nr);
        }
      }
      fc[b * NC * NC + fidx(NC, I, J)] = nr * rden[I];   // rden = 1 / (2 (area_2I + area_2I+1))
      n0 = b0;
      n1 = b1;
      a0 = s0;
      a1 = s1;
    }
  }
  if (threadIdx.x == 0) umma::bulk_wait_all();
}

template <typename T, int N>
__global__ void __launch_bounds__(kBandThreads) k_band_prolong_smooth(
    const T* __restrict__ u_in, T* __restrict__ u_out, const T* __restrict__ f, const T* __restrict__ coef,
    const T* __restrict__ invd, const T* __restrict__ diag, const T* __restrict__ uc, int nu, int* d_err) {
  using G = BandGeo<N>;
  constexpr int NC = N / 2, Pc = NC + 2;
  extern __shared__ __align__(128) unsigned char smem_bps[];
  __shared__ uint64_t bar;
  const int halo = 2 * nu;
  const Band<T, N> B = band_carve<T, N>(smem_bps, halo);
  const size_t b = blockIdx.z;
  band_issue(B, &bar, u_in + b * upatch(N), f + b * N * N, coef, invd, diag, halo > 0 ? 1 : B.W);
  // while the region arrives: coarse correction of coarse rows gi0 / 2 - 1 ..
  // gi0 / 2 - 1 + Wc - 1 and columns -1 .. NC (both clamped to the patch) at E[row][J + 1]
  T* E = B.f + 2 * B.fplane;
  const int Wc = (B.W >> 1) + 2, Ic0 = (B.gi0 >> 1) - 1;
  const T* Cc = uc + b * upatch(NC);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = warp; a < Wc; a += nw) {
    const int I = min(max(Ic0 + a, 0), NC - 1);
    for (int c = lane; c < Pc; c += 32) {
      const int J = min(max(c - 1, 0), NC - 1);
      E[a * Pc + c] = Cc[uidx(NC, I, J)];
    }
  }
  if (!band_wait(&bar, d_err)) return;
  // u += P(e) for the region cells in the patch: fine columns 2J, 2J + 1 of
  // a row take the coarse columns J - 1, J, J + 1 of two coarse rows.  With
  // nu >= 1 the first (red) half-sweep overwrites every red cell it reaches
  // without reading it, and the red cells it does not reach are never read:
  // only black cells need the correction.
  for (int r = warp; r < B.W; r += nw) {
    const int i = B.gi0 + r;
    if (i < 0 || i >= N) continue;
    const int a = (i >> 1) - Ic0, da = (i & 1) ? a + 1 : a - 1;
    const T* Ea = E + a * Pc;
    const T* Ed = E + da * Pc;
    T* u0 = B.u + (i & 1) * B.uplane + r * G::P;         // column 2J at J + 1
    T* u1 = B.u + ((i + 1) & 1) * B.uplane + r * G::P;   // column 2J + 1 at J + 1
    const bool rowedge = i == 0 || i == N - 1;
    const bool do0 = nu == 0 || (i & 1), do1 = nu == 0 || !(i & 1);   // column 2J black in odd rows
    for (int J = lane; J < NC; J += 32) {
      const int bc = J + 1;
      const T e11 = Ea[bc], d11 = Ed[bc];
      if (do0)
        u0[bc] += (rowedge || J == 0) ? e11 : fma((T)9, e11, fma((T)3, d11 + Ea[bc - 1], Ed[bc - 1])) * (T)0.0625;
      if (do1)
        u1[bc] += (rowedge || J == NC - 1) ? e11
                                             : fma((T)9, e11, fma((T)3, d11 + Ea[bc + 1], Ed[bc + 1])) * (T)0.0625;
    }
  }
  __syncthreads();
  band_sweeps(B, nu, halo - 1);
  band_store(B, u_out + b * upatch(N));
  if (threadIdx.x == 0) umma::bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Register-resident form of the two fused band kernels (FP32, nu = 2, patches
// of 128 and 256 cells a side).  A CTA still owns a band of BR rows of one
// patch with its halo rows (the region), but the region lives in registers:
// the region's rows are cut into NV parts of H rows, and thread (part v,
// quad q) holds the columns 4q .. 4q + 3 of the H rows of its part as two
// pairs, A = (4q, 4q + 2) and B = (4q + 1, 4q + 3).  A pair's two cells have
// one colour and share their row's coefficients, so a half-sweep relaxes both
// with packed two-wide FP32 instructions (correctly rounded per lane, the
// same values as the scalar ones).  Vertical neighbours are the thread's own
// registers; the column beyond the quad comes from the adjacent lane by a
// warp shuffle; the warps' outer columns and the rows where the parts meet
// pass through shared memory.
//
// Every region row is relaxed in every half-sweep.  Rows beyond the patch
// have zero coefficients and zero sources, so they keep the value zero; a
// row next to the region's edge reads zeros beyond it, and the error this
// introduces moves in by one row per half-sweep, so after 2 nu half-sweeps
// the band rows (and, with the halo of the pre-smoothing kernel, one row
// beyond them) hold exactly what sweeping the whole patch gives.  The
// arithmetic per cell is that of band_half_sweep, operation for operation,
// and the residual and prolongation formulas are those of the shared-memory
// kernels, so both give the same values.  The sources of the region's rows
// arrive in shared memory by one bulk copy per colour while the threads load
// their cells.
//
// Shared exchange slots: per part, eL slot w holds the column 4q of lane 0 of
// warp w (slot NWH: zeros, the ghost column beyond the patch) and oR slot
// w + 1 the column 4q + 3 of lane 31 (slot 0: zeros); TA / TB [v] hold the
// pairs of part v's first row, BA / BB [v + 1] those of its last row (slot
// NV of T and slot 0 of B: zeros beyond the region).  A half-sweep of one
// colour reads only the other colour's cells and publishes the cells it
// relaxes; in one row these are different slots (the A and B pairs, the even
// and the odd outer column), so the reads and writes of a half-sweep never
// meet and one barrier per half-sweep orders them.

template <int N, int HALO, int NV>
struct QBand {
  static constexpr int NH = N / 2;                  // source entries per colour row
  static constexpr int NQ = N / 4;                  // column quads = threads per part
  static constexpr int NWH = NQ / 32;               // warps per part
  static constexpr int BR = kBandRows;              // band rows
  static constexpr int W = BR + 2 * HALO, H = W / NV;   // region rows, rows per part
  static constexpr int NT = NQ * NV;                // threads
  static constexpr int NC = N / 2, Wc = W / 2 + 2, Pc = upitch(NC);   // coarse rows / pitch (prolongation)
  static constexpr size_t f_bytes = (size_t)2 * W * NH * sizeof(float);
  static constexpr size_t e_bytes = (size_t)2 * Wc * Pc * sizeof(float);
  static_assert(NQ % 32 == 0 && H * NV == W && H % 2 == 0 && H >= 2, "quad band geometry");
  static_assert(NT % 32 == 0, "whole warps: the shuffles name every lane");
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int N, int HALO, int NV>
struct QShared {
  using G = QBand<N, HALO, NV>;
  // per region row r, four float4 at rq[4 r]: (aS, aS, aN, aN), (b, b, 1/d, 1/d),
  // (1/d_edge, 1/d, 1/d, 1/d_edge), (d, d_edge, area, 0), with d the diagonal
  // of an interior cell, d_edge that of a first or last cell (zeros beyond the patch)
  float4 rq[4 * G::W];
  float eL[NV][G::NWH + 1][G::H], oR[NV][G::NWH + 1][G::H];
  float2 TA[NV + 1][G::NQ], TB[NV + 1][G::NQ], BA[NV + 1][G::NQ], BB[NV + 1][G::NQ];
  uint64_t bar;
};

template <int N, int HALO, int NV>
struct QState {
  using G = QBand<N, HALO, NV>;
  float2 A[G::H], B[G::H];
};

// Stage the row coefficients; bulk copy the sources of the region's rows in
// the patch, colour planes [2][W][NH], and zero those of rows beyond it; the
// barrier also expects `extra` bytes that the caller's thread 0 copies next.
template <int N, int HALO, int NV>
__device__ __forceinline__ void q_begin(QShared<N, HALO, NV>& X, float* Fs, const float* __restrict__ Fb, int gi0,
                                        const float* __restrict__ coef, const float* __restrict__ invd,
                                        const float* __restrict__ diag, uint32_t extra) {
  using G = QBand<N, HALO, NV>;
  const int fa = max(gi0, 0), fb = min(gi0 + G::W, N);
  if (threadIdx.x == 0) {
    umma::mbar_init(&X.bar, 1);
    umma::fence_mbar_init();
    const uint32_t bytes = (uint32_t)((fb - fa) * G::NH * sizeof(float));
    umma::mbar_arrive_expect_tx(&X.bar, 2 * bytes + extra);
#pragma unroll
    for (int c = 0; c < 2; ++c)
      umma::bulk_g2s(Fs + (c * G::W + fa - gi0) * G::NH, Fb + ((size_t)c * N + fa) * G::NH, bytes, &X.bar);
  }
  for (int r = threadIdx.x; r < G::W; r += blockDim.x) {
    const int gi = gi0 + r;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f), p0 = z, p1 = z, p2 = z, p3 = z;
    if (gi >= 0 && gi < N) {
      const size_t row = (size_t)gi * N;
      const float aS = coef[gi], aN = coef[N + gi], bh = coef[2 * N + gi], id = invd[row + 1], ide = invd[row];
      p0 = make_float4(aS, aS, aN, aN);
      p1 = make_float4(bh, bh, id, id);
      p2 = make_float4(ide, id, id, ide);
      p3 = make_float4(diag[row + 1], diag[row], coef[3 * N + gi], 0.f);
    }
    X.rq[4 * r] = p0;
    X.rq[4 * r + 1] = p1;
    X.rq[4 * r + 2] = p2;
    X.rq[4 * r + 3] = p3;
  }
  // rows beyond the patch (edge bands only): zero sources
  const int nlo = fa - gi0, nhi = gi0 + G::W - fb;
  for (int e = threadIdx.x; e < (nlo + nhi) * G::NH; e += blockDim.x) {
    const int rr = e / G::NH, k = e - rr * G::NH;
    const int r = rr < nlo ? rr : fb - gi0 + (rr - nlo);
    Fs[r * G::NH + k] = 0.f;
    Fs[(G::W + r) * G::NH + k] = 0.f;
  }
}

// load the thread's cells (rows beyond the patch are the zero rows of the layout)
template <int N, int HALO, int NV>
__device__ __forceinline__ void q_load(QState<N, HALO, NV>& S, const float* __restrict__ Ub, int g0, int q) {
  using G = QBand<N, HALO, NV>;
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int gi = g0 + r;
    if (Ub) {
      S.A[r] = f2(Ub[uidx(N, gi, 4 * q)], Ub[uidx(N, gi, 4 * q + 2)]);
      S.B[r] = f2(Ub[uidx(N, gi, 4 * q + 1)], Ub[uidx(N, gi, 4 * q + 3)]);
    } else {
      S.A[r] = S.B[r] = f2(0.f, 0.f);
    }
  }
}

// publish every exchange value of the thread (before the first half-sweep)
template <int N, int HALO, int NV>
__device__ __forceinline__ void q_publish_all(const QState<N, HALO, NV>& S, QShared<N, HALO, NV>& X, int v, int q) {
  using G = QBand<N, HALO, NV>;
  const int lane = threadIdx.x & 31, wh = q >> 5;
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < G::H; ++r) X.eL[v][wh][r] = S.A[r].x;
  }
  if (lane == 31) {
#pragma unroll
    for (int r = 0; r < G::H; ++r) X.oR[v][wh + 1][r] = S.B[r].y;
  }
  X.TA[v][q] = S.A[0];
  X.TB[v][q] = S.B[0];
  X.BA[v + 1][q] = S.A[G::H - 1];
  X.BB[v + 1][q] = S.B[G::H - 1];
  if (v == 0) {
    X.TA[NV][q] = X.TB[NV][q] = X.BA[0][q] = X.BB[0][q] = f2(0.f, 0.f);
    if (q < G::H) {
      for (int u = 0; u < NV; ++u) {
        X.eL[u][G::NWH][q] = 0.f;
        X.oR[u][0][q] = 0.f;
      }
    }
  }
}

// One half-sweep of colour C over the thread's rows; rb = v H, the part's
// first region row (even, so the colour of column 4q in row r is (r + HALO) & 1).
template <int N, int HALO, int NV, int C>
__device__ __forceinline__ void q_half_sweep(QState<N, HALO, NV>& S, QShared<N, HALO, NV>& X,
                                             const float* __restrict__ Fs, int v, int q, int offA, int offB) {
  using G = QBand<N, HALO, NV>;
  const int lane = threadIdx.x & 31, wh = q >> 5, rb = v * G::H;
  const float* Fr = Fs + (C * G::W + rb) * G::NH + 2 * q;
  const float4* R = X.rq + 4 * rb;
  const float* eLv = &X.eL[v][0][0];
  const float* oRv = &X.oR[v][0][0];
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const float4 p0 = R[4 * r], p1 = R[4 * r + 1];
    const float2 F = *reinterpret_cast<const float2*>(Fr + r * G::NH);
    const char* rqb = reinterpret_cast<const char*>(R + 4 * r);
    if (((r + HALO) & 1) == C) {
      // A = columns 4q, 4q + 2: west 4q - 1 (lane q - 1) and 4q + 1, east 4q + 1 and 4q + 3
      float w = __shfl_up_sync(0xffffffffu, S.B[r].y, 1);
      if (lane == 0) w = oRv[wh * G::H + r];
      const float2 nN = r > 0 ? S.A[r - 1] : X.BA[v][q];
      const float2 nS = r + 1 < G::H ? S.A[r + 1] : X.TA[v + 1][q];
      const float2 id = *reinterpret_cast<const float2*>(rqb + offA);
      const float2 s = __fadd2_rn(S.B[r], f2(w, S.B[r].x));
      const float2 t = __ffma2_rn(f2(p1.x, p1.y), s, __ffma2_rn(f2(p0.z, p0.w), nN, __ffma2_rn(f2(p0.x, p0.y), nS, neg2(F))));
      S.A[r] = __fmul2_rn(t, id);
      if (lane == 0) X.eL[v][wh][r] = S.A[r].x;
      if (r == 0) X.TA[v][q] = S.A[r];
      if (r == G::H - 1) X.BA[v + 1][q] = S.A[r];
    } else {
      // B = columns 4q + 1, 4q + 3: west 4q and 4q + 2, east 4q + 2 and 4q + 4 (lane q + 1)
      float e = __shfl_down_sync(0xffffffffu, S.A[r].x, 1);
      if (lane == 31) e = eLv[(wh + 1) * G::H + r];
      const float2 nN = r > 0 ? S.B[r - 1] : X.BB[v][q];
      const float2 nS = r + 1 < G::H ? S.B[r + 1] : X.TB[v + 1][q];
      const float2 id = *reinterpret_cast<const float2*>(rqb + offB);
      const float2 s = __fadd2_rn(S.A[r], f2(S.A[r].y, e));
      const float2 t = __ffma2_rn(f2(p1.x, p1.y), s, __ffma2_rn(f2(p0.z, p0.w), nN, __ffma2_rn(f2(p0.x, p0.y), nS, neg2(F))));
      S.B[r] = __fmul2_rn(t, id);
      if (lane == 31) X.oR[v][wh + 1][r] = S.B[r].y;
      if (r == 0) X.TB[v][q] = S.B[r];
      if (r == G::H - 1) X.BB[v + 1][q] = S.B[r];
    }
  }
}

// the four half-sweeps of nu = 2 (red, black, red, black), each closed by a
// barrier; the sweep loop stays rolled to keep the code in the instruction cache
template <int N, int HALO, int NV>
__device__ __forceinline__ void q_sweeps(QState<N, HALO, NV>& S, QShared<N, HALO, NV>& X, const float* __restrict__ Fs,
                                         int v, int q) {
  using G = QBand<N, HALO, NV>;
  // byte offsets of the thread's inverse diagonals in a row's rq block:
  // (1/d_edge, 1/d) for the first quad's A pair, (1/d, 1/d_edge) for the last quad's B pair
  const int offA = q == 0 ? 32 : 24, offB = q == G::NQ - 1 ? 40 : 24;
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    q_half_sweep<N, HALO, NV, 0>(S, X, Fs, v, q, offA, offB);
    __syncthreads();
    q_half_sweep<N, HALO, NV, 1>(S, X, Fs, v, q, offA, offB);
    __syncthreads();
  }
}

// store the band rows among the thread's rows
template <int N, int HALO, int NV>
__device__ __forceinline__ void q_store(const QState<N, HALO, NV>& S, float* __restrict__ Ub, int gi0, int v, int q) {
  using G = QBand<N, HALO, NV>;
  const int rb = v * G::H;
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r;
    if (rg < HALO || rg >= HALO + G::BR) continue;
    const int gi = gi0 + rg;
    Ub[uidx(N, gi, 4 * q)] = S.A[r].x;
    Ub[uidx(N, gi, 4 * q + 1)] = S.B[r].x;
    Ub[uidx(N, gi, 4 * q + 2)] = S.A[r].y;
    Ub[uidx(N, gi, 4 * q + 3)] = S.B[r].y;
  }
}

// halo rows of the pre-smoothing kernel's region: 2 nu, plus one for the
// restriction's stencil (more only to make the region split evenly)
constexpr int kSRHalo = 5;

template <int N, int NV>
__global__ void __launch_bounds__(QBand<N, kSRHalo, NV>::NT) k_reg_smooth_restrict(
    const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ f,
    const float* __restrict__ coef, const float* __restrict__ invd, const float* __restrict__ diag,
    const float* __restrict__ rden, float* __restrict__ fc, int* d_err) {
  constexpr int HALO = kSRHalo;
  using G = QBand<N, HALO, NV>;
  extern __shared__ __align__(128) unsigned char smem_rsr[];
  float* Fs = reinterpret_cast<float*>(smem_rsr);
  __shared__ QShared<N, HALO, NV> X;
  const size_t b = blockIdx.z;
  const int gi0 = blockIdx.x * G::BR - HALO;
  const int v = threadIdx.x / G::NQ, q = threadIdx.x % G::NQ, lane = threadIdx.x & 31, wh = q >> 5;
  const int rb = v * G::H;
  q_begin<N, HALO, NV>(X, Fs, f + b * N * N, gi0, coef, invd, diag, 0);
  QState<N, HALO, NV> S;
  q_load<N, HALO, NV>(S, u_in ? u_in + b * upatch(N) : nullptr, gi0 + rb, q);   // while the sources arrive
  q_publish_all<N, HALO, NV>(S, X, v, q);
  if (!band_wait(&X.bar, d_err)) return;
  q_sweeps<N, HALO, NV>(S, X, Fs, v, q);
  q_store<N, HALO, NV>(S, u_out + b * upatch(N), gi0, v, q);
  // Residual of the red cells of the band rows among the thread's rows (the
  // black residuals vanish after the last, black, half-sweep, which also
  // published the black values read here), r = 0 + (f - (aS uS + aN uN +
  // b (uE + uW) - diag u)), written over the red source it used.
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r;
    if (rg < HALO || rg >= HALO + G::BR) continue;
    const float4 p0 = X.rq[4 * rg], p1 = X.rq[4 * rg + 1], p3 = X.rq[4 * rg + 3];
    float2* Fr = reinterpret_cast<float2*>(Fs + rg * G::NH + 2 * q);
    float2 nb;
    if (((r + HALO) & 1) == 0) {   // red pair A (row of even gi)
      float w = __shfl_up_sync(0xffffffffu, S.B[r].y, 1);
      if (lane == 0) w = X.oR[v][wh][r];
      const float2 nN = r > 0 ? S.A[r - 1] : X.BA[v][q];
      const float2 nS = r + 1 < G::H ? S.A[r + 1] : X.TA[v + 1][q];
      const float2 d = f2(q == 0 ? p3.y : p3.x, p3.x);
      nb = __ffma2_rn(f2(p1.x, p1.y), __fadd2_rn(S.B[r], f2(w, S.B[r].x)),
                      __ffma2_rn(f2(p0.z, p0.w), nN, __ffma2_rn(f2(p0.x, p0.y), nS, __fmul2_rn(neg2(d), S.A[r]))));
    } else {                        // red pair B (row of odd gi)
      float e = __shfl_down_sync(0xffffffffu, S.A[r].x, 1);
      if (lane == 31) e = X.eL[v][wh + 1][r];
      const float2 nN = r > 0 ? S.B[r - 1] : X.BB[v][q];
      const float2 nS = r + 1 < G::H ? S.B[r + 1] : X.TB[v + 1][q];
      const float2 d = f2(p3.x, q == G::NQ - 1 ? p3.y : p3.x);
      nb = __ffma2_rn(f2(p1.x, p1.y), __fadd2_rn(S.A[r], f2(S.A[r].y, e)),
                      __ffma2_rn(f2(p0.z, p0.w), nN, __ffma2_rn(f2(p0.x, p0.y), nS, __fmul2_rn(neg2(d), S.B[r]))));
    }
    *Fr = __fadd2_rn(f2(0.f, 0.f), __fadd2_rn(*Fr, neg2(nb)));
  }
  __syncthreads();
  // Restriction: coarse cells (I, 2q), (I, 2q + 1) from the red residuals of
  // rows 2I and 2I + 1 weighted by their areas, in that order, times rden(I).
  constexpr int NC = G::NC;
  float* fcb = fc + b * NC * NC;
  for (int Il = v; Il < G::BR / 2; Il += NV) {
    const int rg = HALO + 2 * Il, I = (gi0 + rg) >> 1;
    const float a0 = X.rq[4 * rg + 3].z, a1 = X.rq[4 * rg + 7].z;
    const float2 rs0 = *reinterpret_cast<const float2*>(Fs + rg * G::NH + 2 * q);
    const float2 rs1 = *reinterpret_cast<const float2*>(Fs + (rg + 1) * G::NH + 2 * q);
    float2 nr = __ffma2_rn(f2(a0, a0), rs0, f2(0.f, 0.f));
    nr = __ffma2_rn(f2(a1, a1), rs1, nr);
    const float rd = rden[I];
    const float2 out = __fmul2_rn(nr, f2(rd, rd));
    fcb[fidx(NC, I, 2 * q)] = out.x;
    fcb[fidx(NC, I, 2 * q + 1)] = out.y;
  }
}

template <int N, int NV>
__global__ void __launch_bounds__(QBand<N, 4, NV>::NT) k_reg_prolong_smooth(
    const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ f,
    const float* __restrict__ coef, const float* __restrict__ invd, const float* __restrict__ diag,
    const float* __restrict__ uc, int* d_err) {
  constexpr int HALO = 4;
  using G = QBand<N, HALO, NV>;
  constexpr int NC = G::NC, Wc = G::Wc, Pc = G::Pc;
  extern __shared__ __align__(128) unsigned char smem_rps[];
  float* Fs = reinterpret_cast<float*>(smem_rps);
  float* E = Fs + 2 * G::W * G::NH;
  __shared__ QShared<N, HALO, NV> X;
  const size_t b = blockIdx.z;
  const int gi0 = blockIdx.x * G::BR - HALO;
  const int v = threadIdx.x / G::NQ, q = threadIdx.x % G::NQ;
  const int rb = v * G::H;
  // with the sources, the coarse correction's rows gi0 / 2 - 1 .. + Wc - 1 of
  // both colour planes (rows beyond the coarse patch are zero rows of the layout)
  const uint32_t cbytes = (uint32_t)(Wc * Pc * sizeof(float));
  q_begin<N, HALO, NV>(X, Fs, f + b * N * N, gi0, coef, invd, diag, 2 * cbytes);
  if (threadIdx.x == 0) {
    const float* Cc = uc + b * upatch(NC) + (size_t)((gi0 >> 1) - 1 + 1 + kUHalo) * Pc;
#pragma unroll
    for (int c = 0; c < 2; ++c) umma::bulk_g2s(E + c * Wc * Pc, Cc + c * uplane_of(NC), cbytes, &X.bar);
  }
  QState<N, HALO, NV> S;
  q_load<N, HALO, NV>(S, u_in + b * upatch(N), gi0 + rb, q);   // while the sources and the coarse rows arrive
  if (!band_wait(&X.bar, d_err)) return;
  // u += P(e_c) on the black cells of the thread's rows (the red ones are
  // overwritten by the first half-sweep before anything reads them): in row
  // gi the black cells are the A pair for odd gi, the B pair for even gi;
  // fine row gi takes coarse rows I = gi / 2 and I -+ 1 (gi0 is even).  E
  // holds coarse rows gi0 / 2 - 1 .. in the correction layout: coarse cell
  // (I, J) at entry J / 2 + 1 of colour plane (I + J) & 1.  Rows and columns
  // beyond the coarse patch hold zeros, read only where the patch's edge cells
  // take the injected value instead; rows beyond the patch stay zero.
  const float2 nine = f2(9.f, 9.f), three = f2(3.f, 3.f), sixteenth = f2(0.0625f, 0.0625f);
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r, gi = gi0 + rg;
    if ((unsigned)gi >= (unsigned)N) continue;
    const bool rowedge = gi == 0 || gi == N - 1;
    const int a = (rg >> 1) + 1, da = (r & 1) ? a + 1 : a - 1;
    // plane of coarse column 2q in coarse row I = gi0 / 2 - 1 + a: the parity of I
    const int pa = (a + (gi0 >> 1) + 1) & 1, pd = pa ^ 1;
    const float* Ea0 = E + (pa * Wc + a) * Pc + q;        // even coarse columns 2q - 2 + 2j (entry q + j)
    const float* Ea1 = E + ((pa ^ 1) * Wc + a) * Pc + q;  // odd coarse columns 2q - 1 + 2j
    const float* Ed0 = E + (pd * Wc + da) * Pc + q;       // row I -+ 1: even columns in the other plane
    const float* Ed1 = E + ((pd ^ 1) * Wc + da) * Pc + q;
    const float2 e11 = f2(Ea0[1], Ea1[1]), d11 = f2(Ed0[1], Ed1[1]);   // columns 2q, 2q + 1
    if (r & 1) {   // odd row: A = coarse columns 2q, 2q + 1, outer neighbours 2q - 1, 2q
      const float2 c = __fmul2_rn(__ffma2_rn(nine, e11, __ffma2_rn(three, __fadd2_rn(d11, f2(Ea1[0], Ea0[1])), f2(Ed1[0], Ed0[1]))),
                                  sixteenth);
      S.A[r] = __fadd2_rn(S.A[r], f2((rowedge || q == 0) ? e11.x : c.x, rowedge ? e11.y : c.y));
    } else {       // even row: B = coarse columns 2q, 2q + 1, outer neighbours 2q + 1, 2q + 2
      const float2 c = __fmul2_rn(__ffma2_rn(nine, e11, __ffma2_rn(three, __fadd2_rn(d11, f2(Ea1[1], Ea0[2])), f2(Ed1[1], Ed0[2]))),
                                  sixteenth);
      S.B[r] = __fadd2_rn(S.B[r], f2(rowedge ? e11.x : c.x, (rowedge || q == G::NQ - 1) ? e11.y : c.y));
    }
  }
  q_publish_all<N, HALO, NV>(S, X, v, q);
  __syncthreads();
  q_sweeps<N, HALO, NV>(S, X, Fs, v, q);
  q_store<N, HALO, NV>(S, u_out + b * upatch(N), gi0, v, q);
}

// ---------------------------------------------------------------------------
// Eight columns per thread (256-cell patches): the same register-resident
// band kernels with thread (part v, octet o) holding the columns 8o .. 8o + 7
// of its part's rows as four same-colour pairs, A0 = (8o, 8o + 2),
// A1 = (8o + 4, 8o + 6), B0 = (8o + 1, 8o + 3), B1 = (8o + 5, 8o + 7).  A
// row is one warp, so the horizontal neighbours beyond the octet come by
// shuffle alone and the patch's ghost columns are zeros at the row's first
// and last lane; the sources of a pair of pairs arrive as one 16-byte
// shared-memory load.  Operation for operation the arithmetic of the
// four-column kernels.

template <int N, int HALO, int NV>
struct OBand {
  static constexpr int NH = N / 2;                  // source entries per colour row
  static constexpr int NO = N / 8;                  // octets = threads per part
  static constexpr int BR = kBandRows;
  static constexpr int W = BR + 2 * HALO, H = W / NV;
  static constexpr int NT = NO * NV;
  static constexpr int WID = 32;                    // shuffle width
  static constexpr int NC = N / 2, Wc = W / 2 + 2, Pc = upitch(NC);
  static constexpr size_t f_bytes = (size_t)2 * W * NH * sizeof(float);
  static constexpr size_t e_bytes = (size_t)2 * Wc * Pc * sizeof(float);
  static_assert(NO == 32, "a part row is one warp");
  static_assert(NT % 32 == 0, "whole warps: the shuffles name every lane");
  static_assert(H * NV == W && H % 2 == 0, "octet band geometry");
};

template <int N, int HALO, int NV>
struct OShared {
  using G = OBand<N, HALO, NV>;
  float4 rq[4 * G::W];
  float4 TA[NV + 1][G::NO], TB[NV + 1][G::NO], BA[NV + 1][G::NO], BB[NV + 1][G::NO];
  uint64_t bar;
};

template <int N, int HALO, int NV>
struct OState {
  using G = OBand<N, HALO, NV>;
  float2 A0[G::H], A1[G::H], B0[G::H], B1[G::H];
};

__device__ __forceinline__ float4 pk4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

// row coefficients and sources (as the four-column kernels, rq rows of 64 B)
template <int N, int HALO, int NV>
__device__ __forceinline__ void o_begin(OShared<N, HALO, NV>& X, float* Fs, const float* __restrict__ Fb, int gi0,
                                        const float* __restrict__ coef, const float* __restrict__ invd,
                                        const float* __restrict__ diag, uint32_t extra) {
  using G = OBand<N, HALO, NV>;
  const int fa = max(gi0, 0), fb = min(gi0 + G::W, N);
  if (threadIdx.x == 0) {
    umma::mbar_init(&X.bar, 1);
    umma::fence_mbar_init();
    const uint32_t bytes = (uint32_t)((fb - fa) * G::NH * sizeof(float));
    umma::mbar_arrive_expect_tx(&X.bar, 2 * bytes + extra);
#pragma unroll
    for (int c = 0; c < 2; ++c)
      umma::bulk_g2s(Fs + (c * G::W + fa - gi0) * G::NH, Fb + ((size_t)c * N + fa) * G::NH, bytes, &X.bar);
  }
  for (int r = threadIdx.x; r < G::W; r += blockDim.x) {
    const int gi = gi0 + r;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f), p0 = z, p1 = z, p2 = z, p3 = z;
    if (gi >= 0 && gi < N) {
      const size_t row = (size_t)gi * N;
      const float aS = coef[gi], aN = coef[N + gi], bh = coef[2 * N + gi], id = invd[row + 1], ide = invd[row];
      p0 = make_float4(aS, aS, aN, aN);
      p1 = make_float4(bh, bh, id, id);
      p2 = make_float4(ide, id, id, ide);
      p3 = make_float4(diag[row + 1], diag[row], coef[3 * N + gi], 0.f);
    }
    X.rq[4 * r] = p0;
    X.rq[4 * r + 1] = p1;
    X.rq[4 * r + 2] = p2;
    X.rq[4 * r + 3] = p3;
  }
  const int nlo = fa - gi0, nhi = gi0 + G::W - fb;
  for (int e = threadIdx.x; e < (nlo + nhi) * G::NH; e += blockDim.x) {
    const int rr = e / G::NH, k = e - rr * G::NH;
    const int r = rr < nlo ? rr : fb - gi0 + (rr - nlo);
    Fs[r * G::NH + k] = 0.f;
    Fs[(G::W + r) * G::NH + k] = 0.f;
  }
}

template <int N, int HALO, int NV>
__device__ __forceinline__ void o_load(OState<N, HALO, NV>& S, const float* __restrict__ Ub, int g0, int o) {
  using G = OBand<N, HALO, NV>;
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int gi = g0 + r;
    if (Ub) {
      const float* ev = Ub + uidx(N, gi, 8 * o);       // even columns 8o, 8o + 2, 8o + 4, 8o + 6
      const float* od = Ub + uidx(N, gi, 8 * o + 1);   // odd columns
      S.A0[r] = f2(ev[0], ev[1]);
      S.A1[r] = f2(ev[2], ev[3]);
      S.B0[r] = f2(od[0], od[1]);
      S.B1[r] = f2(od[2], od[3]);
    } else {
      S.A0[r] = S.A1[r] = S.B0[r] = S.B1[r] = f2(0.f, 0.f);
    }
  }
}

template <int N, int HALO, int NV>
__device__ __forceinline__ void o_store(const OState<N, HALO, NV>& S, float* __restrict__ Ub, int gi0, int v, int o) {
  using G = OBand<N, HALO, NV>;
  const int rb = v * G::H;
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r;
    if (rg < HALO || rg >= HALO + G::BR) continue;
    float* ev = Ub + uidx(N, gi0 + rg, 8 * o);
    float* od = Ub + uidx(N, gi0 + rg, 8 * o + 1);
    ev[0] = S.A0[r].x; ev[1] = S.A0[r].y; ev[2] = S.A1[r].x; ev[3] = S.A1[r].y;
    od[0] = S.B0[r].x; od[1] = S.B0[r].y; od[2] = S.B1[r].x; od[3] = S.B1[r].y;
  }
}

template <int N, int HALO, int NV>
__device__ __forceinline__ void o_publish_all(const OState<N, HALO, NV>& S, OShared<N, HALO, NV>& X, int v, int o) {
  using G = OBand<N, HALO, NV>;
  X.TA[v][o] = pk4(S.A0[0], S.A1[0]);
  X.TB[v][o] = pk4(S.B0[0], S.B1[0]);
  X.BA[v + 1][o] = pk4(S.A0[G::H - 1], S.A1[G::H - 1]);
  X.BB[v + 1][o] = pk4(S.B0[G::H - 1], S.B1[G::H - 1]);
  if (v == 0) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    X.TA[NV][o] = X.TB[NV][o] = X.BA[0][o] = X.BB[0][o] = z;
  }
}

// one half-sweep of colour C over the thread's rows (rb = v H even)
template <int N, int HALO, int NV, int C>
__device__ __forceinline__ void o_half_sweep(OState<N, HALO, NV>& S, OShared<N, HALO, NV>& X,
                                             const float* __restrict__ Fs, int v, int o) {
  using G = OBand<N, HALO, NV>;
  const int rb = v * G::H;
  const bool first = o == 0, last = o == G::NO - 1;
  const float* Fr = Fs + (C * G::W + rb) * G::NH + 4 * o;
  const float4* R = X.rq + 4 * rb;
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const float4 p0 = R[4 * r], p1 = R[4 * r + 1];
    const float2 idi = f2(p1.z, p1.w);
    const float4 F = *reinterpret_cast<const float4*>(Fr + r * G::NH);
    const float2 qS = f2(p0.x, p0.y), qN = f2(p0.z, p0.w), qB = f2(p1.x, p1.y);
    if (((r + HALO) & 1) == C) {
      // A0 = (8o, 8o + 2): west 8o - 1 (lane o - 1's B1.y) and B0.x, east B0.x and B0.y;
      // A1 = (8o + 4, 8o + 6): west B0.y and B1.x, east B1.x and B1.y
      float w = __shfl_up_sync(0xffffffffu, S.B1[r].y, 1, G::WID);
      if (first) w = 0.f;
      const float4 nN = r > 0 ? pk4(S.A0[r - 1], S.A1[r - 1]) : X.BA[v][o];
      const float4 nS = r + 1 < G::H ? pk4(S.A0[r + 1], S.A1[r + 1]) : X.TA[v + 1][o];
      const float2 id0 = first ? f2(R[4 * r + 2].x, R[4 * r + 2].y) : idi;
      const float2 s0 = __fadd2_rn(S.B0[r], f2(w, S.B0[r].x));
      const float2 s1 = __fadd2_rn(S.B1[r], f2(S.B0[r].y, S.B1[r].x));
      const float2 t0 = __ffma2_rn(qB, s0, __ffma2_rn(qN, lo2(nN), __ffma2_rn(qS, lo2(nS), neg2(lo2(F)))));
      const float2 t1 = __ffma2_rn(qB, s1, __ffma2_rn(qN, hi2(nN), __ffma2_rn(qS, hi2(nS), neg2(hi2(F)))));
      S.A0[r] = __fmul2_rn(t0, id0);
      S.A1[r] = __fmul2_rn(t1, idi);
      if (r == 0) X.TA[v][o] = pk4(S.A0[r], S.A1[r]);
      if (r == G::H - 1) X.BA[v + 1][o] = pk4(S.A0[r], S.A1[r]);
    } else {
      // B0 = (8o + 1, 8o + 3): west A0.x and A0.y, east A0.y and A1.x;
      // B1 = (8o + 5, 8o + 7): west A1.x and A1.y, east A1.y and 8o + 8 (lane o + 1's A0.x)
      float e = __shfl_down_sync(0xffffffffu, S.A0[r].x, 1, G::WID);
      if (last) e = 0.f;
      const float4 nN = r > 0 ? pk4(S.B0[r - 1], S.B1[r - 1]) : X.BB[v][o];
      const float4 nS = r + 1 < G::H ? pk4(S.B0[r + 1], S.B1[r + 1]) : X.TB[v + 1][o];
      const float2 id1 = last ? f2(R[4 * r + 2].z, R[4 * r + 2].w) : idi;
      const float2 s0 = __fadd2_rn(S.A0[r], f2(S.A0[r].y, S.A1[r].x));
      const float2 s1 = __fadd2_rn(S.A1[r], f2(S.A1[r].y, e));
      const float2 t0 = __ffma2_rn(qB, s0, __ffma2_rn(qN, lo2(nN), __ffma2_rn(qS, lo2(nS), neg2(lo2(F)))));
      const float2 t1 = __ffma2_rn(qB, s1, __ffma2_rn(qN, hi2(nN), __ffma2_rn(qS, hi2(nS), neg2(hi2(F)))));
      S.B0[r] = __fmul2_rn(t0, idi);
      S.B1[r] = __fmul2_rn(t1, id1);
      if (r == 0) X.TB[v][o] = pk4(S.B0[r], S.B1[r]);
      if (r == G::H - 1) X.BB[v + 1][o] = pk4(S.B0[r], S.B1[r]);
    }
  }
}

template <int N, int HALO, int NV>
__device__ __forceinline__ void o_sweeps(OState<N, HALO, NV>& S, OShared<N, HALO, NV>& X, const float* __restrict__ Fs,
                                         int v, int o) {
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    o_half_sweep<N, HALO, NV, 0>(S, X, Fs, v, o);
    __syncthreads();
    o_half_sweep<N, HALO, NV, 1>(S, X, Fs, v, o);
    __syncthreads();
  }
}

template <int N, int NV>
__global__ void __launch_bounds__(OBand<N, kSRHalo, NV>::NT) k_oct_smooth_restrict(
    const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ f,
    const float* __restrict__ coef, const float* __restrict__ invd, const float* __restrict__ diag,
    const float* __restrict__ rden, float* __restrict__ fc, int* d_err) {
  constexpr int HALO = kSRHalo;
  using G = OBand<N, HALO, NV>;
  extern __shared__ __align__(128) unsigned char smem_osr[];
  float* Fs = reinterpret_cast<float*>(smem_osr);
  __shared__ OShared<N, HALO, NV> X;
  const size_t b = blockIdx.z;
  const int gi0 = blockIdx.x * G::BR - HALO;
  const int v = threadIdx.x / G::NO, o = threadIdx.x % G::NO;
  const int rb = v * G::H;
  const bool first = o == 0, last = o == G::NO - 1;
  o_begin<N, HALO, NV>(X, Fs, f + b * N * N, gi0, coef, invd, diag, 0);
  OState<N, HALO, NV> S;
  o_load<N, HALO, NV>(S, u_in ? u_in + b * upatch(N) : nullptr, gi0 + rb, o);
  o_publish_all<N, HALO, NV>(S, X, v, o);
  if (!band_wait(&X.bar, d_err)) return;
  o_sweeps<N, HALO, NV>(S, X, Fs, v, o);
  o_store<N, HALO, NV>(S, u_out + b * upatch(N), gi0, v, o);
  // red residuals of the band rows, written over their sources
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r;
    if (rg < HALO || rg >= HALO + G::BR) continue;
    const float4 p0 = X.rq[4 * rg], p1 = X.rq[4 * rg + 1], p3 = X.rq[4 * rg + 3];
    const float2 qS = f2(p0.x, p0.y), qN = f2(p0.z, p0.w), qB = f2(p1.x, p1.y), dgi = f2(p3.x, p3.x);
    float4* Fr = reinterpret_cast<float4*>(Fs + rg * G::NH + 4 * o);
    float2 nb0, nb1;
    if (((r + HALO) & 1) == 0) {   // red pairs A0, A1
      float w = __shfl_up_sync(0xffffffffu, S.B1[r].y, 1, G::WID);
      if (first) w = 0.f;
      const float4 nN = r > 0 ? pk4(S.A0[r - 1], S.A1[r - 1]) : X.BA[v][o];
      const float4 nS = r + 1 < G::H ? pk4(S.A0[r + 1], S.A1[r + 1]) : X.TA[v + 1][o];
      const float2 d0 = f2(first ? p3.y : p3.x, p3.x);
      nb0 = __ffma2_rn(qB, __fadd2_rn(S.B0[r], f2(w, S.B0[r].x)),
                       __ffma2_rn(qN, lo2(nN), __ffma2_rn(qS, lo2(nS), __fmul2_rn(neg2(d0), S.A0[r]))));
      nb1 = __ffma2_rn(qB, __fadd2_rn(S.B1[r], f2(S.B0[r].y, S.B1[r].x)),
                       __ffma2_rn(qN, hi2(nN), __ffma2_rn(qS, hi2(nS), __fmul2_rn(neg2(dgi), S.A1[r]))));
    } else {                        // red pairs B0, B1
      float e = __shfl_down_sync(0xffffffffu, S.A0[r].x, 1, G::WID);
      if (last) e = 0.f;
      const float4 nN = r > 0 ? pk4(S.B0[r - 1], S.B1[r - 1]) : X.BB[v][o];
      const float4 nS = r + 1 < G::H ? pk4(S.B0[r + 1], S.B1[r + 1]) : X.TB[v + 1][o];
      const float2 d1 = f2(p3.x, last ? p3.y : p3.x);
      nb0 = __ffma2_rn(qB, __fadd2_rn(S.A0[r], f2(S.A0[r].y, S.A1[r].x)),
                       __ffma2_rn(qN, lo2(nN), __ffma2_rn(qS, lo2(nS), __fmul2_rn(neg2(dgi), S.B0[r]))));
      nb1 = __ffma2_rn(qB, __fadd2_rn(S.A1[r], f2(S.A1[r].y, e)),
                       __ffma2_rn(qN, hi2(nN), __ffma2_rn(qS, hi2(nS), __fmul2_rn(neg2(d1), S.B1[r]))));
    }
    const float4 Fv = *Fr;
    const float2 z = f2(0.f, 0.f);
    *Fr = pk4(__fadd2_rn(z, __fadd2_rn(lo2(Fv), neg2(nb0))), __fadd2_rn(z, __fadd2_rn(hi2(Fv), neg2(nb1))));
  }
  __syncthreads();
  // restriction: coarse cells (I, 4o .. 4o + 3)
  constexpr int NC = G::NC;
  float* fcb = fc + b * NC * NC;
  for (int Il = v; Il < G::BR / 2; Il += NV) {
    const int rg = HALO + 2 * Il, I = (gi0 + rg) >> 1;
    const float a0 = X.rq[4 * rg + 3].z, a1 = X.rq[4 * rg + 7].z;
    const float4 rs0 = *reinterpret_cast<const float4*>(Fs + rg * G::NH + 4 * o);
    const float4 rs1 = *reinterpret_cast<const float4*>(Fs + (rg + 1) * G::NH + 4 * o);
    const float2 z = f2(0.f, 0.f), A0v = f2(a0, a0), A1v = f2(a1, a1);
    const float rd = rden[I];
    const float2 outl = __fmul2_rn(__ffma2_rn(A1v, lo2(rs1), __ffma2_rn(A0v, lo2(rs0), z)), f2(rd, rd));
    const float2 outh = __fmul2_rn(__ffma2_rn(A1v, hi2(rs1), __ffma2_rn(A0v, hi2(rs0), z)), f2(rd, rd));
    // coarse columns 4o, 4o + 2 in colour plane I & 1, 4o + 1, 4o + 3 in the other (entries 2o, 2o + 1)
    *reinterpret_cast<float2*>(fcb + fidx(NC, I, 4 * o)) = f2(outl.x, outh.x);
    *reinterpret_cast<float2*>(fcb + fidx(NC, I, 4 * o + 1)) = f2(outl.y, outh.y);
  }
}

template <int N, int NV>
__global__ void __launch_bounds__(OBand<N, 4, NV>::NT) k_oct_prolong_smooth(
    const float* __restrict__ u_in, float* __restrict__ u_out, const float* __restrict__ f,
    const float* __restrict__ coef, const float* __restrict__ invd, const float* __restrict__ diag,
    const float* __restrict__ uc, int* d_err) {
  constexpr int HALO = 4;
  using G = OBand<N, HALO, NV>;
  constexpr int NC = G::NC, Wc = G::Wc, Pc = G::Pc;
  extern __shared__ __align__(128) unsigned char smem_ops[];
  float* Fs = reinterpret_cast<float*>(smem_ops);
  float* E = Fs + 2 * G::W * G::NH;
  __shared__ OShared<N, HALO, NV> X;
  const size_t b = blockIdx.z;
  const int gi0 = blockIdx.x * G::BR - HALO;
  const int v = threadIdx.x / G::NO, o = threadIdx.x % G::NO;
  const int rb = v * G::H;
  const uint32_t cbytes = (uint32_t)(Wc * Pc * sizeof(float));
  o_begin<N, HALO, NV>(X, Fs, f + b * N * N, gi0, coef, invd, diag, 2 * cbytes);
  if (threadIdx.x == 0) {
    const float* Cc = uc + b * upatch(NC) + (size_t)((gi0 >> 1) - 1 + 1 + kUHalo) * Pc;
#pragma unroll
    for (int c = 0; c < 2; ++c) umma::bulk_g2s(E + c * Wc * Pc, Cc + c * uplane_of(NC), cbytes, &X.bar);
  }
  OState<N, HALO, NV> S;
  o_load<N, HALO, NV>(S, u_in + b * upatch(N), gi0 + rb, o);
  if (!band_wait(&X.bar, d_err)) return;
  // black cells += P(e_c): the A pairs of odd rows (coarse columns 4o .. 4o + 3, outer
  // neighbours 4o - 1 .. 4o + 2), the B pairs of even rows (outer neighbours 4o + 1 .. 4o + 4)
  const float2 nine = f2(9.f, 9.f), three = f2(3.f, 3.f), sixteenth = f2(0.0625f, 0.0625f);
#pragma unroll
  for (int r = 0; r < G::H; ++r) {
    const int rg = rb + r, gi = gi0 + rg;
    if ((unsigned)gi >= (unsigned)N) continue;
    const bool rowedge = gi == 0 || gi == N - 1;
    const int a = (rg >> 1) + 1, da = (r & 1) ? a + 1 : a - 1;
    const int pa = (a + (gi0 >> 1) + 1) & 1, pd = pa ^ 1;
    // entry 2o + j of the row's even / odd coarse columns: columns 4o - 2 + 2j / 4o - 1 + 2j
    const float* Ea0 = E + (pa * Wc + a) * Pc + 2 * o;
    const float* Ea1 = E + ((pa ^ 1) * Wc + a) * Pc + 2 * o;
    const float* Ed0 = E + (pd * Wc + da) * Pc + 2 * o;
    const float* Ed1 = E + ((pd ^ 1) * Wc + da) * Pc + 2 * o;
    // coarse columns 4o, 4o + 1 (pair 0) and 4o + 2, 4o + 3 (pair 1)
    const float2 e0 = f2(Ea0[1], Ea1[1]), e1 = f2(Ea0[2], Ea1[2]);
    const float2 d0 = f2(Ed0[1], Ed1[1]), d1 = f2(Ed0[2], Ed1[2]);
    if (r & 1) {   // odd row: A0 (4o, 4o + 1), A1 (4o + 2, 4o + 3); neighbours J - 1
      const float2 c0 = __fmul2_rn(__ffma2_rn(nine, e0, __ffma2_rn(three, __fadd2_rn(d0, f2(Ea1[0], Ea0[1])), f2(Ed1[0], Ed0[1]))), sixteenth);
      const float2 c1 = __fmul2_rn(__ffma2_rn(nine, e1, __ffma2_rn(three, __fadd2_rn(d1, f2(Ea1[1], Ea0[2])), f2(Ed1[1], Ed0[2]))), sixteenth);
      S.A0[r] = __fadd2_rn(S.A0[r], f2((rowedge || o == 0) ? e0.x : c0.x, rowedge ? e0.y : c0.y));
      S.A1[r] = __fadd2_rn(S.A1[r], f2(rowedge ? e1.x : c1.x, rowedge ? e1.y : c1.y));
    } else {       // even row: B0, B1; neighbours J + 1
      const float2 c0 = __fmul2_rn(__ffma2_rn(nine, e0, __ffma2_rn(three, __fadd2_rn(d0, f2(Ea1[1], Ea0[2])), f2(Ed1[1], Ed0[2]))), sixteenth);
      const float2 c1 = __fmul2_rn(__ffma2_rn(nine, e1, __ffma2_rn(three, __fadd2_rn(d1, f2(Ea1[2], Ea0[3])), f2(Ed1[2], Ed0[3]))), sixteenth);
      S.B0[r] = __fadd2_rn(S.B0[r], f2(rowedge ? e0.x : c0.x, rowedge ? e0.y : c0.y));
      S.B1[r] = __fadd2_rn(S.B1[r], f2(rowedge ? e1.x : c1.x, (rowedge || o == G::NO - 1) ? e1.y : c1.y));
    }
  }
  o_publish_all<N, HALO, NV>(S, X, v, o);
  __syncthreads();
  o_sweeps<N, HALO, NV>(S, X, Fs, v, o);
  o_store<N, HALO, NV>(S, u_out + b * upatch(N), gi0, v, o);
}

// ---------------------------------------------------------------------------
// The coarse end of a V-cycle in one launch: the levels of at most kSubMax
// cells a side, from a level's pre-smoothing down to the exact solve of the
// 8 x 8 coarsest level and back up through every prolongation and
// post-smoothing, one CTA per patch with every level's correction, source
// and row coefficients in shared memory.  The separate band kernels spend
// most of their time on launch and memory latency at these sizes; here only
// the top level's source (in) and correction (out) cross HBM.  Each sweep,
// restriction and prolongation is that of the band kernels, operation for
// operation.  The coarsest solve is the dense inverse applied in FP64 for
// FP64 V-cycles and in FP32 for the FP32 ones (four lanes per row, partial
// sums added by shuffles; its rounding is that of the FP32 cycle around it).
// Corrections are dense (n + 2)^2 arrays with a zero ghost ring, sources
// dense n^2.  (At 64 cells a side the whole-patch arrays leave room for too
// few CTAs per SM: that level stays with the band kernels.)
constexpr int kSubMax = 32, kSubThreads = 256, kSubCoarse = 8;

template <typename T>
struct SubLev {
  const T* coef;   // [4 n]: aS, aN, b, area per row
  const T* invd;   // [n n]: 1 / diagonal (column 0: edge cells, 1: interior)
  const T* diag;
  const T* rden;   // [n / 2]
};

template <typename T>
struct SubArgs {
  SubLev<T> lev[4];     // levels n0, n0 / 2, .. down to 16 (the 8 x 8 level needs none)
  int nu1, nu2;
  const double* minv;   // the 8 x 8 level's dense inverse [64][64]
  const float* minv32;  // the same in FP32
};

// row coefficients of a level in shared memory: aS, aN, b, area, 1/d (edge,
// interior), d (edge, interior) per row, rden per coarse row
template <typename T, int N>
struct SubRows {
  T aS[N], aN[N], bh[N], area[N], ide[N], idi[N], dge[N], dgi[N], rden[N / 2];
};

template <typename T, int N>
__device__ __forceinline__ void sub_stage_rows(SubRows<T, N>& R, const SubLev<T>& L) {
  for (int i = threadIdx.x; i < N; i += kSubThreads) {
    R.aS[i] = L.coef[i];
    R.aN[i] = L.coef[N + i];
    R.bh[i] = L.coef[2 * N + i];
    R.area[i] = L.coef[3 * N + i];
    R.ide[i] = L.invd[i * N];
    R.idi[i] = L.invd[i * N + 1];
    R.dge[i] = L.diag[i * N];
    R.dgi[i] = L.diag[i * N + 1];
    if (i < N / 2) R.rden[i] = L.rden[i];
  }
}

template <typename T, int N>
__device__ __forceinline__ void sub_half_sweep(T* __restrict__ u, const T* __restrict__ f, const SubRows<T, N>& R,
                                               int colour) {
  constexpr int P = N + 2, NH = N / 2, CELLS = N * NH;
#pragma unroll
  for (int t0 = 0; t0 < CELLS; t0 += kSubThreads) {
    const int t = t0 + threadIdx.x;
    if (CELLS % kSubThreads != 0 && t >= CELLS) break;
    const int i = t / NH, j = 2 * (t % NH) + ((i + colour) & 1);
    T* c = u + (i + 1) * P + (j + 1);
    const T id = (j == 0 || j == N - 1) ? R.ide[i] : R.idi[i];
    const T v = fma(R.bh[i], c[1] + c[-1], fma(R.aN[i], c[-P], fma(R.aS[i], c[P], -f[i * N + j])));
    *c = v * id;
  }
  __syncthreads();
}

// red-child residuals of level N restricted into the level N / 2 source
template <typename T, int N>
__device__ __forceinline__ void sub_restrict(const T* __restrict__ u, const T* __restrict__ f,
                                             const SubRows<T, N>& R, T* __restrict__ fc) {
  constexpr int P = N + 2, NC = N / 2;
#pragma unroll
  for (int t0 = 0; t0 < NC * NC; t0 += kSubThreads) {
    const int t = t0 + threadIdx.x;
    if ((NC * NC) % kSubThreads != 0 && t >= NC * NC) break;
    const int I = t / NC, J = t % NC, i0 = 2 * I, i1 = i0 + 1;
    const T* r0 = u + (i0 + 1) * P + (2 * J + 1);   // (2I, 2J)
    const T* r1 = r0 + P;                           // (2I + 1, 2J)
    const T a0 = r0[0], a1 = r0[1], w = r0[-1], n0v = r0[-P], b0 = r1[0], b1 = r1[1], e = r1[2], s1 = r1[P + 1];
    const T d0 = J == 0 ? R.dge[i0] : R.dgi[i0];
    const T d1 = J == NC - 1 ? R.dge[i1] : R.dgi[i1];
    const T nb0 = fma(R.bh[i0], a1 + w, fma(R.aN[i0], n0v, fma(R.aS[i0], b0, -d0 * a0)));
    const T nb1 = fma(R.bh[i1], e + b0, fma(R.aN[i1], a1, fma(R.aS[i1], s1, -d1 * b1)));
    T rs0 = 0, rs1 = 0;
    rs0 += f[i0 * N + 2 * J] - nb0;
    rs1 += f[i1 * N + 2 * J + 1] - nb1;
    T nr = 0;
    nr = fma(R.area[i0], rs0, nr);
    nr = fma(R.area[i1], rs1, nr);
    fc[I * NC + J] = nr * R.rden[I];
  }
  __syncthreads();
}

// u += P(e_c) on the black cells of level N (every cell without post-smoothing)
template <typename T, int N>
__device__ __forceinline__ void sub_prolong(T* __restrict__ u, const T* __restrict__ E, bool black_only) {
  constexpr int P = N + 2, NC = N / 2, Pc = NC + 2;
#pragma unroll
  for (int t0 = 0; t0 < N * N; t0 += kSubThreads) {
    const int t = t0 + threadIdx.x;
    if ((N * N) % kSubThreads != 0 && t >= N * N) break;
    const int i = t / N, j = t % N;
    if (black_only && !((i + j) & 1)) continue;
    const int I = i >> 1, Id = (i & 1) ? I + 1 : I - 1, J = j >> 1;
    const bool rowedge = i == 0 || i == N - 1;
    const T* Ea = E + (I + 1) * Pc + (J + 1);
    const T* Ed = E + (Id + 1) * Pc + (J + 1);
    const T e11 = Ea[0], d11 = Ed[0];
    T c;
    if (!(j & 1)) c = (rowedge || J == 0) ? e11 : fma((T)9, e11, fma((T)3, d11 + Ea[-1], Ed[-1])) * (T)0.0625;
    else c = (rowedge || J == NC - 1) ? e11 : fma((T)9, e11, fma((T)3, d11 + Ea[1], Ed[1])) * (T)0.0625;
    u[(i + 1) * P + (j + 1)] += c;
  }
  __syncthreads();
}

template <typename T, int N>
struct SubLevel {
  T u[(N + 2) * (N + 2)];
  T f[N * N];
  SubRows<T, N> R;
};

// shared memory of the levels N .. 16 and the 8 x 8 level
template <typename T, int N>
struct SubStack {
  SubLevel<T, N> top;
  SubStack<T, N / 2> rest;
};
template <typename T>
struct SubStack<T, kSubCoarse> {
  T u[(kSubCoarse + 2) * (kSubCoarse + 2)];
  T f[kSubCoarse * kSubCoarse];
  double rhs[kSubCoarse * kSubCoarse];
};

template <typename T, int N>
__device__ __forceinline__ void sub_zero(SubStack<T, N>& S) {
  if constexpr (N == kSubCoarse) {
    for (int t = threadIdx.x; t < (N + 2) * (N + 2); t += kSubThreads) S.u[t] = (T)0;
  } else {
    for (int t = threadIdx.x; t < (N + 2) * (N + 2); t += kSubThreads) S.top.u[t] = (T)0;
    sub_zero<T, N / 2>(S.rest);
  }
}

template <typename T, int N>
__device__ __forceinline__ void sub_stage(SubStack<T, N>& S, const SubArgs<T>& a, int k) {
  if constexpr (N != kSubCoarse) {
    sub_stage_rows<T, N>(S.top.R, a.lev[k]);
    sub_stage<T, N / 2>(S.rest, a, k + 1);
  }
}

// one V-cycle from level N on the source already in S.top.f (coarser levels from zero)
template <typename T, int N>
__device__ __forceinline__ void sub_cycle(SubStack<T, N>& S, const SubArgs<T>& a) {
  if constexpr (N == kSubCoarse) {
    constexpr int nn = N * N;
    if constexpr (sizeof(T) == 4) {
      static_assert(kSubThreads == 4 * nn, "four lanes per row of the coarsest inverse");
      const int t = threadIdx.x >> 2, part = threadIdx.x & 3;
      const float* m = a.minv32 + (size_t)t * nn + part * (nn / 4);
      const T* fv = S.f + part * (nn / 4);
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < nn / 4; ++q) acc = fmaf(m[q], fv[q], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (part == 0) S.u[(t / N + 1) * (N + 2) + (t % N + 1)] = acc;
    } else {
      for (int t = threadIdx.x; t < nn; t += kSubThreads) S.rhs[t] = (double)S.f[t];
      __syncthreads();
      for (int t = threadIdx.x; t < nn; t += kSubThreads) {
        double acc = 0.0;
        for (int q = 0; q < nn; ++q) acc += a.minv[(size_t)t * nn + q] * S.rhs[q];
        S.u[(t / N + 1) * (N + 2) + (t % N + 1)] = (T)acc;
      }
    }
    __syncthreads();
  } else {
    auto& L = S.top;
    for (int s = 0; s < a.nu1; ++s) {
      sub_half_sweep<T, N>(L.u, L.f, L.R, 0);
      sub_half_sweep<T, N>(L.u, L.f, L.R, 1);
    }
    if constexpr (N / 2 == kSubCoarse) sub_restrict<T, N>(L.u, L.f, L.R, S.rest.f);
    else sub_restrict<T, N>(L.u, L.f, L.R, S.rest.top.f);
    sub_cycle<T, N / 2>(S.rest, a);
    if constexpr (N / 2 == kSubCoarse) sub_prolong<T, N>(L.u, S.rest.u, a.nu2 > 0);
    else sub_prolong<T, N>(L.u, S.rest.top.u, a.nu2 > 0);
    for (int s = 0; s < a.nu2; ++s) {
      sub_half_sweep<T, N>(L.u, L.f, L.R, 0);
      sub_half_sweep<T, N>(L.u, L.f, L.R, 1);
    }
  }
}

template <typename T, int N0>
__global__ void __launch_bounds__(kSubThreads) k_sub_vcycle(T* __restrict__ ug, const T* __restrict__ fg, int zero,
                                                            SubArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_sub[];
  SubStack<T, N0>& S = *reinterpret_cast<SubStack<T, N0>*>(smem_sub);
  const size_t b = blockIdx.x;
  sub_zero<T, N0>(S);
  sub_stage<T, N0>(S, a, 0);
  __syncthreads();
  for (int t = threadIdx.x; t < N0 * N0; t += kSubThreads) {
    const int i = t / N0, j = t % N0;
    S.top.f[t] = fg[b * N0 * N0 + fidx(N0, i, j)];
    if (!zero) S.top.u[(i + 1) * (N0 + 2) + (j + 1)] = ug[b * upatch(N0) + uidx(N0, i, j)];
  }
  __syncthreads();
  sub_cycle<T, N0>(S, a);
  for (int t = threadIdx.x; t < N0 * N0; t += kSubThreads) {
    const int i = t / N0, j = t % N0;
    ug[b * upatch(N0) + uidx(N0, i, j)] = S.top.u[(i + 1) * (N0 + 2) + (j + 1)];
  }
}

// Exact solve of the coarsest level (nc^2 <= 256 unknowns), one CTA per patch:
// u = Minv (f - ghost contributions), in FP64.
template <typename T>
__global__ void k_coarse_solve(T* __restrict__ u, const T* __restrict__ f, const double* __restrict__ coef,
                               const double* __restrict__ minv, int nc) {
  extern __shared__ double rhs[];
  const size_t b = blockIdx.x;
  const int nn = nc * nc;
  T* U = u + b * upatch(nc);
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = t / nc, j = t % nc;
    double g = 0.0;
    if (i == nc - 1) g += coef[i] * (double)U[uidx(nc, i + 1, j)];
    if (i == 0) g += coef[nc + i] * (double)U[uidx(nc, i - 1, j)];
    if (j == nc - 1) g += coef[2 * nc + i] * (double)U[uidx(nc, i, j + 1)];
    if (j == 0) g += coef[2 * nc + i] * (double)U[uidx(nc, i, j - 1)];
    rhs[t] = (double)f[b * nn + fidx(nc, i, j)] - g;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nn; ++k) acc += minv[(size_t)t * nn + k] * rhs[k];
    U[uidx(nc, t / nc, t % nc)] = (T)acc;
  }
}

// ||f' - L e||^2 per patch (f' the defect source, e the correction)
template <typename T>
__global__ void k_resnorm(const T* __restrict__ u, const T* __restrict__ f, const double* __restrict__ coef,
                          const double* __restrict__ diag, int n, double* __restrict__ norms) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  double rr = 0.0;
  if (i < n && j < n) {
    const T* U = u + (size_t)b * upatch(n);
    const double nb = coef[i] * (double)U[uidx(n, i + 1, j)] + coef[n + i] * (double)U[uidx(n, i - 1, j)] +
                      coef[2 * n + i] * ((double)U[uidx(n, i, j + 1)] + (double)U[uidx(n, i, j - 1)]);
    const double r = (double)f[(size_t)b * n * n + fidx(n, i, j)] - (nb - (double)U[uidx(n, i, j)] * diag[i * n + j]);
    rr = r * r;
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (threadIdx.x == 0 && rr != 0.0) atomicAdd(norms + b, rr);
}

// Block maximum of non-negative doubles (NaN ignored, as fmax does) folded
// into *out, which starts at 0: non-negative doubles order like their bits.
__device__ __forceinline__ void block_max_into(double mx, double* out) {
  __shared__ double s[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0 && mx > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(mx));
  }
}

// max over patches of ||r|| / ||f|| (one patch per thread, *out zeroed first)
__global__ void k_max_ratio(const double* __restrict__ rr, const double* __restrict__ ff, int npatch,
                            double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (b < npatch) {
    const double fn = sqrt(ff[b]);
    mx = fmax(mx, sqrt(rr[b]) / (fn > 0 ? fn : 1.0));
  }
  block_max_into(mx, out);
}

// Mixed refinement step, fused: e_new = e_old + d (d = the last FP32
// V-cycle's correction, NULL before the first cycle), r = f' - L e_new with
// e, f' and the operator in float-float (FP64-level accuracy on the FP32
// pipe), r rounded to FP32 as the next V-cycle's source, ||r||^2 per patch.
// e is kept in the layout of the correction arrays (colour-split rows).  A
// thread takes the cells (i, 2k) and (i, 2k + 1), which sit at the same
// entry of the two colour rows of row i, and walks kWalk rows of that column
// pair: every e + d is formed once, kept for the rows above and below in
// registers, and handed to the horizontal neighbours by warp shuffles; the
// sums use ff_add_lite.  Every load and store of a warp is contiguous.
constexpr int kWalk = 32;

__global__ void __launch_bounds__(kBX * kBY) k_resid_ff_walk(const float2* __restrict__ e_old,
                                                              const float* __restrict__ d,
                                                              const float2* __restrict__ fd,
                                                              const float2* __restrict__ coef,
                                                              const float2* __restrict__ diag, int n,
                                                              float2* __restrict__ e_new, float* __restrict__ r32,
                                                              double* __restrict__ norms) {
  const int b = blockIdx.z, nh = n >> 1;
  const int k = blockIdx.x * kBX + threadIdx.x;
  const int lane = threadIdx.x;
  const bool live = k < nh;
  const size_t pb = (size_t)b * upatch(n), pl = uplane_of(n), P = upitch(n);
  const float2* E = e_old + pb;
  const float* D = d ? d + pb : nullptr;
  auto ld = [&](int i, int col, int entry) -> float2 {   // e + d at colour `col`, row i, entry
    const size_t o = (size_t)col * pl + (size_t)(i + 1 + kUHalo) * P + entry;
    float2 v = E[o];
    if (D) v = ff_add_f(v, D[o]);
    return v;
  };
  const int i0 = (blockIdx.y * kBY + threadIdx.y) * kWalk;
  if (i0 >= n) return;   // whole warps: every lane of the warp has the same rows
  const int i1 = min(n, i0 + kWalk);
  // cells (i, 2k) and (i, 2k + 1): entry k + 1 of colours i & 1 and (i + 1) & 1
  float2 pa{0.f, 0.f}, pbv{0.f, 0.f}, ca{0.f, 0.f}, cbv{0.f, 0.f};
  if (live) {
    pa = ld(i0 - 1, (i0 - 1) & 1, k + 1);
    pbv = ld(i0 - 1, i0 & 1, k + 1);
    ca = ld(i0, i0 & 1, k + 1);
    cbv = ld(i0, (i0 + 1) & 1, k + 1);
  }
  float rr = 0.f;
  for (int i = i0; i < i1; ++i) {
    float2 sa{0.f, 0.f}, sb{0.f, 0.f};
    if (live) {
      sa = ld(i + 1, (i + 1) & 1, k + 1);
      sb = ld(i + 1, i & 1, k + 1);
    }
    // horizontal neighbours (i, 2k - 1) = lane - 1's second cell, (i, 2k + 2) = lane + 1's first
    float2 w, e;
    w.x = __shfl_up_sync(0xffffffffu, cbv.x, 1);
    w.y = __shfl_up_sync(0xffffffffu, cbv.y, 1);
    e.x = __shfl_down_sync(0xffffffffu, ca.x, 1);
    e.y = __shfl_down_sync(0xffffffffu, ca.y, 1);
    if (live) {
      if (lane == 0) w = ld(i, (i + 1) & 1, k);          // entry k: column 2k - 1 (0 at the ghost ring)
      if (lane == kBX - 1 || k == nh - 1) e = ld(i, i & 1, k + 2);
      const float2 cS = coef[i], cN = coef[n + i], cB = coef[2 * n + i];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * k + h;
        const float2 eC = h ? cbv : ca, eS = h ? sb : sa, eN = h ? pbv : pa;
        const float2 eE = h ? e : cbv, eW = h ? ca : w;
        const float2 nb = ff_add_lite(ff_add_lite(ff_mul(cS, eS), ff_mul(cN, eN)),
                                      ff_add_lite(ff_mul(cB, ff_add_lite(eE, eW)), ff_neg(ff_mul(diag[i * n + j], eC))));
        const size_t pos = (size_t)b * n * n + fidx(n, i, j);
        const float2 r = ff_add_lite(fd[pos], ff_neg(nb));
        r32[pos] = r.x + r.y;
        e_new[pb + (size_t)((i + h) & 1) * pl + (size_t)(i + 1 + kUHalo) * P + (k + 1)] = eC;
        rr = fmaf(r.x, r.x, rr);
      }
    }
    pa = ca;
    pbv = cbv;
    ca = sa;
    cbv = sb;
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (lane == 0 && rr != 0.f) atomicAdd(norms + b, (double)rr);
}

// First residual of a mixed solve, where e = 0: r = f' (the float-float
// defect; with the operator's terms all zero the walk above returns its
// renormalised sum), the FP32 source fl(hi + lo) and ||r||^2 per patch,
// without the stencil: f' and the source are the patches' contiguous arrays
// (same cell order), read and written as one stream.  e stays zero.
constexpr int kFirstThreads = 256, kFirstPer = 16;   // cells per thread and block pass
__global__ void __launch_bounds__(kFirstThreads) k_resid_first_ff(const float2* __restrict__ fd, int nn,
                                                                  float* __restrict__ r32,
                                                                  double* __restrict__ norms) {
  const int b = blockIdx.y;
  const size_t pb = (size_t)b * nn;
  float rr = 0.f;
  for (int i = blockIdx.x * kFirstThreads + threadIdx.x; i < nn; i += gridDim.x * kFirstThreads) {
    const float2 f = fd[pb + i];
    const float r = f.x + f.y;
    r32[pb + i] = r;
    rr = fmaf(r, r, rr);
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  __shared__ float part[kFirstThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = rr;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kFirstThreads / 32; ++w) t += part[w];
    if (t != 0.f) atomicAdd(norms + b, (double)t);
  }
}

// final potential u = base + e for a float-float correction
__global__ void k_combine_ff(double* __restrict__ base, const float2* __restrict__ e, int n) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  if (i >= n || j >= n) return;
  const size_t side = n + 2;
  const size_t c = (size_t)b * side * side + (size_t)(i + 1) * side + (j + 1);
  const float2 v = e[(size_t)b * upatch(n) + uidx(n, i, j)];
  base[c] += f2d_exact(v.x) + f2d_exact(v.y);
}

// final potential u = base + e (interior cells)
template <typename T>
__global__ void k_combine(double* __restrict__ base, const T* __restrict__ e, int n) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  if (i >= n || j >= n) return;
  const size_t side = n + 2;
  const size_t c = (size_t)b * side * side + (size_t)(i + 1) * side + (j + 1);
  base[c] += (double)e[(size_t)b * upatch(n) + uidx(n, i, j)];
}

// lens fields at every pixel centre of nside_fine, each in its own bundle's patch
__global__ void k_fields_at_pixels(MGView V, int nf, int nb, double* a_th, double* a_ph, double* u_tt,
                                   double* u_pp, double* u_tp) {
  const int64_t np = 12ll * nf * nf;
  const int shift = 2 * (ilog2(nf) - ilog2(nb));
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t j;
    const int i = pix2ring(nf, p, &j);
    const Ring r = ring_geom(nf, i);
    const double phi = r.phi0 + (2.0 * kPi) * (double)j / (double)r.npix;
    const int64_t pn = ang2pix_nest(nf, r.z, phi);
    const int b = (int)(pn >> shift);
    const double nv[3] = {r.s * cos(phi), r.s * sin(phi), r.z};
    double o[5];
    double et[3], ep[3];
    tangent_basis(nv, et, ep);
    patch_lens_fields(V, b, nv, et, ep, o);
    if (a_th) a_th[p] = o[0];
    if (a_ph) a_ph[p] = o[1];
    if (u_tt) u_tt[p] = o[2];
    if (u_pp) u_pp[p] = o[3];
    if (u_tp) u_tp[p] = o[4];
  }
}

__global__ void k_fields_at_points(MGView V, const double* z, const double* phi, const int32_t* bundle, int64_t n,
                                   int nb, double* a_th, double* a_ph, double* u_tt, double* u_pp, double* u_tp) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double zz = z[k], pp = phi[k];
    const double s = sqrt((1.0 - zz) * (1.0 + zz));
    const double nv[3] = {s * cos(pp), s * sin(pp), zz};
    const int b = bundle ? bundle[k] : (int)ang2pix_nest(nb, zz, pp);
    double o[5];
    double et[3], ep[3];
    tangent_basis(nv, et, ep);
    patch_lens_fields(V, b, nv, et, ep, o);
    if (a_th) a_th[k] = o[0];
    if (a_ph) a_ph[k] = o[1];
    if (u_tt) u_tt[k] = o[2];
    if (u_pp) u_pp[k] = o[3];
    if (u_tp) u_tp[k] = o[4];
  }
}

static int blocks_for(clc_ctx* ctx, size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  const size_t cap = (size_t)num_sms(ctx) * 32;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// host: invert a dense matrix (Gauss-Jordan with partial pivoting)
static bool invert(std::vector<double>& A, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] *= d;
      inv[(size_t)c * n + k] *= d;
    }
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double fct = A[(size_t)r * n + c];
        if (fct != 0.0)
          for (int k = 0; k < n; ++k) {
            A[(size_t)r * n + k] -= fct * A[(size_t)c * n + k];
            inv[(size_t)r * n + k] -= fct * inv[(size_t)c * n + k];
          }
      }
  }
  A.swap(inv);
  return true;
}

struct LevelCoef {
  std::vector<double> coef;  // aS, aN, b, area
  std::vector<double> invd;  // 1 / diagonal
  std::vector<double> diag;  // diagonal (ghost extrapolation terms included)
  std::vector<double> rden;  // 1 / (2 (area_2I + area_2I+1)) for the coarse rows
};

static LevelCoef level_coef(int n, double h) {
  LevelCoef L;
  L.coef.resize(4 * (size_t)n);
  L.invd.resize((size_t)n * n);
  L.diag.resize((size_t)n * n);
  for (int i = 0; i < n; ++i) {
    const double th = 0.5 * kPi + (i + 0.5 - 0.5 * n) * h;
    const double s = std::sin(th), sp = std::sin(th + 0.5 * h), sm = std::sin(th - 0.5 * h);
    L.coef[i] = sp / (h * h * s);
    L.coef[n + i] = sm / (h * h * s);
    L.coef[2 * n + i] = 1.0 / (h * h * s * s);
    L.coef[3 * n + i] = std::cos(th - 0.5 * h) - std::cos(th + 0.5 * h);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double aS = L.coef[i], aN = L.coef[n + i], b = L.coef[2 * n + i];
      double d = aS + aN + 2.0 * b;
      if (i == 0) d += aN;
      if (i == n - 1) d += aS;
      if (j == 0) d += b;
      if (j == n - 1) d += b;
      L.diag[(size_t)i * n + j] = d;
      L.invd[(size_t)i * n + j] = 1.0 / d;
    }
  L.rden.resize(n / 2 > 0 ? n / 2 : 1);
  for (int I = 0; I < n / 2; ++I) L.rden[I] = 1.0 / (2.0 * (L.coef[3 * n + 2 * I] + L.coef[3 * n + 2 * I + 1]));
  return L;
}

static dim3 grid3(int nx, int ny, int npatch) { return dim3((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY, npatch); }

// ---------------------------------------------------------------------------
// The paper's stopping rule (Sec. 3.2): ||r|| < eps ||tau||, tau = L_c R u -
// R L_f u the truncation-error estimate of the full approximation scheme on
// the next coarser level, u = base + e with its Dirichlet ghost ring.

// 2 psi_SHT at the centres of the coarse level's edge faces (the coarse
// ghost ring), per patch [top J, bottom J, left I, right I] x nc
__global__ void k_mg_coarse_ghosts(int nc, double hc, const double* __restrict__ rot, const double* __restrict__ psi,
                                   int ns, const double* __restrict__ ring_th, double* __restrict__ gc) {
  const int b = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * nc) return;
  const int side = t / nc, k = t % nc;
  const double edge = 0.5 * nc * hc, cen = (k + 0.5 - 0.5 * nc) * hc;
  double dth, dph;   // theta' - pi/2 and phi' of the face centre
  if (side == 0) { dth = -edge; dph = cen; }
  else if (side == 1) { dth = edge; dph = cen; }
  else if (side == 2) { dth = cen; dph = -edge; }
  else { dth = cen; dph = edge; }
  // theta' = pi/2 + dth: sin theta' = cos dth, cos theta' = -sin dth
  double sd, cd, sp, cp;
  sincos(dth, &sd, &cd);
  sincos(dph, &sp, &cp);
  const double v[3] = {cd * cp, cd * sp, -sd};
  double th, ph;
  cell_angles(rot + 9 * (size_t)b, v, &th, &ph);
  gc[(size_t)b * 4 * nc + t] = 2.0 * interp_map_tab(psi, ns, ring_th, th, ph);
}

template <typename E>
__device__ __forceinline__ double e_at(const E* e, size_t k) { return (double)e[k]; }
template <>
__device__ __forceinline__ double e_at<float2>(const float2* e, size_t k) {
  const float2 v = e[k];
  return f2d_exact(v.x) + f2d_exact(v.y);
}

// ||tau||^2 per patch over the coarse cells
template <typename E>
__global__ void k_tau_norm(int n, const double* __restrict__ base, const E* __restrict__ e,
                           const double* __restrict__ cf, const double* __restrict__ df,
                           const double* __restrict__ cc, const double* __restrict__ dc,
                           const double* __restrict__ rd, const double* __restrict__ gc, double* __restrict__ tau2) {
  const int b = blockIdx.z;
  const int nc = n / 2, side = n + 2;
  const int I = blockIdx.y * kBY + threadIdx.y, J = blockIdx.x * kBX + threadIdx.x;
  double tt = 0.0;
  if (I < nc && J < nc) {
    const double* B = base + (size_t)b * side * side;
    const E* Eb = e + (size_t)b * upatch(n);
    // fine u at -1 <= i, j <= n (the correction's ghost ring is zero)
    auto u = [&](int i, int j) -> double { return B[(size_t)(i + 1) * side + (j + 1)] + e_at(Eb, uidx(n, i, j)); };
    auto Ru = [&](int Ic, int Jc) -> double {
      if (Ic < 0) return gc[(size_t)b * 4 * nc + Jc];
      if (Ic >= nc) return gc[(size_t)b * 4 * nc + nc + Jc];
      if (Jc < 0) return gc[(size_t)b * 4 * nc + 2 * nc + Ic];
      if (Jc >= nc) return gc[(size_t)b * 4 * nc + 3 * nc + Ic];
      const int i = 2 * Ic, j = 2 * Jc;
      return (cf[3 * n + i] * (u(i, j) + u(i, j + 1)) + cf[3 * n + i + 1] * (u(i + 1, j) + u(i + 1, j + 1))) * rd[Ic];
    };
    auto Lf = [&](int i, int j) -> double {
      return cf[i] * u(i + 1, j) + cf[n + i] * u(i - 1, j) + cf[2 * n + i] * (u(i, j + 1) + u(i, j - 1)) -
             df[(size_t)i * n + j] * u(i, j);
    };
    const double Lc = cc[I] * Ru(I + 1, J) + cc[nc + I] * Ru(I - 1, J) + cc[2 * nc + I] * (Ru(I, J + 1) + Ru(I, J - 1)) -
                      dc[(size_t)I * nc + J] * Ru(I, J);
    const int i = 2 * I, j = 2 * J;
    const double RL = (cf[3 * n + i] * (Lf(i, j) + Lf(i, j + 1)) + cf[3 * n + i + 1] * (Lf(i + 1, j) + Lf(i + 1, j + 1))) *
                      rd[I];
    const double t = Lc - RL;
    tt = t * t;
  }
  for (int o = 16; o > 0; o >>= 1) tt += __shfl_xor_sync(0xffffffffu, tt, o);
  if (threadIdx.x == 0 && tt != 0.0) atomicAdd(tau2 + b, tt);
}

// max over patches of rms(r) / rms(tau) = sqrt(rr / tau2) / 2 (n^2 fine
// cells against (n/2)^2 coarse ones)
__global__ void k_max_ratio_tau(const double* __restrict__ rr, const double* __restrict__ t2, int npatch,
                                double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (b < npatch) {
    const double r = rr[b], t = t2[b];
    const double q = t > 0.0 ? 0.5 * sqrt(r / t) : (r > 0.0 ? HUGE_VAL : 0.0);
    mx = fmax(mx, q);
  }
  block_max_into(mx, out);
}

template <typename T>
struct MG {
  clc_plane_solution* s;
  clc_ctx* ctx;
  bool mixed = false;  // FP32 V-cycles on an FP64 residual equation
  T* U(int l) { return (T*)s->u[l].p; }
  T* U2(int l) { return (T*)s->u2[l].p; }
  T* F(int l) { return (T*)s->f[l].p; }
  static constexpr bool kF32 = sizeof(T) == 4;
  const T* C(int l) { return (const T*)(kF32 ? s->coef32[l].p : s->coef[l].p); }
  const T* D(int l) { return (const T*)(kF32 ? s->invd32[l].p : s->invd[l].p); }
  const T* G(int l) { return (const T*)(kF32 ? s->diag32[l].p : s->diag[l].p); }
  const T* RD(int l) { return (const T*)(kF32 ? s->rden32[l].p : s->rden[l].p); }
  const double* C64(int l) { return (const double*)s->coef[l].p; }
  const double* G64(int l) { return (const double*)s->diag[l].p; }

  // nu red-black sweeps at level l, one colour per launch
  // shared memory a CTA may use (opt-in limit of the device)
  size_t smem_cap() {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    return (size_t)v;
  }

  template <int N>
  void band_smooth_restrict(int l, bool zero, size_t smb) {
    cudaFuncSetAttribute(k_band_smooth_restrict<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    CLC_LAUNCH(ctx, "k_smooth_restrict", (k_band_smooth_restrict<T, N>), dim3(N / BandGeo<N>::br, 1, s->npatch),
               dim3(kBandThreads), smb, zero ? nullptr : U(l), U2(l), F(l), C(l), D(l), G(l), RD(l), s->p.nu1,
               F(l + 1), ctx->d_err);
  }
  template <int N>
  void band_prolong_smooth(int l, size_t smb) {
    cudaFuncSetAttribute(k_band_prolong_smooth<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    CLC_LAUNCH(ctx, "k_prolong_smooth", (k_band_prolong_smooth<T, N>), dim3(N / BandGeo<N>::br, 1, s->npatch),
               dim3(kBandThreads), smb, U2(l), U(l), F(l), C(l), D(l), G(l), U(l + 1), s->p.nu2, ctx->d_err);
  }

  // pre-smoothing (u -> u2; u taken as zero when `zero`) and restriction of
  // the residual to level l + 1: row bands for patches of 16 .. kBandMaxN
  // cells a side, square blocks beyond
  // register-resident band kernels: FP32, two sweeps, 128 or 256 cells a side
  static constexpr int kRegPartsSR = 3, kRegPartsPS = 2;   // row parts of the two kernels' regions
  template <int N>
  void reg_smooth_restrict(int l, bool zero) {
    using QB = QBand<N, kSRHalo, kRegPartsSR>;
    // static plus dynamic shared memory goes beyond 48 KB: opt in
    cudaFuncSetAttribute(k_reg_smooth_restrict<N, kRegPartsSR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)QB::f_bytes);
    CLC_LAUNCH(ctx, "k_smooth_restrict", (k_reg_smooth_restrict<N, kRegPartsSR>), dim3(N / QB::BR, 1, s->npatch),
               dim3(QB::NT), QB::f_bytes, zero ? nullptr : (const float*)U(l), (float*)U2(l), (const float*)F(l),
               (const float*)C(l), (const float*)D(l), (const float*)G(l), (const float*)RD(l), (float*)F(l + 1),
               ctx->d_err);
  }
  template <int N>
  void reg_prolong_smooth(int l) {
    using QB = QBand<N, 4, kRegPartsPS>;
    constexpr size_t smb = QB::f_bytes + QB::e_bytes;
    cudaFuncSetAttribute(k_reg_prolong_smooth<N, kRegPartsPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    CLC_LAUNCH(ctx, "k_prolong_smooth", (k_reg_prolong_smooth<N, kRegPartsPS>), dim3(N / QB::BR, 1, s->npatch),
               dim3(QB::NT), smb, (const float*)U2(l), (float*)U(l), (const float*)F(l), (const float*)C(l),
               (const float*)D(l), (const float*)G(l), (const float*)U(l + 1), ctx->d_err);
  }
  // eight columns per thread (k_oct_*, 256-cell patches) or four (k_reg_*) in
  // the register band kernels; row parts 3 and 4 measured fastest at Nside 2048
  static constexpr bool kOctSR = true, kOctPS = true;
  static constexpr int kOctPartsSR = 3, kOctPartsPS = 4;
  template <int N>
  void oct_smooth_restrict(int l, bool zero) {
    using OB = OBand<N, kSRHalo, kOctPartsSR>;
    cudaFuncSetAttribute(k_oct_smooth_restrict<N, kOctPartsSR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)OB::f_bytes);
    CLC_LAUNCH(ctx, "k_smooth_restrict", (k_oct_smooth_restrict<N, kOctPartsSR>), dim3(N / OB::BR, 1, s->npatch),
               dim3(OB::NT), (OB::f_bytes), zero ? nullptr : (const float*)U(l), (float*)U2(l), (const float*)F(l),
               (const float*)C(l), (const float*)D(l), (const float*)G(l), (const float*)RD(l), (float*)F(l + 1),
               ctx->d_err);
  }
  template <int N>
  void oct_prolong_smooth(int l) {
    using OB = OBand<N, 4, kOctPartsPS>;
    constexpr size_t smb = OB::f_bytes + OB::e_bytes;
    cudaFuncSetAttribute(k_oct_prolong_smooth<N, kOctPartsPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    CLC_LAUNCH(ctx, "k_prolong_smooth", (k_oct_prolong_smooth<N, kOctPartsPS>), dim3(N / OB::BR, 1, s->npatch),
               dim3(OB::NT), smb, (const float*)U2(l), (float*)U(l), (const float*)F(l), (const float*)C(l),
               (const float*)D(l), (const float*)G(l), (const float*)U(l + 1), ctx->d_err);
  }
  bool use_reg(int n, int nu) const { return kF32 && nu == 2 && (n == 128 || n == 256); }

  void smooth_restrict(int l, bool zero) {
    const int n = s->sizes[l], nu = s->p.nu1;
    if (use_reg(n, nu)) {
      if (kOctSR && n == 256) {
        oct_smooth_restrict<256>(l, zero);
      } else {
        if (n == 128) reg_smooth_restrict<128>(l, zero);
        else reg_smooth_restrict<256>(l, zero);
      }
      return;
    }
    const size_t smb = band_smem<T>(n, 2 * nu + 1);
    if (n >= 16 && n <= kBandMaxN && smb <= smem_cap()) {
      switch (n) {
        case 16: band_smooth_restrict<16>(l, zero, smb); return;
        case 32: band_smooth_restrict<32>(l, zero, smb); return;
        case 64: band_smooth_restrict<64>(l, zero, smb); return;
        case 128: band_smooth_restrict<128>(l, zero, smb); return;
        case 256: band_smooth_restrict<256>(l, zero, smb); return;
        default: break;
      }
    }
    const int ts = tile_side(n);
    const size_t sm = tile_smem<T>(n, 2 * nu + 1);
    cudaFuncSetAttribute(k_smooth_restrict<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    CLC_LAUNCH(ctx, "k_smooth_restrict", k_smooth_restrict<T>, dim3((n / ts) * (n / ts), 1, s->npatch),
               dim3(kBX, kBY), sm, zero ? nullptr : U(l), U2(l), F(l), C(l), D(l), G(l), RD(l), n, nu, F(l + 1));
  }

  // prolongation of the level l + 1 correction and post-smoothing (u2 -> u)
  void prolong_smooth(int l) {
    const int n = s->sizes[l], nu = s->p.nu2;
    if (use_reg(n, nu)) {
      if (kOctPS && n == 256) {
        oct_prolong_smooth<256>(l);
      } else {
        if (n == 128) reg_prolong_smooth<128>(l);
        else reg_prolong_smooth<256>(l);
      }
      return;
    }
    const int wcb = ((n < kBandRows ? n : kBandRows) + 4 * nu) / 2 + 2;
    const size_t smb = band_smem<T>(n, 2 * nu) + (size_t)wcb * (n / 2 + 2) * sizeof(T);
    if (n >= 16 && n <= kBandMaxN && smb <= smem_cap()) {
      switch (n) {
        case 16: band_prolong_smooth<16>(l, smb); return;
        case 32: band_prolong_smooth<32>(l, smb); return;
        case 64: band_prolong_smooth<64>(l, smb); return;
        case 128: band_prolong_smooth<128>(l, smb); return;
        case 256: band_prolong_smooth<256>(l, smb); return;
        default: break;
      }
    }
    const int ts = tile_side(n);
    const int wc = (ts + 4 * nu) / 2 + 2;
    const size_t sm = tile_smem<T>(n, 2 * nu) + (size_t)wc * wc * sizeof(T);
    cudaFuncSetAttribute(k_prolong_smooth<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    CLC_LAUNCH(ctx, "k_prolong_smooth", k_prolong_smooth<T>, dim3((n / ts) * (n / ts), 1, s->npatch),
               dim3(kBX, kBY), sm, U2(l), U(l), F(l), C(l), D(l), G(l), U(l + 1), n, nu);
  }

  // V-cycle at level l on L e = f; `zero`: e starts at zero (coarse levels,
  // and the finest one when its correction was just reset).  For the linear
  // operator the coarse equation of the full approximation scheme, written
  // for e_c = u_c - R u, is L_c e_c = R (f - L u) from e_c = 0: the same
  // iterates with no restricted copy of u and no coarse source update.
  // the levels from l down in one launch (k_sub_vcycle) when they are small
  // enough: 16 or 32 cells a side, halving to the 8 x 8 coarsest level
  bool use_sub(int l) {
    const int n = s->sizes[l];
    return (n == 16 || n == kSubMax) && s->sizes[s->nlev - 1] == kSubCoarse && s->p.nu1 >= 1 &&
           sub_bytes(n) <= smem_cap();
  }
  static size_t sub_bytes(int n) { return n == 32 ? sizeof(SubStack<T, 32>) : sizeof(SubStack<T, 16>); }
  template <int N0>
  void sub_launch(int l, bool zero, const SubArgs<T>& a) {
    const size_t smb = sizeof(SubStack<T, N0>);
    cudaFuncSetAttribute(k_sub_vcycle<T, N0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    CLC_LAUNCH(ctx, "k_sub_vcycle", (k_sub_vcycle<T, N0>), s->npatch, kSubThreads, smb, U(l), (const T*)F(l),
               zero ? 1 : 0, a);
  }
  void sub_vcycle(int l, bool zero) {
    SubArgs<T> a{};
    a.nu1 = s->p.nu1;
    a.nu2 = s->p.nu2;
    for (int k = 0; l + k < s->nlev - 1 && k < 4; ++k)
      a.lev[k] = SubLev<T>{(const T*)C(l + k), (const T*)D(l + k), (const T*)G(l + k), (const T*)RD(l + k)};
    a.minv = (const double*)s->coarse_inv.p;
    a.minv32 = (const float*)s->coarse_inv32.p;
    if (s->sizes[l] == 32) sub_launch<32>(l, zero, a);
    else sub_launch<16>(l, zero, a);
  }

  void vcycle(int l, bool zero) {
    const int n = s->sizes[l];
    if (use_sub(l)) {
      sub_vcycle(l, zero);
      return;
    }
    if (l == s->nlev - 1) {
      CLC_LAUNCH(ctx, "k_coarse_solve", k_coarse_solve<T>, s->npatch, 64, n * n * sizeof(double), U(l), F(l), C64(l),
                 (const double*)s->coarse_inv.p, n);
      return;
    }
    smooth_restrict(l, zero);
    vcycle(l + 1, true);
    prolong_smooth(l);
  }

  // the paper's rule applies when asked for and when there is a coarser level
  bool tau_rule() const { return s->p.stop_rule == CLC_STOP_TAU && s->nlev > 1; }

  // ratio of the stopping rule into s->ratio from the per-patch residual
  // norms in s->norms: ||r|| / ||f|| (relative residual) or rms(r) / rms(tau)
  // with tau from u = base + e
  template <typename E>
  void stop_ratio(const E* e, bool tau) {
    const int n = s->sizes[0];
    if (!tau) {
      cudaMemsetAsync(s->ratio.p, 0, sizeof(double), ctx->stream);
      CLC_LAUNCH(ctx, "k_max_ratio", k_max_ratio, (s->npatch + 255) / 256, 256, 0, (const double*)s->norms.p,
                 (const double*)s->fnorm.p,
                 s->npatch, (double*)s->ratio.p);
      return;
    }
    cudaMemsetAsync(s->tau2.p, 0, sizeof(double) * s->npatch, ctx->stream);
    CLC_LAUNCH(ctx, "k_tau_norm", k_tau_norm<E>, grid3(n / 2, n / 2, s->npatch), dim3(kBX, kBY), 0, n,
               (const double*)s->base.p, e, C64(0), G64(0), C64(1), G64(1), (const double*)s->rden[0].p,
               (const double*)s->gc.p, (double*)s->tau2.p);
    cudaMemsetAsync(s->ratio.p, 0, sizeof(double), ctx->stream);
    CLC_LAUNCH(ctx, "k_max_ratio", k_max_ratio_tau, (s->npatch + 255) / 256, 256, 0, (const double*)s->norms.p,
               (const double*)s->tau2.p,
               s->npatch, (double*)s->ratio.p);
  }

  int residual(double* ratio_host, bool tau = false) {
    const int n = s->sizes[0];
    cudaMemsetAsync(s->norms.p, 0, sizeof(double) * s->npatch, ctx->stream);
    CLC_LAUNCH(ctx, "k_resnorm", k_resnorm<T>, grid3(n, n, s->npatch), dim3(kBX, kBY), 0, U(0), F(0), C64(0), G64(0), n,
               (double*)s->norms.p);
    stop_ratio<T>(U(0), tau);
    int rc = launch_check(ctx, "MG residual");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpyAsync(ratio_host, s->ratio.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                    "residual copy");
    if (rc) return rc;
    return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "residual sync");
  }

  // base (SHT solution + edge values), defect source f' = kappa - L base,
  // ||kappa||^2 per patch, and a zero starting correction
  int setup(const double* kappa_fine) {
    if (tau_rule()) {
      const int nc = s->sizes[1];
      CLC_LAUNCH(ctx, "k_mg_coarse_ghosts", k_mg_coarse_ghosts, dim3((4 * nc + 127) / 128, s->npatch), 128, 0, nc,
                 2.0 * s->h, (const double*)s->rot.p, (const double*)s->psi_sht.p, s->p.nside_sht,
                 (const double*)s->ring_th_sht.p, (double*)s->gc.p);
    }
    if (mixed && s->plan) return setup_ff(kappa_fine);
    if (mixed) return setup_t<float2>(kappa_fine, (float2*)s->fd64.p);
    return setup_t<T>(kappa_fine, F(0));
  }

  // mixed set-up in float-float arithmetic: both maps split once, then the
  // plans applied on the FP32 pipe
  int setup_ff(const double* kappa_fine) {
    const int n = s->sizes[0];
    const dim3 blk(kBX, kBY);
    const int64_t ns2 = 12ll * s->p.nside_sht * s->p.nside_sht, nf2 = 12ll * s->nside_fine * s->nside_fine;
    cudaMemsetAsync(s->fnorm.p, 0, sizeof(double) * s->npatch, ctx->stream);
    CLC_LAUNCH(ctx, "k_split_ff", k_split_ff, blocks_for(ctx, ns2, 256), 256, 0, (const double*)s->psi_sht.p,
               (float2*)s->psi_ff.p, ns2);
    CLC_LAUNCH(ctx, "k_split_ff", k_split_ff, blocks_for(ctx, nf2, 256), 256, 0, kappa_fine, (float2*)s->kap_ff.p,
               nf2);
    const dim3 gb = grid3(n + 2, n + 2, s->npatch);
    const dim3 gd((n + kBX - 1) / kBX, (n + kBY * kSetupRows - 1) / (kBY * kSetupRows), s->npatch);
    CLC_LAUNCH(ctx, "k_mg_setup_base", k_mg_setup_base_ff, gb, blk, 0, n,
               (const int4*)s->plan_psi_idx.p, (const double4_32a*)s->plan_psi_w.p, (const float2*)s->psi_ff.p,
               (const double*)s->psi_sht.p, s->p.nside_sht, (const double*)s->ring_th_sht.p, (float2*)s->base_ff.p,
               (double*)s->base.p);
    CLC_LAUNCH(ctx, "k_mg_setup_defect", k_mg_setup_defect_ff, gd, blk, 0, n,
               (const int4*)s->plan_kap_idx.p, (const double4_32a*)s->plan_kap_w.p, (const float2*)s->kap_ff.p,
               kappa_fine, s->nside_fine, (const double*)s->ring_th_fine.p, (const float2*)s->base_ff.p,
               (const float2*)s->coef_ff.p, (const float2*)s->diag_ff.p, (float2*)s->fd64.p, (double*)s->fnorm.p);
    cudaMemsetAsync(s->e64.p, 0, s->e64.bytes, ctx->stream);
    return launch_check(ctx, "MG set-up (float-float)");
  }

  template <typename S>
  int setup_t(const double* kappa_fine, S* fdst) {
    const int n = s->sizes[0];
    const dim3 blk(kBX, kBY);
    cudaMemsetAsync(s->fnorm.p, 0, sizeof(double) * s->npatch, ctx->stream);
    if (s->plan) {
      CLC_LAUNCH(ctx, "k_mg_setup_base", k_mg_setup_base_plan, grid3(n + 2, n + 2, s->npatch), blk, 0, n,
                 (const int4*)s->plan_psi_idx.p, (const double4_32a*)s->plan_psi_w.p, (const double*)s->psi_sht.p,
                 s->p.nside_sht, (const double*)s->ring_th_sht.p, (double*)s->base.p);
      CLC_LAUNCH(ctx, "k_mg_setup_defect", k_mg_setup_defect_plan<S>, grid3(n, n, s->npatch), blk, 0, n,
                 (const int4*)s->plan_kap_idx.p, (const double4_32a*)s->plan_kap_w.p, kappa_fine, s->nside_fine,
                 (const double*)s->ring_th_fine.p, (const double*)s->base.p, C64(0), G64(0), fdst,
                 (double*)s->fnorm.p);
    } else {
      CLC_LAUNCH(ctx, "k_mg_setup_base", k_mg_setup_base, grid3(n + 2, n + 2, s->npatch), blk, 0, n,
                 (const double*)s->rot.p, (const double*)s->pvec.p, (const double*)s->psi_sht.p, s->p.nside_sht,
                 (const double*)s->ring_th_sht.p, (double*)s->base.p);
      CLC_LAUNCH(ctx, "k_mg_setup_defect", k_mg_setup_defect<S>, grid3(n, n, s->npatch), blk, 0, n,
                 (const double*)s->rot.p, (const double*)s->pvec.p, kappa_fine, s->nside_fine,
                 (const double*)s->ring_th_fine.p, (const double*)s->base.p, C64(0), G64(0), fdst,
                 (double*)s->fnorm.p);
    }
    cudaMemsetAsync(mixed ? s->e64.p : s->u[0].p, 0, mixed ? s->e64.bytes : s->u[0].bytes, ctx->stream);
    return launch_check(ctx, "MG setup");
  }

  // CLC_MIXED, before the first V-cycle (e = 0): r = f'
  int residual_first(const float2* e_zero, double* ratio_host) {
    const int n = s->sizes[0], nn = n * n;
    cudaMemsetAsync(s->norms.p, 0, sizeof(double) * s->npatch, ctx->stream);
    const dim3 grid((nn + kFirstThreads * kFirstPer - 1) / (kFirstThreads * kFirstPer), s->npatch);
    CLC_LAUNCH(ctx, "k_resid_mixed", k_resid_first_ff, grid, kFirstThreads, 0, (const float2*)s->fd64.p, nn,
               (float*)s->f[0].p, (double*)s->norms.p);
    stop_ratio<float2>(e_zero, tau_rule());
    int rc = launch_check(ctx, "MG mixed residual");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpyAsync(ratio_host, s->ratio.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                    "residual copy");
    if (rc) return rc;
    return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "residual sync");
  }

  // CLC_MIXED: r = f' - L e in float-float (also the next FP32 source), FP32
  // V-cycle on L d = r from d = 0, e += d; u = base + e at the end
  int residual_mixed(const float2* e_old, const float* d, float2* e_new, double* ratio_host) {
    const int n = s->sizes[0];
    cudaMemsetAsync(s->norms.p, 0, sizeof(double) * s->npatch, ctx->stream);
    const dim3 grid((n / 2 + kBX - 1) / kBX, (n + kBY * kWalk - 1) / (kBY * kWalk), s->npatch);
    CLC_LAUNCH(ctx, "k_resid_mixed", k_resid_ff_walk, grid, dim3(kBX, kBY), 0, e_old, d, (const float2*)s->fd64.p,
               (const float2*)s->coef_ff.p, (const float2*)s->diag_ff.p, n, e_new, (float*)s->f[0].p,
               (double*)s->norms.p);
    stop_ratio<float2>(e_new, tau_rule());
    int rc = launch_check(ctx, "MG mixed residual");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaMemcpyAsync(ratio_host, s->ratio.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                    "residual copy");
    if (rc) return rc;
    return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "residual sync");
  }

  int solve_mixed() {
    int rc;
    double rr = 0.0;
    s->cycles = 0;
    const int n = s->sizes[0];
    const bool fixed = s->p.fixed_cycles > 0;
    float2* cur = (float2*)s->e64.p;
    float2* nxt = (float2*)s->e64b.p;
    if ((rc = residual_first(cur, &rr))) return rc;   // cur: zero since the set-up
    const double limit = tau_rule() ? s->p.eps : s->p.tol;
    const int per = s->p.refine_cycles > 0 ? s->p.refine_cycles : 2;
    while (fixed ? s->cycles < s->p.fixed_cycles : (rr >= limit && s->cycles < s->p.max_cycles)) {
      // `per` FP32 V-cycles on L d = r (each continuing from the last) per
      // refinement of the FP64-accurate residual, the bandwidth-heavy part
      const int left = fixed ? s->p.fixed_cycles - s->cycles : s->p.max_cycles - s->cycles;
      const int inner = left < per ? left : per;
      for (int k = 0; k < inner; ++k) vcycle(0, k == 0);   // d starts at zero in each refinement
      s->cycles += inner - 1;
      if ((rc = launch_check(ctx, "mixed V-cycle"))) return rc;
      if ((rc = residual_mixed(cur, (const float*)s->u[0].p, nxt, &rr))) return rc;
      std::swap(cur, nxt);
      ++s->cycles;
    }
    s->residual = rr;
    CLC_LAUNCH(ctx, "k_combine", k_combine_ff, grid3(n, n, s->npatch), dim3(kBX, kBY), 0, (double*)s->base.p,
               (const float2*)cur, n);
    if ((rc = launch_check(ctx, "MG combine"))) return rc;
    if (!fixed && rr >= limit) return set_err(ctx, CLC_ENOTCONVERGED, "MG stopped at max_cycles above tol");
    return CLC_OK;
  }

  int finish() {
    const int n = s->sizes[0];
    CLC_LAUNCH(ctx, "k_combine", k_combine<T>, grid3(n, n, s->npatch), dim3(kBX, kBY), 0, (double*)s->base.p, U(0), n);
    return launch_check(ctx, "MG combine");
  }

  int solve() {
    int rc;
    double rr = 0.0;
    s->cycles = 0;
    int st = CLC_OK;
    const bool tau = tau_rule();
    const double limit = tau ? s->p.eps : s->p.tol;
    if (s->p.fixed_cycles > 0) {
      for (int k = 0; k < s->p.fixed_cycles; ++k) {
        vcycle(0, false);
        if ((rc = launch_check(ctx, "V-cycle"))) return rc;
      }
      s->cycles = s->p.fixed_cycles;
      if ((rc = residual(&rr, tau))) return rc;
    } else {
      if ((rc = residual(&rr, tau))) return rc;
      while (rr >= limit && s->cycles < s->p.max_cycles) {
        vcycle(0, false);
        if ((rc = launch_check(ctx, "V-cycle"))) return rc;
        ++s->cycles;
        if ((rc = residual(&rr, tau))) return rc;
      }
      if (rr >= limit) st = set_err(ctx, CLC_ENOTCONVERGED, "MG stopped at max_cycles above tol");
    }
    s->residual = rr;
    if ((rc = finish())) return rc;
    return st;
  }
};

// ---------------------------------------------------------------------------
// Adjoint of the converged patch solve (the SHT+MG adjoint).
//
// Converged, the interior potential of a patch is u = L^-1 (f - L_g G): L the
// interior operator with the Dirichlet extrapolation on its diagonal, L_g the
// coupling of the edge rows and columns to the ghost ring G = 2 g (g =
// psi_SHT at the edge-face centres) and f = kappa at the cell centres (the
// interior starting guess drops out).  Given the adjoint ubar of u,
// lambda = L^-T ubar, fbar = lambda and gbar = -2 L_g^T lambda.  W L is
// symmetric for W = diag(cos((i + 1/2 - n/2) h)) = diag(sin theta'_i) (the
// finite-volume fluxes between rows i, i + 1 carry sin theta'_{i+1/2} on both
// sides; the phi fluxes and the diagonal are local to a row), so
// L^T = W L W^-1 and lambda = W mu with L mu = W^-1 ubar: the forward
// V-cycles from zero with zero Dirichlet data, run to the tolerance.  fbar
// and gbar then go back through the transposed interpolations to kappa_fine
// and psi_SHT.

__global__ void k_adj_rhs(int n, const double* __restrict__ ubar, const double* __restrict__ wrow,
                          double* __restrict__ f, double* __restrict__ fnorm) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  double ff = 0.0;
  if (i < n && j < n) {
    const double r = ubar[(size_t)b * n * n + (size_t)i * n + j] / wrow[i];
    f[(size_t)b * n * n + fidx(n, i, j)] = r;
    ff = r * r;
  }
  for (int o = 16; o > 0; o >>= 1) ff += __shfl_xor_sync(0xffffffffu, ff, o);
  if (threadIdx.x == 0 && ff != 0.0) atomicAdd(fnorm + b, ff);
}

// v at (theta, phi) scattered into map through the ring-bilinear weights
__device__ __forceinline__ void scatter_at(double* __restrict__ map, int nside, const double* __restrict__ ring_th,
                                           double th, double ph, double v) {
  const Interp8 o = interp_weights_tab(nside, ring_th, th, ph);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (o.w[k] != 0.0) atomicAdd(map + o.p[k], o.w[k] * v);
}

// v at plan position pos (or, without plans, at patch-frame position `cell`
// of patch b) scattered into map: the transpose of the set-up interpolation
__device__ __forceinline__ void scatter_plan(double* __restrict__ map, int nside, const double* __restrict__ ring_th,
                                             const int4* __restrict__ idx, const double4_32a* __restrict__ w,
                                             size_t pos, const double* __restrict__ R, const double* __restrict__ pv,
                                             double v) {
  if (idx) {
    const int4 ix = idx[pos];
    const double4_32a ww = w[pos];
    if (ix.x < 0) {
      scatter_at(map, nside, ring_th, ww.x, ww.y, v);
    } else {
      atomicAdd(map + ix.x, ww.x * v);
      atomicAdd(map + ix.y, ww.y * v);
      atomicAdd(map + ix.z, ww.z * v);
      atomicAdd(map + ix.w, ww.w * v);
    }
    return;
  }
  double th, ph;
  cell_angles(R, pv, &th, &ph);
  scatter_at(map, nside, ring_th, th, ph, v);
}

// lambda = W mu from the converged correction array; kappa_bar += I_kappa^T
// lambda; psi_bar += I_psi^T (-2 L_g^T lambda) at the ghost positions
__global__ void k_adj_scatter(int n, const double* __restrict__ U, const double* __restrict__ wrow,
                              const double* __restrict__ coef, const int4* __restrict__ kidx,
                              const double4_32a* __restrict__ kw, const int4* __restrict__ pidx,
                              const double4_32a* __restrict__ pw, const double* __restrict__ rot,
                              const double* __restrict__ pvec, int nf, const double* __restrict__ th_fine, int ns,
                              const double* __restrict__ th_sht, double* __restrict__ kbar,
                              double* __restrict__ psibar) {
  const int b = blockIdx.z;
  const int i = blockIdx.y * kBY + threadIdx.y, j = blockIdx.x * kBX + threadIdx.x;
  if (i >= n || j >= n) return;
  const int side = n + 2;
  const double lam = wrow[i] * U[(size_t)b * upatch(n) + uidx(n, i, j)];
  if (lam == 0.0) return;
  const double* R = rot + 9 * (size_t)b;
  scatter_plan(kbar, nf, th_fine, kidx, kw, (size_t)b * n * n + (size_t)i * n + j, R,
               pvec + 3 * (size_t)((i + 1) * side + (j + 1)), lam);
  const size_t pb = (size_t)b * side * side;
  // ghost couplings: aN_0 above row 0, aS_{n-1} below row n - 1, b_i left and right
  if (i == 0)
    scatter_plan(psibar, ns, th_sht, pidx, pw, pb + (size_t)(j + 1), R, pvec + 3 * (size_t)(j + 1),
                 -2.0 * coef[n] * lam);
  if (i == n - 1)
    scatter_plan(psibar, ns, th_sht, pidx, pw, pb + (size_t)(n + 1) * side + (j + 1), R,
                 pvec + 3 * (size_t)((n + 1) * side + (j + 1)), -2.0 * coef[n - 1] * lam);
  if (j == 0)
    scatter_plan(psibar, ns, th_sht, pidx, pw, pb + (size_t)(i + 1) * side, R, pvec + 3 * (size_t)((i + 1) * side),
                 -2.0 * coef[2 * n + i] * lam);
  if (j == n - 1)
    scatter_plan(psibar, ns, th_sht, pidx, pw, pb + (size_t)(i + 1) * side + (n + 1), R,
                 pvec + 3 * (size_t)((i + 1) * side + (n + 1)), -2.0 * coef[2 * n + i] * lam);
}

int mg_adjoint_solve(clc_ctx* ctx, clc_plane_solution* s, const double* ubar, double tol, int max_cycles,
                     double* kbar_fine, double* psibar_sht, int* cycles_out, double* ratio_out) {
  if (s->p.precision != CLC_FP64) return set_err(ctx, CLC_EINVAL, "SHT+MG adjoint needs a CLC_FP64 solution");
  const int n = s->sizes[0];
  if (!s->wrow.p) {
    std::vector<double> w(n);
    for (int i = 0; i < n; ++i) w[i] = std::cos((i + 0.5 - 0.5 * n) * s->h);
    s->wrow.bytes = n * sizeof(double);
    if (cudaMalloc(&s->wrow.p, s->wrow.bytes) != cudaSuccess) {
      cudaGetLastError();
      s->wrow.p = nullptr;
      return set_err(ctx, CLC_ENOMEM, "adjoint row weights");
    }
    int rc = cuda_check(ctx, cudaMemcpy(s->wrow.p, w.data(), s->wrow.bytes, cudaMemcpyHostToDevice), "row weights");
    if (rc) return rc;
  }
  MG<double> mg{s, ctx};
  cudaMemsetAsync(s->fnorm.p, 0, sizeof(double) * s->npatch, ctx->stream);
  CLC_LAUNCH(ctx, "k_adj_rhs", k_adj_rhs, grid3(n, n, s->npatch), dim3(kBX, kBY), 0, n, ubar,
             (const double*)s->wrow.p, mg.F(0), (double*)s->fnorm.p);
  int rc = launch_check(ctx, "k_adj_rhs");
  if (rc) return rc;
  double rr = 0.0;
  int cyc = 0;
  do {
    mg.vcycle(0, cyc == 0);
    if ((rc = launch_check(ctx, "adjoint V-cycle"))) return rc;
    ++cyc;
    if ((rc = mg.residual(&rr))) return rc;
  } while (rr >= tol && cyc < max_cycles);
  if (cycles_out) *cycles_out = cyc;
  if (ratio_out) *ratio_out = rr;
  const bool pl = s->plan;
  CLC_LAUNCH(ctx, "k_adj_scatter", k_adj_scatter, grid3(n, n, s->npatch), dim3(kBX, kBY), 0, n,
             (const double*)mg.U(0), (const double*)s->wrow.p, mg.C64(0),
             pl ? (const int4*)s->plan_kap_idx.p : nullptr, (const double4_32a*)s->plan_kap_w.p,
             pl ? (const int4*)s->plan_psi_idx.p : nullptr, (const double4_32a*)s->plan_psi_w.p,
             (const double*)s->rot.p, (const double*)s->pvec.p, s->nside_fine, (const double*)s->ring_th_fine.p,
             s->p.nside_sht, (const double*)s->ring_th_sht.p, kbar_fine, psibar_sht);
  if ((rc = launch_check(ctx, "k_adj_scatter"))) return rc;
  return rr < tol ? CLC_OK : set_err(ctx, CLC_ENOTCONVERGED, "SHT+MG adjoint solve stopped at max_cycles above tol");
}

static int check_params(clc_ctx* ctx, int nf, const clc_mg_params* p) {
  if (!p) return set_err(ctx, CLC_EINVAL, "null MG parameters");
  if (!valid_nside(nf) || !valid_nside(p->nside_sht) || !valid_nside(p->nside_bundle) || p->nside_bundle > nf ||
      p->nside_sht > 4096)
    return set_err(ctx, CLC_EINVAL, "MG: bad nside");
  if (p->lmax < 1 || p->lmax > 4 * p->nside_sht) return set_err(ctx, CLC_EINVAL, "MG: lmax must be in [1, 4 nside_sht]");
  if (p->ncell < 16 || p->ncell > 4096 || (p->ncell & (p->ncell - 1)))
    return set_err(ctx, CLC_EINVAL, "MG: ncell must be a power of two in [16, 4096]");
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1 || p->nu1 > kMaxSweeps || p->nu2 > kMaxSweeps ||
      p->max_cycles < 0 || p->fixed_cycles < 0)
    return set_err(ctx, CLC_EINVAL, "MG: need 0 <= nu1, nu2 <= 8, nu1 + nu2 >= 1 and cycle counts >= 0");
  if (p->precision != CLC_FP64 && p->precision != CLC_FP32 && p->precision != CLC_MIXED)
    return set_err(ctx, CLC_EINVAL, "MG: bad precision");
  if ((p->stop_rule != CLC_STOP_RESIDUAL && p->stop_rule != CLC_STOP_TAU) ||
      (p->stop_rule == CLC_STOP_TAU && !(p->eps > 0.0)) || p->refine_cycles < 0 || p->refine_cycles > 16)
    return set_err(ctx, CLC_EINVAL, "MG: bad stopping rule, eps or refine_cycles");
  return CLC_OK;
}

}  // namespace clc

using namespace clc;

static int solution_create(clc_ctx* ctx, int nf, const clc_mg_params* p, const int32_t* domain, int ndomain,
                           clc_plane_solution** out) {
  if (!ctx || !out) return CLC_EINVAL;
  *out = nullptr;
  int rc = check_params(ctx, nf, p);
  if (rc) return rc;
  const int nbund = 12 * p->nside_bundle * p->nside_bundle;
  std::vector<int32_t> bslot;
  if (domain) {
    if (ndomain < 1 || ndomain > nbund) return set_err(ctx, CLC_EINVAL, "solution domain: 1 .. 12 nside_bundle^2 bundles");
    bslot.assign(nbund, -1);
    for (int k = 0; k < ndomain; ++k) {
      const int b = domain[k];
      if (b < 0 || b >= nbund || bslot[b] >= 0)
        return set_err(ctx, CLC_EINVAL, "solution domain: bundles must be distinct NEST indices below 12 nside_bundle^2");
      bslot[b] = k;
    }
  }
  cudaSetDevice(ctx->device);
  auto* s = new clc_plane_solution();
  s->ctx = ctx;
  s->nside_fine = nf;
  s->p = *p;
  s->partial = domain != nullptr;
  s->npatch = domain ? ndomain : nbund;
  s->h = 4.0 * std::sqrt(kPi / 3.0) / p->nside_bundle / p->ncell;
  for (int n = p->ncell;; n /= 2) {
    s->sizes.push_back(n);
    if (n <= 8) break;
  }
  s->nlev = (int)s->sizes.size();
  const size_t es = p->precision == CLC_FP64 ? sizeof(double) : sizeof(float);
  size_t need = 0;
  for (int l = 0; l < s->nlev; ++l) {
    const size_t n = s->sizes[l];
    need += s->npatch * (2 * upatch((int)n) + n * n) * es;
  }
  need += (size_t)s->npatch * (p->ncell + 2) * (p->ncell + 2) * sizeof(double) *
          (p->precision == CLC_MIXED ? 4 : 1);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  if (need + (size_t)(1ull << 30) > freeb) {
    delete s;
    return set_err(ctx, CLC_ENOMEM, "MG state of " + std::to_string(need >> 20) + " MiB does not fit");
  }
  auto alloc = [&](Buffer& b, size_t bytes) -> bool {
    b.bytes = bytes;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return false;
    }
    return true;
  };
  bool ok = true;
  for (int l = 0; l < s->nlev && ok; ++l) {
    const size_t n = s->sizes[l];
    const double hl = s->h * (p->ncell / (int)n);
    ok = alloc(s->u[l], s->npatch * upatch((int)n) * es) && alloc(s->f[l], s->npatch * n * n * es) &&
         (l == s->nlev - 1 || alloc(s->u2[l], s->npatch * upatch((int)n) * es));
    if (!ok) break;
    // the ghost rings of the correction stay zero (homogeneous Dirichlet data)
    cudaMemset(s->u[l].p, 0, s->u[l].bytes);
    if (l < s->nlev - 1) cudaMemset(s->u2[l].p, 0, s->u2[l].bytes);
    LevelCoef lc = level_coef((int)n, hl);
    auto put = [&](Buffer& b64, Buffer& b32, const std::vector<double>& v) -> bool {
      if (!alloc(b64, v.size() * sizeof(double)) || !alloc(b32, v.size() * sizeof(float))) return false;
      std::vector<float> v32(v.begin(), v.end());
      cudaMemcpy(b64.p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
      cudaMemcpy(b32.p, v32.data(), v32.size() * sizeof(float), cudaMemcpyHostToDevice);
      return true;
    };
    ok = put(s->coef[l], s->coef32[l], lc.coef) && put(s->invd[l], s->invd32[l], lc.invd) &&
         put(s->diag[l], s->diag32[l], lc.diag) && put(s->rden[l], s->rden32[l], lc.rden);
    if (ok && l == 0 && p->precision == CLC_MIXED) {
      // the finest operator as float-float pairs for the mixed residual
      auto put_ff = [&](Buffer& bf, const std::vector<double>& v) -> bool {
        std::vector<float2> w(v.size());
        for (size_t k = 0; k < v.size(); ++k) {
          w[k].x = (float)v[k];
          w[k].y = (float)(v[k] - (double)w[k].x);
        }
        if (!alloc(bf, w.size() * sizeof(float2))) return false;
        cudaMemcpy(bf.p, w.data(), w.size() * sizeof(float2), cudaMemcpyHostToDevice);
        return true;
      };
      ok = put_ff(s->coef_ff, lc.coef) && put_ff(s->diag_ff, lc.diag);
    }
  }
  const size_t n0 = s->sizes[0];
  ok = ok && alloc(s->base, s->npatch * (n0 + 2) * (n0 + 2) * sizeof(double)) &&
       alloc(s->pvec, (n0 + 2) * (n0 + 2) * 3 * sizeof(double)) &&
       alloc(s->ring_th_sht, (4 * p->nside_sht - 1) * sizeof(double)) &&
       alloc(s->ring_th_fine, (4 * nf - 1) * sizeof(double)) && alloc(s->fnorm, s->npatch * sizeof(double)) &&
       (p->precision != CLC_MIXED || (alloc(s->e64, s->npatch * upatch(n0) * sizeof(float2)) &&
                                     alloc(s->e64b, s->npatch * upatch(n0) * sizeof(float2)) &&
                                     alloc(s->fd64, s->npatch * n0 * n0 * sizeof(double))));
  if (ok && p->precision == CLC_MIXED) cudaMemset(s->e64b.p, 0, s->e64b.bytes);
  if (ok) {
    // patch-frame unit vectors: cell centres inside, edge-face centres on the ring
    std::vector<double> pv((n0 + 2) * (n0 + 2) * 3);
    auto pos = [&](size_t k) {
      if (k == 0) return -0.5 * n0 * s->h;
      if (k == n0 + 1) return 0.5 * n0 * s->h;
      return ((double)k - 0.5 - 0.5 * n0) * s->h;
    };
    for (size_t k1 = 0; k1 < n0 + 2; ++k1)
      for (size_t k2 = 0; k2 < n0 + 2; ++k2) {
        const double tp = 0.5 * kPi + pos(k1), pp = pos(k2);
        double* v = &pv[3 * (k1 * (n0 + 2) + k2)];
        v[0] = std::sin(tp) * std::cos(pp);
        v[1] = std::sin(tp) * std::sin(pp);
        v[2] = std::cos(tp);
      }
    cudaMemcpy(s->pvec.p, pv.data(), pv.size() * sizeof(double), cudaMemcpyHostToDevice);
    for (int which = 0; which < 2; ++which) {
      const int ns = which ? nf : p->nside_sht;
      std::vector<double> th(4 * ns - 1);
      for (int i = 1; i <= 4 * ns - 1; ++i) {
        const Ring r = ring_geom(ns, i);
        th[i - 1] = std::atan2(r.s, r.z);
      }
      cudaMemcpy(which ? s->ring_th_fine.p : s->ring_th_sht.p, th.data(), th.size() * sizeof(double),
                 cudaMemcpyHostToDevice);
    }
  }
  const int nc = s->sizes.back();
  const size_t ns2 = 12ull * p->nside_sht * p->nside_sht;
  if (ok && s->partial) {
    ok = alloc(s->slot_bundle, sizeof(int32_t) * s->npatch) && alloc(s->bundle_slot, sizeof(int32_t) * nbund) &&
         alloc(s->outside, sizeof(unsigned long long));
    if (ok) {
      cudaMemcpy(s->slot_bundle.p, domain, sizeof(int32_t) * s->npatch, cudaMemcpyHostToDevice);
      cudaMemcpy(s->bundle_slot.p, bslot.data(), sizeof(int32_t) * nbund, cudaMemcpyHostToDevice);
      cudaMemset(s->outside.p, 0, sizeof(unsigned long long));
    }
  }
  ok = ok && alloc(s->rot, 9 * sizeof(double) * s->npatch) && alloc(s->coarse_inv, sizeof(double) * nc * nc * nc * nc) &&
       alloc(s->coarse_inv32, sizeof(float) * nc * nc * nc * nc) &&
       alloc(s->tau2, sizeof(double) * s->npatch) &&
       alloc(s->gc, sizeof(double) * s->npatch * 4 * (s->nlev > 1 ? s->sizes[1] : 1)) &&
       alloc(s->psi_sht, sizeof(double) * ns2) && alloc(s->kappa_sht, sizeof(double) * ns2) &&
       alloc(s->norms, sizeof(double) * s->npatch) && alloc(s->ratio, sizeof(double));
  if (!ok) {
    delete s;
    return set_err(ctx, CLC_ENOMEM, "MG allocation failed");
  }
  // dense coarsest operator (interior unknowns; boundary terms excluded)
  {
    const double hc = s->h * (p->ncell / nc);
    LevelCoef lc = level_coef(nc, hc);
    const int nn = nc * nc;
    std::vector<double> A((size_t)nn * nn, 0.0);
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < nc; ++j) {
        const int r = i * nc + j;
        A[(size_t)r * nn + r] = -1.0 / lc.invd[(size_t)i * nc + j];
        if (i + 1 < nc) A[(size_t)r * nn + r + nc] += lc.coef[i];
        if (i > 0) A[(size_t)r * nn + r - nc] += lc.coef[nc + i];
        if (j + 1 < nc) A[(size_t)r * nn + r + 1] += lc.coef[2 * nc + i];
        if (j > 0) A[(size_t)r * nn + r - 1] += lc.coef[2 * nc + i];
      }
    if (!invert(A, nn)) {
      delete s;
      return set_err(ctx, CLC_ECUDA, "coarsest MG operator is singular");
    }
    cudaMemcpy(s->coarse_inv.p, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<float> A32(A.begin(), A.end());
    cudaMemcpy(s->coarse_inv32.p, A32.data(), A32.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  CLC_LAUNCH(ctx, "k_mg_rotations", k_mg_rotations, (s->npatch + 127) / 128, 128, 0, p->nside_bundle, s->npatch,
             s->partial ? (const int32_t*)s->slot_bundle.p : nullptr, (double*)s->rot.p);
  // interpolation plans, if they fit with 4 GiB to spare
  {
    const size_t pr = (size_t)s->npatch * (n0 + 2) * (n0 + 2), pk = (size_t)s->npatch * n0 * n0;
    const size_t bytes = (pr + pk) * (sizeof(int4) + 4 * sizeof(double));
    size_t fb = 0, tb = 0;
    cudaMemGetInfo(&fb, &tb);
    const bool mx = p->precision == CLC_MIXED;
    const int64_t ns2 = 12ll * p->nside_sht * p->nside_sht, nf2 = 12ll * nf * nf;
    const size_t ffb = mx ? (pr + ns2 + nf2) * sizeof(float2) : 0;   // base, psi and kappa as float-float
    if (bytes + ffb + (4ull << 30) < fb && alloc(s->plan_psi_idx, pr * sizeof(int4)) &&
        alloc(s->plan_psi_w, pr * 4 * sizeof(double)) && alloc(s->plan_kap_idx, pk * sizeof(int4)) &&
        alloc(s->plan_kap_w, pk * 4 * sizeof(double)) &&
        (!mx || (alloc(s->base_ff, pr * sizeof(float2)) && alloc(s->psi_ff, ns2 * sizeof(float2)) &&
                 alloc(s->kap_ff, nf2 * sizeof(float2))))) {
      const dim3 blk(kBX, kBY);
      CLC_LAUNCH(ctx, "k_mg_plan", k_mg_plan, grid3(n0 + 2, n0 + 2, s->npatch), blk, 0, (int)n0, 1,
                 (const double*)s->rot.p, (const double*)s->pvec.p, p->nside_sht, (const double*)s->ring_th_sht.p,
                 (int)mx, (int4*)s->plan_psi_idx.p, (double4_32a*)s->plan_psi_w.p);
      CLC_LAUNCH(ctx, "k_mg_plan", k_mg_plan, grid3(n0, n0, s->npatch), blk, 0, (int)n0, 0, (const double*)s->rot.p,
                 (const double*)s->pvec.p, nf, (const double*)s->ring_th_fine.p, (int)mx, (int4*)s->plan_kap_idx.p,
                 (double4_32a*)s->plan_kap_w.p);
      s->plan = true;
    }
  }
  rc = launch_check(ctx, "k_mg_rotations / k_mg_plan");
  if (rc) {
    delete s;
    return rc;
  }
  *out = s;
  return CLC_OK;
}

extern "C" int clc_solution_create(clc_ctx* ctx, int nf, const clc_mg_params* p, clc_plane_solution** out) {
  return solution_create(ctx, nf, p, nullptr, 0, out);
}

extern "C" int clc_solution_create_domain(clc_ctx* ctx, int nf, const clc_mg_params* p, const int32_t* bundles_host,
                                          int nbundles, clc_plane_solution** out) {
  if (!bundles_host) return ctx ? set_err(ctx, CLC_EINVAL, "clc_solution_create_domain: null bundle list") : CLC_EINVAL;
  return solution_create(ctx, nf, p, bundles_host, nbundles, out);
}

extern "C" int clc_solution_domain(const clc_plane_solution* s, int* npatch_host, int64_t* outside_host) {
  if (!s || !s->ctx) return CLC_EINVAL;
  if (npatch_host) *npatch_host = s->npatch;
  if (outside_host) {
    *outside_host = 0;
    if (s->partial) {
      unsigned long long v = 0;
      int rc = cuda_check(s->ctx, cudaStreamSynchronize(s->ctx->stream), "domain sync");
      if (rc) return rc;
      rc = cuda_check(s->ctx, cudaMemcpy(&v, s->outside.p, sizeof(v), cudaMemcpyDeviceToHost), "outside count");
      if (rc) return rc;
      *outside_host = (int64_t)v;
    }
  }
  return CLC_OK;
}

extern "C" int clc_solution_destroy(clc_plane_solution* s) {
  if (!s) return CLC_EINVAL;
  if (s->ctx) cudaStreamSynchronize(s->ctx->stream);
  delete s;
  return CLC_OK;
}

extern "C" int clc_solution_info(const clc_plane_solution* s, int* cycles, double* residual) {
  if (!s) return CLC_EINVAL;
  if (cycles) *cycles = s->cycles;
  if (residual) *residual = s->residual;
  return CLC_OK;
}

extern "C" int clc_poisson_shtmg(clc_ctx* ctx, const double* kappa_fine, int nf, const clc_mg_params* p,
                                 clc_plane_solution* s, const clc_derivs* out) {
  if (!ctx) return CLC_EINVAL;
  int rc = check_params(ctx, nf, p);
  if (rc) return rc;
  if (!s || !kappa_fine) return set_err(ctx, CLC_EINVAL, "clc_poisson_shtmg: null pointer");
  if (s->nside_fine != nf || s->p.nside_bundle != p->nside_bundle || s->p.ncell != p->ncell ||
      s->p.precision != p->precision || s->p.nside_sht != p->nside_sht)
    return set_err(ctx, CLC_EINVAL, "clc_poisson_shtmg: solution was created for other parameters");
  cudaSetDevice(ctx->device);
  s->p = *p;
  if (s->partial) cudaMemsetAsync(s->outside.p, 0, sizeof(unsigned long long), ctx->stream);
  // global SHT step on kappa binned at the SHT resolution
  if ((rc = clc_degrade(ctx, kappa_fine, nf, (double*)s->kappa_sht.p, p->nside_sht))) return rc;
  if ((rc = clc_poisson_sht(ctx, (const double*)s->kappa_sht.p, p->nside_sht, p->lmax, CLC_FP64,
                            (double*)s->psi_sht.p, nullptr)))
    return rc;
  int st;
  if (p->precision == CLC_MIXED) {
    MG<float> mg{s, ctx, true};
    if ((rc = mg.setup(kappa_fine))) return rc;
    st = mg.solve_mixed();
  } else if (p->precision == CLC_FP32) {
    MG<float> mg{s, ctx};
    if ((rc = mg.setup(kappa_fine))) return rc;
    st = mg.solve();
  } else {
    MG<double> mg{s, ctx};
    if ((rc = mg.setup(kappa_fine))) return rc;
    st = mg.solve();
  }
  if (st != CLC_OK && st != CLC_ENOTCONVERGED) return st;
  if (out && (out->a_th || out->a_ph || out->u_tt || out->u_pp || out->u_tp)) {
    const int64_t np = 12ll * nf * nf;
    CLC_LAUNCH(ctx, "k_fields_at_pixels", k_fields_at_pixels, blocks_for(ctx, np, 128), 128, 0, mg_view(s), nf,
               p->nside_bundle, out->a_th, out->a_ph, out->u_tt, out->u_pp, out->u_tp);
    if ((rc = launch_check(ctx, "k_fields_at_pixels"))) return rc;
  }
  return st;
}

extern "C" int clc_lens_derivs(clc_ctx* ctx, const clc_plane_solution* s, const double* z, const double* phi,
                               const int32_t* bundle, int64_t n, const clc_derivs* out) {
  if (!ctx) return CLC_EINVAL;
  if (!s || n < 0 || !out) return set_err(ctx, CLC_EINVAL, "clc_lens_derivs: bad arguments");
  if (n == 0) return CLC_OK;
  if (!z || !phi) return set_err(ctx, CLC_EINVAL, "clc_lens_derivs: null positions");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_fields_at_points", k_fields_at_points, blocks_for(ctx, n, 128), 128, 0, mg_view(s), z, phi,
             bundle, n, s->p.nside_bundle, out->a_th, out->a_ph, out->u_tt, out->u_pp, out->u_tp);
  return launch_check(ctx, "k_fields_at_points");
}
