// Split-precision tensor-core GEMM on tcgen05: D = A_hi B_hi^T + A_hi B_lo^T +
// A_lo B_hi^T with FP16 operands and FP32 accumulation in TMEM.  With
// x = x_hi + x_lo (x_hi = fp16(x), x_lo = fp16(x - x_hi)) this recovers a
// product of ~22-bit operands; the dropped lo*lo term is below the FP32
// accumulation error.  This is the contraction the mixed-precision Legendre
// transforms are built on; clc_gemm_f16x3 exposes it for direct testing.
//
// One CTA (4 warps) per 128-row tile of one batch entry.  Each K stage of 64
// stages the four operand tiles into shared memory in the 128-byte swizzled
// K-major layout, then one elected thread issues 4 x 3 MMAs (K = 16 each) and
// commits them to an mbarrier; the epilogue reads the accumulator rows of each
// warp's TMEM sub-partition.
#include "common.cuh"
#include "umma.cuh"

namespace clc {

constexpr long long kWaitPolls = 1ll << 26;

struct GemmArgs {
  const __half *a_hi, *a_lo, *b_hi, *b_lo;
  float* d;
  int M, N, K;
  long long sa, sb, sd;  // batch strides (elements)
};

__global__ void __launch_bounds__(128) k_gemm_f16x3(GemmArgs g, int* d_err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const uint32_t raw = umma::smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int N = g.N;
  uint8_t* sAh = base;
  uint8_t* sAl = sAh + 128 * 128;
  uint8_t* sBh = sAl + 128 * 128;
  uint8_t* sBl = sBh + ((N * 128 + 1023) & ~1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * 128;
  const int bz = blockIdx.y;
  const __half* Ah = g.a_hi + bz * g.sa;
  const __half* Al = g.a_lo + bz * g.sa;
  const __half* Bh = g.b_hi + bz * g.sb;
  const __half* Bl = g.b_lo + bz * g.sb;
  int ncols = 32;
  while (ncols < N) ncols <<= 1;
  if (threadIdx.x == 0) {
    umma::mbar_init(&mbar, 1);
    abort_flag = 0;
  }
  if (warp == 0) umma::tmem_alloc(&tmem_base, ncols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma::idesc_f16_f32(128, N);
  uint32_t phase = 0;
  for (int k0 = 0; k0 < g.K; k0 += 64) {
    // stage the operand tiles (16-byte chunks, swizzled)
    for (int t = threadIdx.x; t < 128 * 8; t += blockDim.x) {
      const int r = t >> 3, c = t & 7;
      uint4 vh = make_uint4(0, 0, 0, 0), vl = vh;
      if (row0 + r < g.M) {
        const size_t off = (size_t)(row0 + r) * g.K + k0 + c * 8;
        vh = *reinterpret_cast<const uint4*>(Ah + off);
        vl = *reinterpret_cast<const uint4*>(Al + off);
      }
      *reinterpret_cast<uint4*>(sAh + umma::sw128_offset(r, c)) = vh;
      *reinterpret_cast<uint4*>(sAl + umma::sw128_offset(r, c)) = vl;
    }
    for (int t = threadIdx.x; t < N * 8; t += blockDim.x) {
      const int r = t >> 3, c = t & 7;
      const size_t off = (size_t)r * g.K + k0 + c * 8;
      *reinterpret_cast<uint4*>(sBh + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Bh + off);
      *reinterpret_cast<uint4*>(sBl + umma::sw128_offset(r, c)) = *reinterpret_cast<const uint4*>(Bl + off);
    }
    umma::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma::fence_after_sync();
      const uint64_t dAh = umma::desc_sw128(umma::smem_u32(sAh)), dAl = umma::desc_sw128(umma::smem_u32(sAl));
      const uint64_t dBh = umma::desc_sw128(umma::smem_u32(sBh)), dBl = umma::desc_sw128(umma::smem_u32(sBl));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t adv = (uint64_t)(kk * 32) >> 4;   // 16 fp16 = 32 bytes along K
        umma::mma_f16(tmem, dAh + adv, dBh + adv, idesc, (k0 | kk) != 0);
        umma::mma_f16(tmem, dAh + adv, dBl + adv, idesc, 1);
        umma::mma_f16(tmem, dAl + adv, dBh + adv, idesc, 1);
      }
      umma::commit(&mbar);
    }
    // all threads wait for the MMAs before the tiles are overwritten
    if (!umma::mbar_wait(&mbar, phase, kWaitPolls)) {
      if (lane == 0) atomicCAS(d_err, 0, kDevTimeout);
      abort_flag = 1;
    }
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
  }
  umma::fence_after_sync();
  if (!abort_flag) {
    const int r = row0 + warp * 32 + lane;
    float* D = g.d + bz * g.sd;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < g.M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) D[(size_t)r * N + c0 + i] = v[i];
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

int gemm_f16x3(clc_ctx* ctx, const GemmArgs& g, int batch) {
  const int smem = 1024 + 2 * 128 * 128 + 2 * ((g.N * 128 + 1023) & ~1023);
  cudaFuncSetAttribute(k_gemm_f16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dim3 grid((g.M + 127) / 128, batch);
  CLC_LAUNCH(ctx, "k_gemm_f16x3", k_gemm_f16x3, grid, 128, smem, g, ctx->d_err);
  return launch_check(ctx, "k_gemm_f16x3");
}

}  // namespace clc

using namespace clc;

extern "C" int clc_gemm_f16x3(clc_ctx* ctx, const void* a_hi, const void* a_lo, const void* b_hi, const void* b_lo,
                              int M, int N, int K, int batch, float* d) {
  if (!ctx) return CLC_EINVAL;
  if (!a_hi || !a_lo || !b_hi || !b_lo || !d) return set_err(ctx, CLC_EINVAL, "clc_gemm_f16x3: null pointer");
  if (M < 1 || N < 16 || N > 256 || (N % 16) || K < 64 || (K % 64) || batch < 1 || batch > 65535)
    return set_err(ctx, CLC_EINVAL, "clc_gemm_f16x3: need M >= 1, N in [16, 256] multiple of 16, K multiple of 64");
  cudaSetDevice(ctx->device);
  GemmArgs g;
  g.a_hi = (const __half*)a_hi;
  g.a_lo = (const __half*)a_lo;
  g.b_hi = (const __half*)b_hi;
  g.b_lo = (const __half*)b_lo;
  g.d = d;
  g.M = M;
  g.N = N;
  g.K = K;
  g.sa = (long long)M * K;
  g.sb = (long long)N * K;
  g.sd = (long long)M * N;
  return gemm_f16x3(ctx, g, batch);
}
