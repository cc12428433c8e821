// Diagnostics of the library's error paths.  The pipelined kernels (the
// tensor-core Legendre contractions, the MG band kernels, the split GEMM)
// wait on mbarriers with a poll limit and record a timeout in the context's
// device error word instead of spinning forever; this entry point runs the
// same bounded wait on an mbarrier that nothing ever completes, so that the
// timeout path can be exercised without a fault and without leaving any copy
// or MMA in flight.
#include "common.cuh"
#include "umma.cuh"

namespace clc {

__global__ void k_bounded_wait(long long polls, int* d_err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    umma::mbar_init(&bar, 1);   // one arrival expected; none ever comes
    umma::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = umma::mbar_wait(&bar, 0, polls);
    if (!ok) record_error(d_err, kDevTimeout);
  }
}

}  // namespace clc

using namespace clc;

extern "C" int clc_diag_bounded_wait(clc_ctx* ctx, int64_t polls) {
  if (!ctx) return CLC_EINVAL;
  if (polls < 1 || polls > (1ll << 20)) return set_err(ctx, CLC_EINVAL, "clc_diag_bounded_wait: polls in [1, 2^20]");
  cudaSetDevice(ctx->device);
  CLC_LAUNCH(ctx, "k_bounded_wait", k_bounded_wait, 1, 32, 0, (long long)polls, ctx->d_err);
  return launch_check(ctx, "k_bounded_wait");
}
