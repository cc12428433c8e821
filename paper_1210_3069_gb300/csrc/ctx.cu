// Context management, error reporting and scratch memory of the C ABI.
#include <cstring>

#include "common.cuh"

namespace clc {

int set_err(clc_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_check(clc_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CLC_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_err(ctx, CLC_ENOMEM, m);
  return set_err(ctx, CLC_ECUDA, m);
}

int launch_check(clc_ctx* ctx, const char* what) {
  if (ctx->launch_err != cudaSuccess) {
    const cudaError_t e = ctx->launch_err;
    const std::string m = std::string(what) + " (" + ctx->launch_err_kernel + ")";
    ctx->launch_err = cudaSuccess;
    cudaGetLastError();
    return cuda_check(ctx, e, m.c_str());
  }
  return cuda_check(ctx, cudaGetLastError(), what);
}

cudaEvent_t pool_event(clc_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

static void prof_reset(clc_ctx* ctx) {
  for (auto& kv : ctx->prof_ev)
    for (auto& pr : kv.second) {
      ctx->ev_pool.push_back(pr.first);
      ctx->ev_pool.push_back(pr.second);
    }
  ctx->prof_ev.clear();
}

void* scratch(clc_ctx* ctx, int slot, size_t bytes) {
  Buffer& b = ctx->scratch[slot];
  if (b.bytes >= bytes && b.p) return b.p;
  if (b.p) {
    // the old buffer may still be in use by enqueued kernels
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    set_err(ctx, CLC_ENOMEM, "scratch allocation of " + std::to_string(want) + " bytes failed");
    return nullptr;
  }
  b.bytes = want;
  return b.p;
}

bool valid_nside(int nside) { return nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0; }

int num_sms(clc_ctx* ctx) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device);
  return v > 0 ? v : 1;
}

}  // namespace clc

using namespace clc;

extern "C" int clc_create(clc_ctx** out, int device, void* stream) {
  if (!out) return CLC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return CLC_EINVAL;
  }
  clc_ctx* ctx = new clc_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  int rc = cuda_check(ctx, cudaSetDevice(device), "cudaSetDevice");
  if (rc == CLC_OK) rc = cuda_check(ctx, cudaMalloc(&ctx->d_err, 16), "cudaMalloc(error word)");
  if (rc == CLC_OK) rc = cuda_check(ctx, cudaMemsetAsync(ctx->d_err, 0, 16, ctx->stream), "memset");
  if (rc != CLC_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return CLC_OK;
}

extern "C" int clc_destroy(clc_ctx* ctx) {
  if (!ctx) return CLC_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  prof_reset(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->tc_batches.clear();
  ctx->tc_tables.clear();
  ctx->fft_plans.clear();
  ctx->leg_tables.clear();
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
  return CLC_OK;
}

extern "C" int clc_release_caches(clc_ctx* ctx) {
  if (!ctx) return CLC_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  ctx->fft_plans.clear();
  ctx->tc_batches.clear();
  ctx->leg_tables.clear();
  ctx->tc_tables.clear();
  return CLC_OK;
}

extern "C" int clc_sync(clc_ctx* ctx) {
  if (!ctx) return CLC_EINVAL;
  int rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (rc != CLC_OK) return rc;
  int h = 0;
  rc = cuda_check(ctx, cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (rc != CLC_OK) return rc;
  if (h != kDevOk) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (h == kDevTimeout) return set_err(ctx, CLC_ETIMEOUT, "a bounded device-side wait gave up");
    if (h == kDevNonFinite) return set_err(ctx, CLC_ECUDA, "non-finite value detected on the device");
    return set_err(ctx, CLC_ECUDA, "device-side index check failed (code " + std::to_string(h) + ")");
  }
  return CLC_OK;
}

extern "C" const char* clc_last_error(const clc_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

extern "C" int clc_profile(clc_ctx* ctx, int enable) {
  if (!ctx) return CLC_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  if (enable) prof_reset(ctx);
  ctx->prof = enable != 0;
  return CLC_OK;
}

extern "C" int clc_profile_query(clc_ctx* ctx, const char* name, int64_t* launches, double* total_ms) {
  if (!ctx || !name) return CLC_EINVAL;
  int rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync");
  if (rc) return rc;
  int64_t n = 0;
  double ms = 0.0;
  auto it = ctx->prof_ev.find(name);
  if (it != ctx->prof_ev.end())
    for (auto& pr : it->second) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) {
        ms += t;
        ++n;
      }
    }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return CLC_OK;
}

extern "C" int64_t clc_launch_count(const clc_ctx* ctx) { return ctx ? ctx->launches : -1; }
