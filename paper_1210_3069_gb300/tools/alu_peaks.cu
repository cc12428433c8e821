// FP64 / FP32 fused-multiply-add throughput and device-copy bandwidth of the
// GPU, timed with CUDA events (the ALU denominators of the rooflines).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_peaks alu_peaks.cu && ./alu_peaks
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  // eight independent FMA chains per thread keep the pipe busy
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void copy16(const double2* __restrict__ a, double2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  void* out = nullptr;
  cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0;
  for (int rep = 0; rep < 3; ++rep) {
    fma_chains<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
    cudaEventRecord(e0);
    fma_chains<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 fma: %.3f ms  %.3f TFLOP/s\n", ms, 2.0 * 8 * iters * (double)blocks * threads / ms / 1e9);
    fma_chains<float><<<blocks, threads>>>((float*)out, iters * 8, 0.999999f, 1e-7f);
    cudaEventRecord(e0);
    fma_chains<float><<<blocks, threads>>>((float*)out, iters * 8, 0.999999f, 1e-7f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32 fma: %.3f ms  %.3f TFLOP/s\n", ms, 2.0 * 8 * iters * 8 * (double)blocks * threads / ms / 1e9);
  }
  const size_t n = (size_t)1 << 28;  // 4 GiB per buffer
  double2 *a = nullptr, *b = nullptr;
  cudaMalloc(&a, n * sizeof(double2));
  cudaMalloc(&b, n * sizeof(double2));
  cudaMemset(a, 0, n * sizeof(double2));
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    copy16<<<sms * 4, 512>>>(a, b, n);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("copy: %.3f ms  %.1f GB/s (read + write)\n", ms, 2.0 * n * sizeof(double2) / ms / 1e6);
  }
  printf("status: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
