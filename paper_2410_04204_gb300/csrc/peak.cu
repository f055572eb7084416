// FP64 roofline denominator: a kernel of independent DFMA chains on every SM.
#include <algorithm>

#include "tgba_internal.h"

namespace tgba {
namespace {

__global__ void __launch_bounds__(256) dfma_chains(double* out, int iters, double a, double c) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, c); x1 = fma(x1, a, c); x2 = fma(x2, a, c); x3 = fma(x3, a, c);
    x4 = fma(x4, a, c); x5 = fma(x5, a, c); x6 = fma(x6, a, c); x7 = fma(x7, a, c);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

tgba_status fp64_peak(int reps, double* gflops) {
  int dev = 0, sms = 0;
  TGBA_CUDA(cudaGetDevice(&dev));
  TGBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 4, iters = 4096;
  double* d = nullptr;
  TGBA_CUDA(cudaMalloc(&d, sizeof(double) * threads * blocks));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < reps + 1; ++r) {
    cudaEventRecord(e0);
    dfma_chains<<<blocks, threads>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, ms);   // first launch is a warm-up
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess) return cuda_fail(err, "dfma_chains");
  *gflops = 2.0 * 8.0 * iters * (double)threads * blocks / (best * 1e-3) / 1e9;
  return TGBA_OK;
}

}  // namespace tgba
