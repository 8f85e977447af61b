// Throughput probe of the FP64 FMA pipe (the roofline of the FP64 arithmetic in recompression):
// every SM runs warps of independent FMA chains long enough (~10 ms) to time with CUDA events.
#include "clr_internal.h"

namespace clr {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) fp64_fma_kernel(double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a = 1, b = 0 in practice: the sum is exact and never 0.5, so no store happens, but the
  // compiler cannot drop the chains
  if (s == 0.5) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace clr

extern "C" int clr_probe_fp64_rate(int device, double* tflops) {
  if (!tflops) return CLR_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return CLR_ECUDA;
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
  const int blocks = n_sm * 8, threads = 256;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * threads) != cudaSuccess) return CLR_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  clr::fp64_fma_kernel<<<blocks, threads>>>(1.0, 0.0, sink);  // warm-up
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) clr::fp64_fma_kernel<<<blocks, threads>>>(1.0, 0.0, sink);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess || !(ms > 0.f)) return CLR_ECUDA;
  const double fmas = (double)reps * blocks * threads * clr::kChains * clr::kIters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return CLR_OK;
}
