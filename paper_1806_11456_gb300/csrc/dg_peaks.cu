// Measurement of the device's fused multiply-add rates in FP64 and FP32: the
// denominators of the roofline of the ALU-bound operator kernels (FP64 for
// the native arithmetic, FP32 for the double-float one).  Not part of the
// paper's method.
//
// Every thread runs kChains independent chains x = fma(x, a, b), so the FMA
// pipes see kChains independent instructions per thread between two
// dependent ones; a grid of 8 CTAs of 256 threads per SM keeps every
// scheduler busy.  The chains are summed and stored under a condition the
// compiler cannot prove false, so no FMA is removed.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "dg_internal.h"

namespace dg {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_rate(T* sink, int iters, T a, T b) {
  T x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == (T)-1) sink[blockIdx.x] = s;  // never true for these inputs (the chains tend to b / (1 - a) > 0)
}

// Best-of-`reps` rate of one precision in TFLOP/s (FMA = 2 flops).
template <typename T>
static int fma_rate(int grid, int iters, int reps, cudaStream_t st, double* tflops) {
  T* sink = nullptr;
  DG_CUDA_TRY(cudaMalloc(&sink, (size_t)grid * sizeof(T)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = DG_ECUDA;
  double best_ms = 1e300;
  for (int r = 0; r <= reps && rc == DG_OK; ++r) {  // r = 0 warms up
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = DG_ECUDA;
    k_fma_rate<T><<<grid, kPeakThreads, 0, st>>>(sink, iters, (T)0.999999, (T)1e-6);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      rc = DG_ECUDA;
    float ms = 0.f;
    if (rc == DG_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = DG_ECUDA;
    if (rc == DG_OK && r > 0) best_ms = std::min(best_ms, (double)ms);
  }
  if (rc != DG_OK) set_error("fma rate probe: CUDA error");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lock(device_sync_mutex());
    cudaFree(sink);
  }
  if (rc != DG_OK) return rc;
  const double flops = 2.0 * kPeakChains * kPeakUnroll * (double)iters * grid * kPeakThreads;
  *tflops = flops / (best_ms * 1e-3) / 1e12;
  return DG_OK;
}

int measure_fma_rates(double* fp64_tflops, double* fp32_tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  DG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 8 * std::max(1, sms);
  int rc = fma_rate<double>(grid, 400, 3, st, fp64_tflops);    // ~30 ms a launch at ~1.2 TFLOP/s
  if (rc == DG_OK) rc = fma_rate<float>(grid, 16000, 3, st, fp32_tflops);  // ~20 ms at ~70 TFLOP/s
  return rc;
}

}  // namespace dg
