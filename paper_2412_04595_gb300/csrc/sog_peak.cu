// Measured arithmetic peaks of the device (sog_measure_fma_peak in sog.h):
// the FP32 or FP64 fused multiply-add rate that the ALU-bound steps of the
// method (near field, gridding, gathering) are reported against.
#include <cuda_runtime.h>

#include "sog_internal.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;  // independent FMA chains per thread

// Each thread runs kPeakChains independent chains of `iters` FMAs, a = a * b + c
// with b slightly below one, so the values stay finite; the sum is written only
// when it equals a sentinel no input produces, which keeps the work live.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T b, T c, T* __restrict__ sink) {
  T a[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) a[k] = T(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += a[k];
  if (s == T(-12345.0)) *sink = s;
}

template <typename T>
sog_status measure(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SOG_ERR_CUDA;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return SOG_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 8 * sms;  // 2048 threads per SM
  const int iters = sizeof(T) == 4 ? 8192 : 512;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, kPeakThreads>>>(iters, T(0.999999), T(1e-3), sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return SOG_ERR_CUDA;
  const double flop = 2.0 * kPeakChains * (double)iters * blocks * kPeakThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return SOG_OK;
}

}  // namespace

extern "C" sog_status sog_measure_fma_peak(int32_t precision, double* tflops) {
  if (!tflops) return SOG_ERR_ARG;
  if (precision == SOG_PREC_FP64) return measure<double>(tflops);
  if (precision == SOG_PREC_MIXED) return measure<float>(tflops);
  return SOG_ERR_ARG;
}
