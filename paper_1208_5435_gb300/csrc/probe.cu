// Measured FP32 FMA throughput of the GPU: the denominator of the float32 ALU roofline that
// the benchmark reports beside HBM for the shared-memory FFT chain (not in the paper).
#include <cuda_runtime.h>

#include "internal.h"

namespace mfipm {
namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (covers the FMA latency)
constexpr int kProbeThreads = 256;
constexpr int kBlocksPerSm = 4;  // 32 resident warps per SM

__global__ void __launch_bounds__(kProbeThreads) fma_peak_kernel(float* out, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (out && s == -1.0f) out[blockIdx.x] = s;  // never true (the chains stay positive); keeps them live
}

}  // namespace
}  // namespace mfipm

namespace mfipm {

// Best of three timed launches (after one warm-up) of the FMA loop on every SM.
cudaError_t measure_fp32_fma_peak(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((err = cudaEventCreate(&e0)) != cudaSuccess) return err;
  if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  const int blocks = sms * kBlocksPerSm, iters = 1 << 15;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    fma_peak_kernel<<<blocks, kProbeThreads, 0, st>>>(nullptr, iters, 0.99999994f, 1e-7f);
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace mfipm
