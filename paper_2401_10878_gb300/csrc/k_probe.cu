// FP32 FFMA issue rate of the device: the measured counterpart of the
// roofline's derived peak (SMs x 128 FP32 lanes x clock).  Every thread runs
// eight independent FFMA chains for a fixed number of iterations (no waits,
// fixed trip counts); the grid fills every SM with eight 256-thread blocks.
#include <cuda_runtime.h>

#include "../../include/contact.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_ffma_rate(float* __restrict__ out, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = static_cast<float>(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" contact_status contact_fp32_ffma_rate(int32_t iters, double* ffma_per_s) {
  if (ffma_per_s == nullptr || iters < 1 || iters > (1 << 20)) return CONTACT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return CONTACT_ECUDA;
  const int blocks = 8 * sms, threads = 256;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return CONTACT_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_ffma_rate<<<blocks, threads>>>(out, iters, 0.999999f, 1e-7f);   // warm-up (clocks, code)
    cudaEventRecord(e0);
    k_ffma_rate<<<blocks, threads>>>(out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.f)) return CONTACT_ECUDA;
  *ffma_per_s = static_cast<double>(blocks) * threads * iters * 16.0 * kChains / (ms * 1e-3);
  return CONTACT_OK;
}
