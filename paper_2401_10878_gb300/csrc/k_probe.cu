// FP32 FFMA and FP64 DFMA issue rates of the device: the measured
// counterparts of the roofline peaks (the node sweep's FP32 lanes, the
// all-FP64 form's FP64 pipe).  Every thread runs eight independent FMA chains
// for a fixed number of iterations (no waits, fixed trip counts); the grid
// fills every SM with eight 256-thread blocks.
#include <cuda_runtime.h>

#include "../../include/contact.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* __restrict__ out, int iters, T m, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = static_cast<T>(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
contact_status fma_rate(int32_t iters, double* per_s, T m, T c) {
  if (per_s == nullptr || iters < 1 || iters > (1 << 20)) return CONTACT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return CONTACT_ECUDA;
  const int blocks = 8 * sms, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return CONTACT_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fma_rate<T><<<blocks, threads>>>(out, iters, m, c);   // warm-up (clocks, code)
    cudaEventRecord(e0);
    k_fma_rate<T><<<blocks, threads>>>(out, iters, m, c);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.f)) return CONTACT_ECUDA;
  *per_s = static_cast<double>(blocks) * threads * iters * 16.0 * kChains / (ms * 1e-3);
  return CONTACT_OK;
}

}  // namespace

extern "C" contact_status contact_fp32_ffma_rate(int32_t iters, double* ffma_per_s) {
  return fma_rate<float>(iters, ffma_per_s, 0.999999f, 1e-7f);
}

extern "C" contact_status contact_fp64_dfma_rate(int32_t iters, double* dfma_per_s) {
  return fma_rate<double>(iters, dfma_per_s, 0.999999999, 1e-15);
}
