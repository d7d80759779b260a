// Measured ALU peaks of the device (measurement only; no counterpart in the
// paper): the roofline denominators of the FP32 sweep kernels and of the
// FP64 apply.  A register-only kernel runs kChains independent multiply-add
// chains per thread on every SM and is timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/sgdg.h"

namespace {

constexpr int kChains = 8;      // independent chains per thread (hides the FMA latency)
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;   // one multiply-add, 2 flops
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) out[blockIdx.x * kThreads + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
sgdg_status run(int device, int iters, double* gflops, double* ms_out) {
  if (cudaSetDevice(device) != cudaSuccess) return SGDG_ECUDA;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SGDG_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kThreads, 0) != cudaSuccess)
    return SGDG_ECUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return SGDG_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_peak<T><<<blocks, kThreads>>>(iters / 8 + 1, a, b, out);   // warm-up
  float best = 0.0f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, kThreads>>>(iters, a, b, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0 || ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return SGDG_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *gflops = flops / (best * 1e-3) / 1e9;
  if (ms_out) *ms_out = best;
  return SGDG_OK;
}

}  // namespace

extern "C" sgdg_status sgdg_alu_peak(int device, int precision, int iters, double* gflops, double* ms) {
  if (!gflops || iters < 1) return SGDG_EINVAL;
  if (precision == SGDG_FP64) return run<double>(device, iters, gflops, ms);
  if (precision == SGDG_MIXED_FP32) return run<float>(device, iters, gflops, ms);
  return SGDG_EINVAL;
}
