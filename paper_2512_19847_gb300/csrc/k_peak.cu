// FMA-chain throughput probe: the measured FP64 (and FP32) arithmetic peak
// that the FP64 form's roofline divides by.  Every thread runs eight
// independent fused multiply-add chains a <- a * b + c (enough independent
// instructions in flight to keep the pipe busy), so the kernel issues nothing
// but FMAs; a never-true comparison of the chains' sum keeps them live.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ap_dvm.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

// Target of the never-taken store (64 slots per type).
__device__ double g_sink64[64];
__device__ float g_sink32[64];

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T b, T c, int iters, T* sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1.25e30)) sink[blockIdx.x & 63] = s;   // a -> c/(1 - b) = 1: never taken
}

template <typename T>
ap_dvm_status run(int iters, int reps, cudaStream_t stream, double* tflops, double* ms_per_launch) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AP_DVM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AP_DVM_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0) != cudaSuccess)
    return AP_DVM_ERR_CUDA;
  const int grid = std::max(1, per_sm) * sms;
  const T b = T(0.999999), c = T(1e-6);
  T* sink = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&sink), sizeof(T) == 8 ? (const void*)&g_sink64 : (const void*)&g_sink32) !=
      cudaSuccess)
    return AP_DVM_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AP_DVM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return AP_DVM_ERR_CUDA; }
  ap_dvm_status st = AP_DVM_OK;
  k_fma_chains<T><<<grid, kThreads, 0, stream>>>(b, c, iters, sink);   // warm-up
  cudaEventRecord(e0, stream);
  for (int r = 0; r < reps; ++r) k_fma_chains<T><<<grid, kThreads, 0, stream>>>(b, c, iters, sink);
  cudaEventRecord(e1, stream);
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    st = AP_DVM_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * kThreads * (double)grid;   // 2 per FMA
  *ms_per_launch = ms / reps;
  *tflops = flops * reps / (ms * 1e-3) / 1e12;
  return AP_DVM_OK;
}

}  // namespace

extern "C" ap_dvm_status ap_dvm_fma_peak(int precision, int iters, int reps, void* cuda_stream, double* tflops,
                                        double* ms_per_launch) {
  if (!tflops || !ms_per_launch || iters < 1 || reps < 1) return AP_DVM_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (precision == AP_DVM_FP64) return run<double>(iters, reps, s, tflops, ms_per_launch);
  if (precision == AP_DVM_FP32_DEV) return run<float>(iters, reps, s, tflops, ms_per_launch);
  return AP_DVM_ERR_ARG;
}
