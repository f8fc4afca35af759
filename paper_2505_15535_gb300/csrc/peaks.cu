// Measured FMA throughput of the device, the denominator of the apply kernels' ALU roofline.
//
// Every thread runs kChains independent FMA chains of kIters steps (x = x * a + b, with a and b
// chosen so that the values stay bounded), which keeps the FMA pipe of every SM busy: the
// dependent latency of one chain is hidden by the others and by the other warps.  The grid
// holds kBlocksPerSM blocks of 256 threads per SM.  The result is written only if it is
// non-zero, so that the compiler cannot drop the chains.
#include <cuda_runtime.h>

#include "internal.h"

namespace nhmf {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(12345.678)) sink[blockIdx.x] = s;
}

template <typename T>
nhmf_status measure(int sms, double* tflops) {
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&sink, sizeof(T) * sms * kBlocksPerSM);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // first repetition warms up
    cudaEventRecord(e0);
    k_fma_chains<T><<<sms * kBlocksPerSM, kThreads>>>(T(0.999), T(1e-4), sink);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? NHMF_ERR_OOM : NHMF_ERR_CUDA;
  const double flops = 2.0 * kChains * kIters * (double)kThreads * sms * kBlocksPerSM;
  *tflops = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
  return NHMF_OK;
}

}  // namespace
}  // namespace nhmf

extern "C" nhmf_status nhmf_measure_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != NHMF_FP64 && precision != NHMF_FP32)) return NHMF_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NHMF_ERR_CUDA;
  return precision == NHMF_FP64 ? nhmf::measure<double>(sms, tflops) : nhmf::measure<float>(sms, tflops);
}
