// Measured FMA throughput of the current device (FP64 and FP32), the
// denominator of the arithmetic roofline of the element kernels: on GB300 the
// FP64 operators are bound by the FP64 FMA pipe, not by HBM bandwidth.
//
// Every thread runs kChains independent dependent chains x <- x a + b (one FMA
// each, a just below 1 so the values stay bounded) for `iters` x kUnroll
// steps; the grid fills every SM with kBlocksPerSm blocks.  Work = 2 flops per
// FMA; time = CUDA events around the launch, best of several launches after a
// warm-up.  The SM count comes from the device properties.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace ceedbp {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-1)) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

template <typename T>
cudaError_t time_fma(int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * kBlocksPerSm;
  T* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(T) * blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(sink, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;  // the first launch is the warm-up
  }
  if (e == cudaSuccess) {
    const double flops = 2.0 * kChains * kUnroll * double(iters) * blocks * kThreads;
    *tflops = flops / (double(best) * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  return e;
}

}  // namespace
}  // namespace ceedbp

extern "C" ceedbp_status ceedbp_fma_peak(int fp64, double* tflops, int* sm_count) {
  if (!tflops) return CEEDBP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CEEDBP_ECUDA;
  if (sm_count) *sm_count = sms;
  // FP64 runs at a small fraction of the FP32 rate: fewer steps give a launch of similar length
  const cudaError_t e = fp64 ? ceedbp::time_fma<double>(2048, tflops) : ceedbp::time_fma<float>(65536, tflops);
  if (e != cudaSuccess) {
    ceedbp::set_thread_error(std::string("ceedbp_fma_peak: ") + cudaGetErrorString(e));
    return CEEDBP_ECUDA;
  }
  return CEEDBP_OK;
}
