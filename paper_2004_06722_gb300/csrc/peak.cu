// Measured FMA throughput of the current device (FP64 and FP32), the
// denominator of the arithmetic roofline of the element kernels: on GB300 the
// FP64 operators are bound by the FP64 FMA pipe, not by HBM bandwidth.  Also
// the throughput of warp-level MMA instructions (FP64, TF32, BF16), which
// decides whether the element contractions (small dense matrix products,
// Sec. 5, Eqs. (29)-(33)) could gain from the tensor cores.
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

// ---- warp-level MMA (mma.sync) throughput: FP64 m8n8k4, TF32 m16n8k8, BF16 m16n8k16.
// Each warp keeps kChains independent accumulator tiles and issues kUnroll x kChains
// MMAs per loop step; flops = 2 m n k per MMA.
constexpr int kMmaChains = 4;

__device__ __forceinline__ void mma_f64(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) mma_chain_kernel(float* sink, int iters) {
  const unsigned lane = threadIdx.x & 31u;
  if constexpr (KIND == 0) {
    double c[kMmaChains][2];
    const double a = 1e-3 * double(lane), b = 0.999;
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) c[k][0] = c[k][1] = double(k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kMmaChains; ++k) mma_f64(c[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) s += c[k][0] + c[k][1];
    if (s == -1.0) sink[blockIdx.x] = float(s);
  } else {
    float c[kMmaChains][4];
    // small operands (tf32 / bf16 bit patterns of values near 1e-3) keep the sums bounded
    const unsigned av = KIND == 1 ? 0x3a800000u + lane : 0x3a803a80u + lane;
    const unsigned a[4] = {av, av, av, av}, b[2] = {av, av};
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) c[k][0] = c[k][1] = c[k][2] = c[k][3] = float(k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kMmaChains; ++k) {
          if constexpr (KIND == 1) mma_tf32(c[k], a, b);
          else mma_bf16(c[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMmaChains; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    if (s == -1.0f) sink[blockIdx.x] = s;
  }
}

template <int KIND>
cudaError_t time_mma(int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * kBlocksPerSm;
  float* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(float) * blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    mma_chain_kernel<KIND><<<blocks, kThreads, 0, s>>>(sink, iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) {
    const double mnk = KIND == 0 ? 8.0 * 8 * 4 : (KIND == 1 ? 16.0 * 8 * 8 : 16.0 * 8 * 16);
    const double warps = double(blocks) * (kThreads / 32);
    const double flops = 2.0 * mnk * kMmaChains * kUnroll * double(iters) * warps;
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

extern "C" ceedbp_status ceedbp_mma_peak(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return CEEDBP_EINVAL;
  cudaError_t e;
  if (kind == 0) e = ceedbp::time_mma<0>(1024, tflops);
  else if (kind == 1) e = ceedbp::time_mma<1>(4096, tflops);
  else e = ceedbp::time_mma<2>(4096, tflops);
  if (e != cudaSuccess) {
    ceedbp::set_thread_error(std::string("ceedbp_mma_peak: ") + cudaGetErrorString(e));
    return CEEDBP_ECUDA;
  }
  return CEEDBP_OK;
}

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
