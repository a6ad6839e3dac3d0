// peak.cu -- FP32 fused-multiply-add throughput of the device, the peak the
// evaluation kernel's roofline is reported against (that kernel is bound by
// FP32 arithmetic, not by memory or tensor cores).  Not part of the paper's
// method.
//
// Every thread runs kChains independent FMA chains, so the FMA pipe is fed
// every cycle; a grid of resident CTAs covers every SM.  The chains'
// arithmetic (x <- x * a + b with a slightly below 1) stays finite for any
// length, and the result is stored only when it takes an impossible value, so
// the work cannot be removed.
#include <cuda_runtime.h>

#include "crgb_internal.cuh"

namespace crgb {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_ffma(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true: keeps the chains alive
}

}  // namespace

}  // namespace crgb

using namespace crgb;

extern "C" cr_status cr_measure_ffma(int32_t iters, float* tflops, float* ms, void* stream) {
  if (iters < 1 || !tflops) return set_error(CR_EINVAL, "cr_measure_ffma: iters < 1 or null output");
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma, kPeakThreads, 0);
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  const int grid = n_sm * (per_sm > 0 ? per_sm : 1);
  const cudaStream_t s = (cudaStream_t)stream;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, (size_t)grid * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_ffma<<<grid, kPeakThreads, 0, s>>>(iters / 8 + 1, 0.9999999f, 1e-7f, sink);  // warm-up
    cudaEventRecord(e0, s);
    k_ffma<<<grid, kPeakThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
  }
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return set_error(CR_ECUDA, cudaGetErrorString(e));
  const double flop = 2.0 * (double)grid * kPeakThreads * kChains * kUnroll * (double)iters;
  *tflops = (float)(flop / (t * 1e-3) / 1e12);
  if (ms) *ms = t;
  return CR_OK;
}
