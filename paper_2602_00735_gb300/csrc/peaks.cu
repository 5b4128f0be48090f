// Arithmetic throughput of the FMA pipes on the current device (the ALU
// rooflines of the FP64-bound kernels: the complex128 apply, SpMV and
// Gram-Schmidt). Each thread runs kChains independent FMA chains of kIters
// steps on values that stay finite and that the compiler cannot fold (the
// coefficients come from kernel arguments); one result per thread is stored
// so that nothing is dead code. A grid of 8 CTAs of 256 threads per SM keeps
// every SM's pipes busy; the time is taken with CUDA events around the second
// of two launches.
#include "host.h"

namespace rp {

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(T a, T b, T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 4
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

template <typename T>
int measure(double* tflops) {
  int dev = 0, sms = 0;
  RP_CUDA(cudaGetDevice(&dev));
  RP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms;
  T* out = nullptr;
  int s = dalloc(&out, (size_t)blocks * kPeakThreads);
  if (s != RASPML_OK) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  // a = 0.5 keeps x + b bounded (x -> 2b); b from the argument list
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      k_fma_peak<T><<<blocks, kPeakThreads>>>((T)0.5, (T)0.25, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.f)) return RASPML_ECUDA;
  const double flops = 2.0 * blocks * kPeakThreads * (double)kIters * kChains;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return RASPML_OK;
}

}  // namespace

}  // namespace rp

extern "C" int ras_pml_fma_peak(int fp64, double* tflops) {
  if (!tflops) return RASPML_EBADARG;
  return fp64 ? rp::measure<double>(tflops) : rp::measure<float>(tflops);
}
