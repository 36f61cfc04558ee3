// lmep_peak.cu -- FMA-chain microbenchmark for the FP64 and FP32 pipe peaks.
//
// Every thread runs 8 independent FMA chains a <- a * x + y (x = 1 - 2^-10,
// y = 2^-10, so every chain converges to 1 and never overflows); the grid
// fills every SM.  Achieved FLOP/s = 2 * FMAs / elapsed time (CUDA events,
// after one warm-up launch).  This is the denominator of the "alu" roofline
// of the expm kernels.
#include <cuda_runtime.h>

#include "lmep_internal.h"

namespace lmep {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters) {
  const T x = T(1) - T(1.0 / 1024), y = T(1.0 / 1024);
  T a0 = T(threadIdx.x) * T(1e-3), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0 = fma(a0, x, y); a1 = fma(a1, x, y); a2 = fma(a2, x, y); a3 = fma(a3, x, y);
      a4 = fma(a4, x, y); a5 = fma(a5, x, y); a6 = fma(a6, x, y); a7 = fma(a7, x, y);
    }
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == T(-12345)) out[blockIdx.x] = s;  // keeps the chains alive
}

template <typename T>
static cudaError_t run_peak(int iters, double* flops) {
  const int sms = device_info().sms;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks);
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k_fma_chain<T><<<blocks, threads>>>(out, iters / 8);
  cudaEventRecord(a);
  k_fma_chain<T><<<blocks, threads>>>(out, iters);
  cudaEventRecord(b);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double fmas = double(blocks) * threads * double(iters) * 4.0 * 8.0;
  *flops = 2.0 * fmas / (double(ms) * 1e-3);
  return cudaGetLastError();
}

cudaError_t fma_peak(bool fp32, double* flops) {
  return fp32 ? run_peak<float>(40000, flops) : run_peak<double>(1000, flops);
}

}  // namespace lmep
