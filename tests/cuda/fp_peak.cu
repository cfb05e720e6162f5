// Test harness (compiled by tests/test_gpu_fp_peak.py): the GPU's double and single precision
// FMA throughput, measured with long independent FMA chains in every thread of a full grid.  The
// FP64 form's roofline uses the double figure as its arithmetic peak.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void k_fma(T *out, T a, T b, int iters) {
  // 8 independent chains per thread keep the FMA pipe busy; a and b are kernel arguments, so the
  // compiler cannot fold the loop
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(-1.2345)) out[0] = s;  // keeps the chains alive; never true for these inputs
}

template <typename T>
double run(int blocks, int threads, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<T><<<blocks, threads>>>(out, T(0.999999), T(1e-7), iters);  // warm-up
  cudaEventRecord(e0);
  k_fma<T><<<blocks, threads>>>(out, T(0.999999), T(1e-7), iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  return flops / (ms * 1e-3);
}

}  // namespace

// flops/s of FP64 (kind 0) or FP32 (kind 1) FMA chains over blocks x threads threads.
extern "C" double fp_peak(int kind, int blocks, int threads, int iters) {
  return kind == 0 ? run<double>(blocks, threads, iters) : run<float>(blocks, threads, iters);
}
