// Test harness (compiled by tests/test_gpu_fp_helpers.py): runs the hand-written double-precision
// helpers of kernels.cuh -- the seeded reciprocal, reciprocal square root, square root and ratio,
// the integer-pipe double <-> float conversions and the exact halving -- next to CUDA's own
// operations on the same inputs, so that the test can compare them element by element.
#include "../../paper_2508_21208_gb300/csrc/kernels.cuh"

namespace {

// out[i * K + j]: result j for input i (see the comments per kind)
__global__ void k_fp(int kind, const double *x, const double *y, double *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i];
  double *o = out + (size_t)i * 4;
  switch (kind) {
    case 0:  // reciprocal: rcp_d, IEEE 1/x (correctly rounded)
      o[0] = dg::rcp_d(a);
      o[1] = __drcp_rn(a);
      break;
    case 1:  // square root: sqrt_d, IEEE sqrt (correctly rounded)
      o[0] = dg::sqrt_d(a);
      o[1] = __dsqrt_rn(a);
      break;
    case 2:  // reciprocal square root: rsqrt_d, CUDA's rsqrt
      o[0] = dg::rsqrt_d(a);
      o[1] = rsqrt(a);
      break;
    case 3:  // ratio y / x: ratio_t, IEEE divide (correctly rounded)
      o[0] = dg::ratio_t<double>(y[i], a);
      o[1] = __ddiv_rn(y[i], a);
      break;
    case 4: {  // double -> float: d2f, the hardware conversion (round to nearest even)
      o[0] = (double)dg::d2f(a);
      o[1] = (double)__double2float_rn(a);
      break;
    }
    case 5: {  // float -> double: f2d, the hardware conversion, for the float a rounds to
      const float f = __double2float_rn(a);
      o[0] = dg::f2d(f);
      o[1] = (double)f;
      break;
    }
    case 6:  // halving: half_exact, x * 0.5 (exact or round to nearest even below 2^-1021)
      o[0] = dg::half_exact(a);
      o[1] = __dmul_rn(a, 0.5);
      break;
  }
}

}  // namespace

extern "C" int fp_run(int kind, const double *x, const double *y, double *out, int n) {
  if (n <= 0) return 0;
  k_fp<<<(n + 255) / 256, 256>>>(kind, x, y, out, n);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
