// compsum.cuh -- compensated double sums shared by the mass kernels (dgswem_mass) and the
// allocation-free mass sums (dgswem_mass_noalloc): Neumaier's step within a thread, the same step
// when two partial sums are combined, and a block reduction in a fixed tree order, so that every
// sum is bitwise reproducible.
#pragma once

namespace dg {

struct Comp {
  double s, c;  // running sum and its accumulated rounding error
};

// Neumaier (1974): add x to (s, c), keeping the rounding error of s + x in c.
__device__ __forceinline__ void comp_add(Comp &a, double x) {
  const double t = a.s + x;
  a.c += fabs(a.s) >= fabs(x) ? (a.s - t) + x : (x - t) + a.s;
  a.s = t;
}
__device__ __forceinline__ Comp comp_merge(Comp a, Comp b) {
  comp_add(a, b.s);
  a.c += b.c;
  return a;
}

// Combine the THREADS threads' pairs (a, b) of a block in a fixed binary tree; thread 0 returns
// with the block's pairs in a and b (the other threads' a, b are unspecified).  Call with the
// whole block.
template <int THREADS>
__device__ __forceinline__ void comp_block_reduce(Comp &a, Comp &b) {
  __shared__ Comp sa[THREADS], sb[THREADS];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] = comp_merge(sa[threadIdx.x], sa[threadIdx.x + w]);
      sb[threadIdx.x] = comp_merge(sb[threadIdx.x], sb[threadIdx.x + w]);
    }
    __syncthreads();
  }
  a = sa[0];
  b = sb[0];
}

}  // namespace dg
