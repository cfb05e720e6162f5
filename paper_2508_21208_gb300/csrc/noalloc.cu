// noalloc.cu -- dgswem_mass_noalloc: the compensated mass / volume sums of dgswem_mass for callers
// that may not allocate device memory.  Its block partials live in a fixed static device buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dgswem.h"
#include "compsum.cuh"

namespace {

using dg::Comp;
using dg::comp_add;
using dg::comp_block_reduce;
using dg::comp_merge;

constexpr int kThreads = 256;
constexpr int kPerBlock = kThreads * 8;  // elements summed by one block
constexpr int kMaxBlocks = (DGSWEM_NOALLOC_MAX_ELEMS + kPerBlock - 1) / kPerBlock;  // 32768
constexpr int kMaxDevices = 64;

// Four doubles (sum, compensation) x (anomaly, volume) per block: 1 MiB.  Host code must not
// pass this name to a kernel (on the host it is only a stand-in); it uses the address looked up
// by cudaGetSymbolAddress below.
static __device__ __align__(256) double g_partials[4 * kMaxBlocks];

std::mutex g_lock;
double *g_addr[kMaxDevices] = {};

__global__ void __launch_bounds__(kThreads) k_partials(const double *z, const double *area, const double *hb,
                                                        int n, double *partials) {
  Comp a{0.0, 0.0}, b{0.0, 0.0};
  const int base = blockIdx.x * kPerBlock;
  for (int i = threadIdx.x; i < kPerBlock; i += kThreads) {
    const int e = base + i;
    if (e >= n) break;
    comp_add(a, area[e] * z[e]);
    comp_add(b, area[e] * (z[e] + hb[e]));
  }
  comp_block_reduce<kThreads>(a, b);
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x + 0] = a.s;
    partials[4 * blockIdx.x + 1] = a.c;
    partials[4 * blockIdx.x + 2] = b.s;
    partials[4 * blockIdx.x + 3] = b.c;
  }
}

__global__ void __launch_bounds__(kThreads) k_total(int nb, const double *partials, double *out) {
  Comp a{0.0, 0.0}, b{0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += kThreads) {
    a = comp_merge(a, Comp{partials[4 * i], partials[4 * i + 1]});
    b = comp_merge(b, Comp{partials[4 * i + 2], partials[4 * i + 3]});
  }
  comp_block_reduce<kThreads>(a, b);
  if (threadIdx.x == 0) {
    out[0] = a.s + a.c;
    out[1] = b.s + b.c;
  }
}

// Device address of the static buffer on the current device, looked up once per device and kept
// for the life of the process: this assumes the device's primary context is not reset
// (cudaDeviceReset) or destroyed while the library is loaded.
int scratch_address(double **ptr) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DGSWEM_ECUDA;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return DGSWEM_ECUDA;
    g_addr[dev] = static_cast<double *>(p);
  }
  *ptr = g_addr[dev];
  return 0;
}

}  // namespace

extern "C" int dgswem_mass_noalloc(const double *d_zeta00, const double *d_area, const double *d_hb_mean,
                                   int32_t n_elems, double *d_out, void *stream) {
  if (!d_zeta00 || !d_area || !d_hb_mean || !d_out || n_elems < 1) return DGSWEM_EINVAL;
  if (n_elems > DGSWEM_NOALLOC_MAX_ELEMS) return DGSWEM_ETOOBIG;
  double *partials = nullptr;
  if (int r = scratch_address(&partials)) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (n_elems + kPerBlock - 1) / kPerBlock;
  k_partials<<<nb, kThreads, 0, s>>>(d_zeta00, d_area, d_hb_mean, n_elems, partials);
  k_total<<<1, kThreads, 0, s>>>(nb, partials, d_out);
  return cudaGetLastError() == cudaSuccess ? 0 : DGSWEM_ECUDA;
}
