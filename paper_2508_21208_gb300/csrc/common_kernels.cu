// common_kernels.cu -- precision-independent kernels: initial state from nodal values, element
// means, the CFL time step, the compensated mass sum, element reordering and the step counter.
#include <cstdint>

#include "compsum.cuh"
#include "internal.h"

namespace dg {

static __constant__ Tab<double> c_tdc[2];

void upload_common_tables(const Tab<double> td[2]) {
  cudaMemcpyToSymbol(c_tdc, td, sizeof(Tab<double>) * 2);
}

static inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

// Linear interpolant of nodal values (a0, a1, a2) at the element's vertices, expressed in the
// Dubiner modes: mean, (a1 - a0)/2, (2 a2 - a0 - a1)/6; higher modes zero.
__global__ void k_init_nodal(int nd, int ne, int nn, const int *vnode, const double *nodal, double *u) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int n0 = vnode[e], n1 = vnode[ne + e], n2 = vnode[2 * (size_t)ne + e];
  for (int v = 0; v < 3; ++v) {
    const double a0 = nodal[(size_t)v * nn + n0], a1 = nodal[(size_t)v * nn + n1], a2 = nodal[(size_t)v * nn + n2];
    double *uv = u + (size_t)v * nd * ne;
    uv[e] = (a0 + a1 + a2) / 3.0;
    uv[(size_t)ne + e] = 0.5 * (a1 - a0);
    uv[2 * (size_t)ne + e] = (2.0 * a2 - a0 - a1) / 6.0;
    for (int k = 3; k < nd; ++k) uv[(size_t)k * ne + e] = 0.0;
  }
}

void launch_init_nodal(int p, const DevMesh &m, const double *nodal, double *u, cudaStream_t s) {
  k_init_nodal<<<nblk(m.ne, 256), 256, 0, s>>>(nd_of(p), m.ne, m.nn, m.vnode, nodal, u);
}

// dt = cfl * 3/(2p+1) * min_e r_e / lambda_e with lambda_e = max over vertices of
// |u| + sqrt(g max(H, h0)).  Positive doubles order like their bit patterns, so the minimum is
// an exact, order-independent atomicMin on the 64-bit pattern.
template <int P>
__global__ void k_dt(const DevMesh m, const double *u, double g, double h0, unsigned long long *best) {
  constexpr int ND = nd_of(P);
  const int ne = m.ne;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double cand = INFINITY;
  if (e < ne) {
    const Tab<double> &t = c_tdc[P - 1];
    double lam = 0.0;
    for (int i = 0; i < 3; ++i) {
      double w[3];
      for (int v = 0; v < 3; ++v) {
        double s = 0.0;
        for (int k = 0; k < ND; ++k) s += u[(size_t)(v * ND + k) * ne + e] * t.phv[i][k];
        w[v] = s;
      }
      const double H = w[0] + m.hbv[(size_t)i * ne + e];
      const double Hc = H > h0 ? H : h0;
      const double um = Hc > 0.0 ? sqrt(w[1] * w[1] + w[2] * w[2]) / Hc : 0.0;
      const double sp = um + sqrt(g * Hc);
      lam = sp > lam ? sp : lam;
    }
    if (lam > 0.0) cand = m.inradius[e] / lam;
  }
  for (int o = 16; o > 0; o >>= 1) cand = fmin(cand, __shfl_xor_sync(0xffffffffu, cand, o));
  if ((threadIdx.x & 31) == 0 && cand < INFINITY)
    atomicMin(best, (unsigned long long)__double_as_longlong(cand));
}

void launch_dt(int p, const DevMesh &m, const double *u, const Phys &ph, unsigned long long *best,
               cudaStream_t s) {
  cudaMemsetAsync(best, 0xff, sizeof(unsigned long long), s);
  if (p == 1)
    k_dt<1><<<nblk(m.ne, 256), 256, 0, s>>>(m, u, ph.g, ph.h0, best);
  else
    k_dt<2><<<nblk(m.ne, 256), 256, 0, s>>>(m, u, ph.g, ph.h0, best);
}

// ---- compensated sums (compsum.cuh), fixed order.
constexpr int MASS_THREADS = 256;
constexpr int MASS_PER_BLOCK = MASS_THREADS * 8;

int mass_partial_count(int ne) { return nblk(ne, MASS_PER_BLOCK); }

// Block b sums elements [b*MASS_PER_BLOCK, (b+1)*MASS_PER_BLOCK); partial[4*b..] = (s, c) of the
// anomaly volume |Omega| zeta_00 and of the water volume |Omega| (zeta_00 + mean h_b).
__global__ void __launch_bounds__(MASS_THREADS) k_mass_partial(const DevMesh m, const double *u, double *partial) {
  const int ne = m.ne;
  Comp a{0.0, 0.0}, b{0.0, 0.0};
  const int base = blockIdx.x * MASS_PER_BLOCK;
  for (int i = threadIdx.x; i < MASS_PER_BLOCK; i += MASS_THREADS) {
    const int e = base + i;
    if (e >= m.nown) break;
    const double z = u[e], ar = m.area[e];
    const double hm = (m.hbv[e] + m.hbv[ne + e] + m.hbv[2 * (size_t)ne + e]) / 3.0;
    comp_add(a, ar * z);
    comp_add(b, ar * (z + hm));
  }
  comp_block_reduce<MASS_THREADS>(a, b);
  if (threadIdx.x == 0) {
    partial[4 * blockIdx.x + 0] = a.s;
    partial[4 * blockIdx.x + 1] = a.c;
    partial[4 * blockIdx.x + 2] = b.s;
    partial[4 * blockIdx.x + 3] = b.c;
  }
}

__global__ void __launch_bounds__(MASS_THREADS) k_mass_final(int nb, const double *partial, double *result) {
  Comp a{0.0, 0.0}, b{0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += MASS_THREADS) {
    a = comp_merge(a, Comp{partial[4 * i], partial[4 * i + 1]});
    b = comp_merge(b, Comp{partial[4 * i + 2], partial[4 * i + 3]});
  }
  comp_block_reduce<MASS_THREADS>(a, b);
  if (threadIdx.x == 0) {
    result[0] = a.s + a.c;
    result[1] = b.s + b.c;
  }
}

void launch_mass(int p, const DevMesh &m, const double *u, double *partial, double *result, cudaStream_t s) {
  (void)p;
  const int nb = mass_partial_count(m.nown);  // a part sums its own elements
  k_mass_partial<<<nb, MASS_THREADS, 0, s>>>(m, u, partial);
  k_mass_final<<<1, MASS_THREADS, 0, s>>>(nb, partial, result);
}

// dst[row][i] = src[row][map[i]]
__global__ void k_permute(const double *src, double *dst, const int *map, int rows, int ne) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)rows * ne) return;
  const long row = i / ne, c = i - row * ne;
  dst[i] = src[row * ne + map[c]];
}

void launch_permute(const double *src, double *dst, const int *map, int rows, int ne, cudaStream_t s) {
  k_permute<<<nblk((long)rows * ne, 256), 256, 0, s>>>(src, dst, map, rows, ne);
}

__global__ void k_permute_u8(const uint8_t *src, uint8_t *dst, const int *map, int ne) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) dst[i] = src[map[i]];
}

void launch_permute_u8(const uint8_t *src, uint8_t *dst, const int *map, int ne, cudaStream_t s) {
  k_permute_u8<<<nblk(ne, 256), 256, 0, s>>>(src, dst, map, ne);
}

// Ghost exchange of a part (Sec. 5.3, the packElems / unpackElems of Listing code:pack): record k of
// the contiguous buffer holds element idx[k]'s modal state, row by row ([3 nd] doubles), then its
// wet/dry flag as a double.
__global__ void k_halo_pack(int rows, int ne, const double *u, const uint8_t *wd, const int *idx, int n,
                            double *buf) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int rec = rows + 1;
  if (i >= (long)n * rec) return;
  const int k = (int)(i / rec), r = (int)(i - (long)k * rec), e = idx[k];
  buf[i] = r < rows ? u[(size_t)r * ne + e] : (double)wd[e];
}

__global__ void k_halo_unpack(int rows, int ne, double *u, uint8_t *wd, const int *idx, int n, const double *buf) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int rec = rows + 1;
  if (i >= (long)n * rec) return;
  const int k = (int)(i / rec), r = (int)(i - (long)k * rec), e = idx[k];
  if (r < rows)
    u[(size_t)r * ne + e] = buf[i];
  else
    wd[e] = (uint8_t)buf[i];
}

void launch_halo_pack(int nd, int ne, const double *u, const uint8_t *wd, const int *idx, int n, double *buf,
                      cudaStream_t s) {
  if (n > 0) k_halo_pack<<<nblk((long)n * (3 * nd + 1), 256), 256, 0, s>>>(3 * nd, ne, u, wd, idx, n, buf);
}
void launch_halo_unpack(int nd, int ne, double *u, uint8_t *wd, const int *idx, int n, const double *buf,
                        cudaStream_t s) {
  if (n > 0) k_halo_unpack<<<nblk((long)n * (3 * nd + 1), 256), 256, 0, s>>>(3 * nd, ne, u, wd, idx, n, buf);
}

__global__ void k_advance(long long *step) { *step += 1; }

void launch_advance(long long *step, cudaStream_t s) { k_advance<<<1, 1, 0, s>>>(step); }

}  // namespace dg
