// kernels.cuh -- device code of one RK stage: forcing (WIND), edge flux (EDGE), element update
// (AREA + GATHER + inverse mass + SSP-RK stage), slope limiter + wetting/drying (SLOPELIM, WETDRY).
// Included by kernels_f64.cu (T = double: the FP64 form) and kernels_f32.cu (T = float: the
// mixed form, where the RK state, the RK update and all wet/dry depth tests stay in double).
#pragma once
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace dg {

// Reference tables; each translation unit holds its own constant-memory copy.
static __constant__ Tab<double> c_td[2];
static __constant__ Tab<float> c_tf[2];

template <typename T>
__device__ __forceinline__ const Tab<T> &ctab(int p);
template <>
__device__ __forceinline__ const Tab<double> &ctab<double>(int p) { return c_td[p - 1]; }
template <>
__device__ __forceinline__ const Tab<float> &ctab<float>(int p) { return c_tf[p - 1]; }

// A physical constant in the arithmetic type: the double itself, or its host-rounded float copy.
template <typename T>
__device__ __forceinline__ T pc(double d, float f);
template <>
__device__ __forceinline__ double pc<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pc<float>(double, float f) { return f; }

__device__ __forceinline__ double stage_time(const Clock &c, double tau, double fixed) {
  return c.step ? c.t0 + ((double)*c.step + tau) * c.dt : fixed;
}

// ------------------------------------------------------------------------ conversions
// double <-> float conversions with integer operations.  double -> float (d2f) serves the FP64
// form's float filters (its kernels are bound by the FP64 pipe, so they keep conversion
// instructions off it); the mixed form converts double -> float with the hardware instruction
// (from_d<float>), which in its latency-bound kernels measured 19% faster per storm step than
// the integer sequence.  float -> double (f2d) serves the mixed form's RK update (to_d<float>),
// where the hardware widening measured slower.
// Round-to-nearest-even double -> float for results in float's normal range (same value as the
// hardware conversion there); smaller magnitudes give a signed zero, larger ones infinity.
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // float-biased exponent
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  unsigned r = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rb = (lo >> 28) & 1u, sticky = (lo & 0x0fffffffu) != 0u;
  r += rb & (sticky | (r & 1u));
  return __uint_as_float(r);
}
// Exact float -> double (zero and subnormals give a signed zero; infinity/NaN stay non-finite).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, sign = u & 0x80000000u;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const unsigned hi = sign | ((e == 255u ? 2047u : e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 0x7u) << 29));
}
template <typename T>
__device__ __forceinline__ T from_d(double x) { return (T)x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return __double2float_rn(x); }
// float copy of a double for a filter: the hardware conversion in the mixed form (T = float),
// the integer one in the FP64 form (T = double)
template <typename T>
__device__ __forceinline__ float filter_f(double x) { return d2f(x); }
template <>
__device__ __forceinline__ float filter_f<float>(double x) { return __double2float_rn(x); }
template <typename T>
__device__ __forceinline__ double to_d(T x) { return (double)x; }
template <>
__device__ __forceinline__ double to_d<float>(float x) { return f2d(x); }
// x / 2 with IEEE round-to-nearest-even, on the integer pipe: lower the exponent field of a
// normal result; below 2^-1021 (|x| = m 2^-1074 with an integer m) halve m and round half to even;
// infinity and NaN pass through.
__device__ __forceinline__ double half_exact(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex > 1 && ex < 0x7ff) return __longlong_as_double(b - (1LL << 52));
  if (ex == 0x7ff) return x;
  const long long m = b & 0x7fffffffffffffffLL;
  const long long h = (m >> 1) + ((m & 1) & ((m >> 1) & 1));
  return __longlong_as_double((b & (long long)0x8000000000000000ULL) | h);
}
__device__ __forceinline__ double halve(double x) { return half_exact(x); }
// finiteness from the exponent bits (no floating-point compare)
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}

// ------------------------------------------------------------------------ FP64 reciprocal and roots
// The FP64 form is bound by GB300's FP64 pipe, where an IEEE divide or square root costs about ten
// instructions.  These take a float seed from the special-function unit (a separate pipe) and
// finish with one third-order correction in double (Newton-Raphson carried to the second-order
// term of the binomial series, i.e. Householder's method of order 3):
//   1/x:        y0 ~ 1/x,        e = 1 - x y0,    1/x       = y0 (1 + e + e^2)          + O(e^3)
//   1/sqrt(x):  y0 ~ 1/sqrt(x),  e = 1 - x y0^2,  1/sqrt(x) = y0 (1 + e/2 + 3e^2/8)    + O(e^3)
//   sqrt(x)   = (x y0) (1 + e/2 + 3e^2/8)                                              + O(e^3)
// The seed reads x's sign, exponent and top 20 mantissa bits (relative error < 2^-20) and the
// approximate MUFU result adds < 2^-22, so |e| < 2^-18 and the truncation error is below 2^-54:
// three (reciprocal) or five (roots) FP64 instructions, results within about an ulp of the
// correctly rounded value.  |x| outside [2^-100, 2^101) (zero, subnormals, infinity, NaN), or a
// negative operand of a root, takes the IEEE operation.
__device__ __forceinline__ bool seed_range(int hi) {
  return (unsigned)(((hi >> 20) & 0x7ff) - 923) <= 200u;
}
__device__ __forceinline__ float seed_float(int hi) {
  return __int_as_float((hi & (int)0x80000000) | ((((hi >> 20) & 0x7ff) - 896) << 23) | ((hi & 0xfffff) << 3));
}
// exact widening of a normal float (the seeds are normal by construction)
__device__ __forceinline__ double widen_normal(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned hi = (u & 0x80000000u) | ((((u >> 23) & 0xffu) + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 0x7u) << 29));
}
__device__ __forceinline__ double rcp_d(double x) {
  const int hi = __double2hiint(x);
  if (!seed_range(hi)) return 1.0 / x;
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(seed_float(hi)));
  const double y0 = widen_normal(yf);
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}
__device__ __forceinline__ double rsqrt_d(double x) {
  const int hi = __double2hiint(x);
  if (hi < 0 || !seed_range(hi)) return rsqrt(x);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(seed_float(hi)));
  const double y0 = widen_normal(yf);
  const double e = fma(-(x * y0), y0, 1.0);
  return fma(y0 * e, fma(0.375, e, 0.5), y0);
}
__device__ __forceinline__ double sqrt_d(double x) {
  const int hi = __double2hiint(x);
  if (hi < 0 || !seed_range(hi)) return sqrt(x);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(seed_float(hi)));
  const double y0 = widen_normal(yf);
  const double a = x * y0;
  const double e = fma(-a, y0, 1.0);
  return fma(a * e, fma(0.375, e, 0.5), a);
}
// the float form keeps the plain operations (its pipe is not the bound)
template <typename T>
__device__ __forceinline__ T rcp_t(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ double rcp_t<double>(double x) { return rcp_d(x); }
template <typename T>
__device__ __forceinline__ T sqrt_t(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt_d(x); }
template <typename T>
__device__ __forceinline__ T rsqrt_t(T x) { return rsqrt(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt_d(x); }
// a / b: through the seeded reciprocal only where b lies in its range; elsewhere the IEEE divide
// (1/b overflows for subnormal b where a/b with |a| <= |b| stays finite)
template <typename T>
__device__ __forceinline__ T ratio_t(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ double ratio_t<double>(double a, double b) {
  return seed_range(__double2hiint(b)) ? a * rcp_d(b) : a / b;
}
// x > 0 from the bits (an integer compare; positive NaN counts as positive and stays non-finite)
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return __float_as_int(x) > 0; }

// Value of a modal expansion at a point: the Dubiner mode psi_00 is identically 1 (Eq. dubiner),
// so its coefficient enters without a multiply.
template <int ND, typename T>
__device__ __forceinline__ T modal_value(const T (&w)[ND], const T *ph) {
  T x = w[0];
#pragma unroll
  for (int k = 1; k < ND; ++k) x += w[k] * ph[k];
  return x;
}

// ------------------------------------------------------------------------ point physics
// Normal flux F(w).n of Eq. SWE with the pressure term (g/2)(H^2 - h_b^2) = (g/2) zeta (zeta + 2 h_b).
// One side of an edge point: q.n, u.n = q.n / H, the wave speed |u.n| + sqrt(g H) and the pressure
// term P = (g/2) zeta (zeta + 2 h_b), so that F(w).n = (q.n, q_x u.n + P n_x, q_y u.n + P n_y).
// 1/H and sqrt(g H) come from one reciprocal square root; where H <= 0 (no water) the velocity
// and the wave speed are zero, in both fluxes, the area integrals and the friction.
template <typename T>
struct Side {
  T qn, un, s, P;
};
template <typename T>
__device__ __forceinline__ Side<T> side_flux(T g, T sqrt_g, const T w[3], T hb, T nx, T ny) {
  Side<T> r;
  const T H = w[0] + hb;
  r.qn = w[1] * nx + w[2] * ny;
  T c;
  if (positive(H)) {
    const T rs = rsqrt_t(H);
    r.un = r.qn * rs * rs;
    c = sqrt_g * H * rs;
  } else {  // no water: zero velocity and wave speed
    r.un = T(0);
    c = T(0);
  }
  r.P = T(0.5) * g * w[0] * (w[0] + T(2) * hb);
  r.s = fabs(r.un) + c;
  return r;
}

// max of two non-negative numbers (ordered like their bit patterns: an integer compare)
__device__ __forceinline__ float max_nonneg(float a, float b) { return __float_as_int(a) > __float_as_int(b) ? a : b; }
__device__ __forceinline__ double max_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}
// x / 2: exact, on the integer pipe for double
__device__ __forceinline__ float halve(float x) { return 0.5f * x; }

// Local Lax-Friedrichs flux (the numerical flux of Eq. elem_weak_form), n from wi to wo:
// (F(wi).n + F(wo).n)/2 - lam (wo - wi)/2 with lam the larger wave speed; the two pressure terms
// are summed before the normal is applied.
template <typename T>
__device__ __forceinline__ void llf(T g, T sqrt_g, const T wi[3], const T wo[3], T hb, T nx, T ny, T out[3]) {
  const Side<T> a = side_flux(g, sqrt_g, wi, hb, nx, ny);
  const Side<T> b = side_flux(g, sqrt_g, wo, hb, nx, ny);
  const T lam = max_nonneg(a.s, b.s);
  const T Ps = a.P + b.P;
  out[0] = halve(a.qn + b.qn - lam * (wo[0] - wi[0]));
  out[1] = halve(fma(wi[1], a.un, wo[1] * b.un) + Ps * nx - lam * (wo[1] - wi[1]));
  out[2] = halve(fma(wi[2], a.un, wo[2] * b.un) + Ps * ny - lam * (wo[2] - wi[2]));
}

// Roe (1981) flux, n from wi to wo.  Edge frame (n, t = (-ny, nx)), state (H, q_n, q_t); Roe
// averages H~ = (Hi + Ho)/2, u~ = sqrt(H)-weighted mean velocity, c~ = sqrt(g H~); eigenvalues
// u~_n -+ c~ (acoustic, Harten entropy fix with delta = c~/10) and u~_n (shear); wave strengths
// a1 = ((u~_n + c~) dH - dq_n)/(2c~), a2 = dq_t - u~_t dH, a3 = (dq_n - (u~_n - c~) dH)/(2c~);
// Fhat = (F(wi) + F(wo)).n / 2 - |A~| dw / 2.  dH = d zeta because h_b is continuous.
template <typename T>
__device__ __forceinline__ T harten(T lam, T d) {
  const T a = fabs(lam);
  return a < d ? T(0.5) * (lam * lam + d * d) / d : a;
}

template <typename T>
__device__ __forceinline__ void roe(T g, const T wi[3], const T wo[3], T hb, T nx, T ny, T out[3]) {
  const T Hi = wi[0] + hb, Ho = wo[0] + hb;
  const T qni = wi[1] * nx + wi[2] * ny, qti = -wi[1] * ny + wi[2] * nx;
  const T qno = wo[1] * nx + wo[2] * ny, qto = -wo[1] * ny + wo[2] * nx;
  const T Pi = T(0.5) * g * wi[0] * (wi[0] + T(2) * hb), Po = T(0.5) * g * wo[0] * (wo[0] + T(2) * hb);
  const T iHi = positive(Hi) ? rcp_t(Hi) : T(0), iHo = positive(Ho) ? rcp_t(Ho) : T(0);
  const T uni = qni * iHi, uno = qno * iHo;
  // F(w).n in the x/y frame: (q_n, q_x u_n + P n_x, q_y u_n + P n_y)
  const T Fi[3] = {qni, wi[1] * uni + Pi * nx, wi[2] * uni + Pi * ny};
  const T Fo[3] = {qno, wo[1] * uno + Po * nx, wo[2] * uno + Po * ny};
  const T si = positive(Hi) ? sqrt_t(Hi) : T(0), so = positive(Ho) ? sqrt_t(Ho) : T(0);
  T un = T(0), ut = T(0);
  if (positive(si + so)) {
    const T inv = rcp_t(si + so);
    un = (si * uni + so * uno) * inv;
    ut = (si * (qti * iHi) + so * (qto * iHo)) * inv;
  }
  const T Hm = T(0.5) * (Hi + Ho);
  const T c = positive(Hm) ? sqrt_t(g * Hm) : T(0);
  const T dH = wo[0] - wi[0], dqn = qno - qni, dqt = qto - qti;
  T dh = T(0), dn = T(0), dt = T(0);
  if (positive(c)) {
    const T i2c = T(0.5) * rcp_t(c);
    const T a1 = ((un + c) * dH - dqn) * i2c;
    const T a3 = (dqn - (un - c) * dH) * i2c;
    const T a2 = dqt - ut * dH;
    const T l1 = harten(un - c, T(0.1) * c), l2 = fabs(un), l3 = harten(un + c, T(0.1) * c);
    dh = l1 * a1 + l3 * a3;
    dn = l1 * a1 * (un - c) + l3 * a3 * (un + c);
    dt = l1 * a1 * ut + l2 * a2 + l3 * a3 * ut;
  }
  out[0] = T(0.5) * (Fi[0] + Fo[0]) - T(0.5) * dh;
  out[1] = T(0.5) * (Fi[1] + Fo[1]) - T(0.5) * (dn * nx - dt * ny);
  out[2] = T(0.5) * (Fi[2] + Fo[2]) - T(0.5) * (dn * ny + dt * nx);
}

// River inflow: the land mirror shifted so that (q+ + q-).n / 2 = -q_in, then the numerical flux.
template <typename T>
__device__ __forceinline__ void river(const Phys &ph, T g, T sqrt_g, const T wi[3], T hb, T nx, T ny, T out[3]);

// The numerical flux selected by the parameters (uniform branch).
template <typename T>
__device__ __forceinline__ void numflux(const Phys &ph, T g, T sqrt_g, const T wi[3], const T wo[3], T hb, T nx,
                                        T ny, T out[3]) {
  if (ph.flux == DGSWEM_FLUX_ROE)
    roe(g, wi, wo, hb, nx, ny, out);
  else
    llf(g, sqrt_g, wi, wo, hb, nx, ny, out);
}

template <typename T>
__device__ __forceinline__ void river(const Phys &ph, T g, T sqrt_g, const T wi[3], T hb, T nx, T ny, T out[3]) {
  const T d = T(2) * (wi[1] * nx + wi[2] * ny + pc<T>(ph.river_q, ph.f.river_q));
  const T wo[3] = {wi[0], wi[1] - d * nx, wi[2] - d * ny};
  numflux(ph, g, sqrt_g, wi, wo, hb, nx, ny, out);
}

// Land (no normal flow): mirror ghost zeta- = zeta+, q- = q+ - 2 (q+.n) n, then the numerical flux.
template <typename T>
__device__ __forceinline__ void wall(const Phys &ph, T g, T sqrt_g, const T wi[3], T hb, T nx, T ny, T out[3]) {
  const T qn = wi[1] * nx + wi[2] * ny;
  const T wo[3] = {wi[0], wi[1] - T(2) * qn * nx, wi[2] - T(2) * qn * ny};
  numflux(ph, g, sqrt_g, wi, wo, hb, nx, ny, out);
}

// Wetting/drying edge rule: an edge touching a dry element carries no flow (each side sees a
// wall) unless the wet side's surface trace rises above the highest bed (-h_b) on the edge.
// The depth test runs in double in both forms.
template <int P>
__device__ __forceinline__ bool edge_flows(const Phys &ph, uint8_t f_self, uint8_t f_nbr,
                                           const double *u, int ne, int e_self, int l_self, int e_nbr,
                                           int l_nbr, double hbA, double hbB) {
  if (!ph.wetdry) return true;
  const bool ds = f_self == 2, dn = f_nbr == 2;
  if (!ds && !dn) return true;
  if (ds && dn) return false;
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const int ew = ds ? e_nbr : e_self, lw = ds ? l_nbr : l_self;
  const Tab<double> &td = c_td[P - 1];
  double zmax = -INFINITY;
#pragma unroll
  for (int g = 0; g < NQE; ++g) {
    double z = u[ew];  // psi_00 = 1
#pragma unroll
    for (int k = 1; k < ND; ++k) z += u[(size_t)k * ne + ew] * td.phe[lw][g][k];
    zmax = z > zmax ? z : zmax;
  }
  const double bed = (-hbA > -hbB) ? -hbA : -hbB;
  return zmax > bed;
}

template <int P, typename T>
__device__ __forceinline__ void load_modes(const double *u, int ne, int e, T w[3][nd_of(P)]) {
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int k = 0; k < nd_of(P); ++k) w[v][k] = from_d<T>(__ldg(&u[(size_t)(v * nd_of(P) + k) * ne + e]));
}

// ------------------------------------------------------------------------ WIND
// Holland (1980) vortex: p = pc + (pn - pc) exp(-(Rmax/r)^B); gradient wind
// V = sqrt(B/rho_a (pn - pc) (Rmax/r)^B exp(-(Rmax/r)^B) + (r f/2)^2) - r f/2; surface wind 0.9 V
// counter-clockwise plus half the translation velocity; Garratt (1977) drag
// C_d = min(0.75 + 0.067 |U|, 3.5) 1e-3.  Output per node: tau/rho_w (x, y) and the pressure
// anomaly (p - pn)/rho_w (only its gradient enters the momentum source).
// Storm centre at time t (double: coordinates are O(1e5) m).
__device__ __forceinline__ void storm_center(const Phys &ph, double t, double &cx, double &cy) {
  cx = ph.x0 + ph.vt * ph.cos_h * t;
  cy = ph.y0 + ph.vt * ph.sin_h * t;
}

// Forcing at a point (dx, dy) from the storm centre: tau/rho_w and (p - pn)/rho_w.
template <typename T>
__device__ __forceinline__ void vortex_at(const Phys &ph, T dx, T dy, T &tx_out, T &ty_out, T &pa_out) {
  const T r = sqrt_t(dx * dx + dy * dy);
  const T dp = (T)(ph.pn - ph.pc);
  const T tx = T(0.5) * (T)(ph.vt * ph.cos_h), ty = T(0.5) * (T)(ph.vt * ph.sin_h);
  T pa, ux, uy;
  if (r < T(1)) {
    pa = -dp;
    ux = tx;
    uy = ty;
  } else {
    // anomaly (pn - pc) (exp(-A) - 1) from expm1: no cancellation where A is small (far field);
    // the usual Holland B = 1.5 takes (Rmax/r)^B = s sqrt(s) instead of a general power
    const T ir = rcp_t(r), sr = (T)ph.rmax * ir;
    const T A = ph.holland15 ? sr * sqrt_t(sr) : pow(sr, (T)ph.hB), em1 = expm1(-A), E = T(1) + em1;
    pa = dp * em1;
    const T hf = T(0.5) * r * (T)ph.flat;
    const T V = sqrt_t((T)ph.hB_rho_air * dp * A * E + hf * hf) - hf;
    ux = T(0.9) * V * (-dy * ir) + tx;
    uy = T(0.9) * V * (dx * ir) + ty;
  }
  const T U = sqrt_t(ux * ux + uy * uy);
  T cd = T(0.75) + T(0.067) * U;
  cd = (cd > T(3.5) ? T(3.5) : cd) * T(1e-3);
  const T k = (T)ph.rho_ratio * cd * U;
  tx_out = k * ux;
  ty_out = k * uy;
  pa_out = pa * (T)ph.inv_rho_w;
}

// The mixed form's vortex: one reciprocal square root for 1/r, the hardware log2/exp2
// approximations for (Rmax/r)^B (a few float ulp), expm1f for the pressure anomaly and
// multiplications by host-computed constants.  Out of line, so that every kernel that evaluates it rounds identically.
static __device__ __noinline__ void vortex_at_f(const Phys &ph, float dx, float dy, float *out) {
  const float r2 = dx * dx + dy * dy;
  const float dp = ph.f.dp;
  const float tx = ph.f.tx, ty = ph.f.ty;
  float pa, ux, uy;
  if (r2 < 1.f) {
    pa = -dp;
    ux = tx;
    uy = ty;
  } else {
    const float ir = rsqrtf(r2), r = r2 * ir;
    const float A = exp2f(ph.f.hB * __log2f(ph.f.rmax * ir)), em1 = expm1f(-A), E = 1.f + em1;
    pa = dp * em1;
    const float hf = 0.5f * r * ph.f.flat;
    const float V = sqrtf(ph.f.hB_rho_air * dp * A * E + hf * hf) - hf;
    ux = 0.9f * V * (-dy * ir) + tx;
    uy = 0.9f * V * (dx * ir) + ty;
  }
  const float U = sqrtf(ux * ux + uy * uy);
  float cd = 0.75f + 0.067f * U;
  cd = (cd > 3.5f ? 3.5f : cd) * 1e-3f;
  const float k = ph.f.rho_ratio * cd * U;
  out[0] = k * ux;
  out[1] = k * uy;
  out[2] = pa * ph.f.inv_rho_w;
}
template <>
__device__ __forceinline__ void vortex_at<float>(const Phys &ph, float dx, float dy, float &tx_out, float &ty_out,
                                                 float &pa_out) {
  float o[3];
  vortex_at_f(ph, dx, dy, o);
  tx_out = o[0];
  ty_out = o[1];
  pa_out = o[2];
}

template <typename T>
__device__ __forceinline__ void forcing_body(const double *nodexy, int nn, const Phys &ph, double t, T *frc,
                                             int n) {
  T a, b, c;
  double cx, cy;
  storm_center(ph, t, cx, cy);
  vortex_at<T>(ph, from_d<T>(nodexy[n] - cx), from_d<T>(nodexy[nn + n] - cy), a, b, c);
  frc[n] = a;
  frc[nn + n] = b;
  frc[2 * nn + n] = c;
}

template <typename T>
__global__ void k_forcing(const double *nodexy, int nn, Phys ph, Clock clk, double tau, double t_fixed,
                          T *frc) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  forcing_body<T>(nodexy, nn, ph, stage_time(clk, tau, t_fixed), frc, n);
}

// Copy the edge basis table of degree P into shared memory (indexed by thread-varying local edges).
template <int P, typename T>
__device__ __forceinline__ void load_phe(T (*s_phe)[nqe_of(P)][nd_of(P)]) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const Tab<T> &tb = ctab<T>(P);
  for (int i = threadIdx.x; i < 3 * NQE * ND; i += blockDim.x)
    s_phe[i / (NQE * ND)][(i / ND) % NQE][i % ND] = tb.phe[i / (NQE * ND)][(i / ND) % NQE][i % ND];
}

// ------------------------------------------------------------------------ EDGE (split variant)
// One thread per interior edge: both traces at the edge Gauss points, the wet/dry flow decision,
// the LLF flux, stored once per edge already multiplied by the quadrature weight and half length
// (the minus side reads it with the opposite sign and reversed point order).
template <int P, typename T>
__global__ void __launch_bounds__(256) k_edge(const DevMesh m, const StageArgs s, const Phys ph) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  __shared__ T s_phe[3][NQE][ND];
  const Tab<T> &tb = ctab<T>(P);
  for (int i = threadIdx.x; i < 3 * NQE * ND; i += blockDim.x)
    s_phe[i / (NQE * ND)][(i / ND) % NQE][i % ND] = tb.phe[i / (NQE * ND)][(i / ND) % NQE][i % ND];
  __syncthreads();
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int nint = m.nint, ne = m.ne;
  if (d >= nint) return;
  const int ep = m.edel[d], em = m.edel[nint + d];
  const int code = m.edle[d], lp = code & 3, lm = code >> 2;
  const T *eg = (const T *)m.edgeo;
  const T nx = eg[d], ny = eg[nint + d], hl = eg[2 * nint + d];
  const uint8_t fp = s.wd ? s.wd[ep] : 0, fm = s.wd ? s.wd[em] : 0;
  // the edge's vertex depths decide only an edge with exactly one dry side
  const bool one_dry = (fp == 2) != (fm == 2);
  const double hbA = one_dry ? m.edhb[d] : 0.0, hbB = one_dry ? m.edhb[nint + d] : 0.0;
  const bool flows = edge_flows<P>(ph, fp, fm, s.uin, ne, ep, lp, em, lm, hbA, hbB);
  s.emode[d] = flows ? 1 : 0;
  if (!flows) return;
  T wp[3][ND], wm[3][ND];
  load_modes<P, T>(s.uin, ne, ep, wp);
  load_modes<P, T>(s.uin, ne, em, wm);
  const T g = pc<T>(ph.g, ph.f.g), sqg = pc<T>(ph.sqrt_g, ph.f.sqrt_g);
  T *F = (T *)s.eflux;
#pragma unroll
  for (int q = 0; q < NQE; ++q) {
    T a[3], b[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      a[v] = modal_value<ND, T>(wp[v], s_phe[lp][q]);
      b[v] = modal_value<ND, T>(wm[v], s_phe[lm][NQE - 1 - q]);
    }
    const T hb = ((const T *)m.edhbq)[(size_t)q * nint + d];  // h_b at the point, host-computed
    T f[3];
    numflux(ph, g, sqg, a, b, hb, nx, ny, f);
    const T wgt = hl * tb.we[q];
#pragma unroll
    for (int v = 0; v < 3; ++v) F[(size_t)(v * NQE + q) * nint + d] = wgt * f[v];
  }
}

// ------------------------------------------------------------------------ element update
// One thread per element.  r_k = (grad phi_k, F)_e + (phi_k, s)_e - <phi_k, Fhat.n>_de
// (Eq. elem_weak_form with the volume term's sign fixed by integration by parts, Alg. 1 and the
// gather of Alg. 3), L_k = r_k / (|J| ||phi_k||^2), then the SSP-RK stage in the two-register
// Shu-Osher form u_out = a u^n + b u_in + c dt L(u_in), in double (SSP-RK2: u1 = u + dt L(u),
// then u_new = (u + (u1 + dt L(u1)))/2).
// Source terms linear in the state (bathymetry slope g zeta dh_b/dx, Coriolis, wind stress,
// pressure gradient -H dp_a/dx with linear p_a) are integrated in closed form through the basis
// orthogonality; the area rule is exact for them, so this is the same discrete operator.
// Per-element quantities shared by the element-update variants.
template <int P, typename T>
struct ElemCtx {
  T w[3][nd_of(P)];
  T rx, ry, sx, sy, dJ;
  double hbd[3];
  T hb[3];
};

template <int P, typename T>
__device__ __forceinline__ void elem_load_geom(const DevMesh &m, int e, ElemCtx<P, T> &c) {
  const int ne = m.ne;
  const T *geo = (const T *)m.geo;
  c.rx = geo[GEO_RX * (size_t)ne + e];
  c.ry = geo[GEO_RY * (size_t)ne + e];
  c.sx = geo[GEO_SX * (size_t)ne + e];
  c.sy = geo[GEO_SY * (size_t)ne + e];
  c.dJ = geo[GEO_DETJ * (size_t)ne + e];
  c.hbd[0] = m.hbv[e];
  c.hbd[1] = m.hbv[ne + e];
  c.hbd[2] = m.hbv[2 * (size_t)ne + e];
  for (int a = 0; a < 3; ++a) {  // the float form's copies are rounded on the host like from_d
    if constexpr (sizeof(T) == sizeof(float)) c.hb[a] = m.elf[(size_t)a * ne + e];
    else c.hb[a] = c.hbd[a];
  }
}

template <int P, typename T>
__device__ __forceinline__ void elem_load(const DevMesh &m, const double *u, int e, ElemCtx<P, T> &c) {
  load_modes<P, T>(u, m.ne, e, c.w);
  elem_load_geom<P, T>(m, e, c);
}

// Area integrals (Alg. 1): advective + pressure flux and friction, r_k set (not accumulated).
// The weight w_q is folded into the velocities, U = w_q q_x / H and V = w_q q_y / H, and the
// pressure term (g/2) zeta (zeta + 2 h_b) is summed without its factor g/2.  At P = 1 (grad phi
// constant) the point sums are G = (Gx, Gy, Hy, Ps): sums of q_x U, q_x V, q_y V and
// w_q zeta (zeta + 2 h_b); at P = 2 the points add to r directly.  fr: the friction integrals.
template <int P, typename T>
struct AreaSums {
  T G[4];
  T fr[2][nd_of(P)];
};

// One area quadrature point's contributions (added to r at P = 2, to a otherwise).
template <int P, typename T>
__device__ __forceinline__ void area_point(const ElemCtx<P, T> &c, const Phys &ph, T r[3][nd_of(P)],
                                           AreaSums<P, T> &a, const DevMesh &m, const int e, const int q) {
  constexpr int ND = nd_of(P);
  const Tab<T> &tb = ctab<T>(P);
  const T g = pc<T>(ph.g, ph.f.g);
  const T rx = c.rx, ry = c.ry, sx = c.sx, sy = c.sy;
  const T (&w)[3][ND] = c.w;
  const T (&hb)[3] = c.hb;
  const T hg = T(0.5) * g;
  const T z = modal_value<ND, T>(w[0], tb.phq[q]);
  const T qx = modal_value<ND, T>(w[1], tb.phq[q]);
  const T qy = modal_value<ND, T>(w[2], tb.phq[q]);
  // h_b at the point: read in the FP64 form (host-computed; an FP64 interpolation costs more
  // issue than the load), interpolated in the latency-bound float form
  T hq;
  if constexpr (sizeof(T) == sizeof(double))
    hq = ((const T *)m.hbq)[(size_t)q * m.ne + e];
  else
    hq = hb[0] * tb.nq[q][0] + hb[1] * tb.nq[q][1] + hb[2] * tb.nq[q][2];
  const T H = z + hq;
  const T wq = tb.wq[q];
  const T iHw = positive(H) ? wq * rcp_t(H) : T(0);  // zero velocity where there is no water
  const T U = qx * iHw, V = qy * iHw;
  const T Pw = wq * (z * (z + T(2) * hq));
  if constexpr (P == 1) {
    a.G[0] += qx * U;
    a.G[1] += qx * V;
    a.G[2] += qy * V;
    a.G[3] += Pw;
  } else {
    const T Pg = hg * Pw;
    const T Fxx = qx * U + Pg, Fxy = qx * V, Fyy = qy * V + Pg;  // w_q F
#pragma unroll
    for (int k = 1; k < ND; ++k) {
      const T gx = rx * tb.dxq[q][k] + sx * tb.dyq[q][k];
      const T gy = ry * tb.dxq[q][k] + sy * tb.dyq[q][k];
      r[0][k] += wq * (gx * qx + gy * qy);
      r[1][k] += gx * Fxx + gy * Fxy;
      r[2][k] += gx * Fxy + gy * Fyy;
    }
  }
  if (ph.friction) {
    // w_q tau_b q = c |q| q / H^2 w_q (times H^-1/3 for Manning) = c |U| U / w_q for H > 0, and
    // zero for H <= 0 (U = V = 0 there)
    T cq = pc<T>(ph.cf, ph.f.cf);
    if (ph.friction == DGSWEM_FRICTION_MANNING) cq = positive(H) ? pc<T>(ph.gn2, ph.f.gn2) * rcbrt(H) : T(0);
    else if (ph.friction != DGSWEM_FRICTION_QUADRATIC) cq = T(0);
    const T Um = sqrt_t(U * U + V * V);
    const T kq = cq * Um * tb.iwq[q];
    const T tx = kq * U, ty = kq * V;
    a.fr[0][0] += tx;  // psi_00 = 1
    a.fr[1][0] += ty;
#pragma unroll
    for (int k = 1; k < ND; ++k) {
      a.fr[0][k] += tx * tb.phq[q][k];
      a.fr[1][k] += ty * tb.phq[q][k];
    }
  }
}

// The area integrals from the point sums: the P = 1 flux terms through the constant gradients,
// the friction, and the factor |J|.
template <int P, typename T>
__device__ __forceinline__ void area_close(const ElemCtx<P, T> &c, const Phys &ph, T r[3][nd_of(P)],
                                           AreaSums<P, T> &a) {
  constexpr int ND = nd_of(P);
  const T g = pc<T>(ph.g, ph.f.g);
  const T rx = c.rx, ry = c.ry, sx = c.sx, sy = c.sy, dJ = c.dJ;
  const T (&w)[3][ND] = c.w;
  const T hg = T(0.5) * g;
  if constexpr (P == 1) {
    T &Gx = a.G[0], &Gy = a.G[1], &Hy = a.G[2], &Ps = a.G[3];
    const T Pg = hg * Ps;
    Gx += Pg;
    Hy += Pg;
    // grad psi_10 = J^-T (1, 1/2), grad psi_01 = J^-T (0, 3/2); the mass flux q is linear, so
    // sum_q w_q q(x_q) = 2 q_00 exactly
    const T g1x = rx + T(0.5) * sx, g1y = ry + T(0.5) * sy;
    const T g2x = T(1.5) * sx, g2y = T(1.5) * sy;
    r[0][1] = T(2) * (g1x * w[1][0] + g1y * w[2][0]);
    r[0][2] = T(2) * (g2x * w[1][0] + g2y * w[2][0]);
    r[1][1] = g1x * Gx + g1y * Gy;
    r[1][2] = g2x * Gx + g2y * Gy;
    r[2][1] = g1x * Gy + g1y * Hy;
    r[2][2] = g2x * Gy + g2y * Hy;
  }
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    r[0][k] *= dJ;
    r[1][k] = (r[1][k] - a.fr[0][k]) * dJ;
    r[2][k] = (r[2][k] - a.fr[1][k]) * dJ;
  }
}

template <int P, typename T>
__device__ __forceinline__ void area_zero(T r[3][nd_of(P)], AreaSums<P, T> &a) {
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int k = 0; k < nd_of(P); ++k) r[v][k] = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) a.G[i] = T(0);
#pragma unroll
  for (int k = 0; k < nd_of(P); ++k) a.fr[0][k] = a.fr[1][k] = T(0);
}

template <int P, typename T>
__device__ __forceinline__ void elem_area(const ElemCtx<P, T> &c, const Phys &ph, T r[3][nd_of(P)],
                                          const DevMesh &m, const int e) {
  AreaSums<P, T> a;
  area_zero<P, T>(r, a);
#pragma unroll
  for (int q = 0; q < nqa_of(P); ++q) area_point<P, T>(c, ph, r, a, m, e, q);
  area_close<P, T>(c, ph, r, a);
}

// Inverse mass matrix, closed-form linear sources and the RK stage; writes u^(s+1) and the means
// (the limiter's copy in MT, the form's type; the double path also writes them to s.mean64 when set).
// ctr: the storm centre at the stage time (once per block), or null; vxy: the element's vertex
// coordinates already in T (x0, x1, x2 at vxy[0], vxy[vs], vxy[2 vs], then y), or null to read the
// nodes.
// DSTEP > 1: this thread writes only the degrees of freedom d = v ND + k with d = dsub (mod DSTEP)
// (a lane group sharing one element: each lane holds the same sums and finishes a few of them).
template <int P, typename T, typename MT = T, int DSTEP = 1>
__device__ __forceinline__ void elem_finish(const DevMesh &m, const StageArgs &s, const Phys &ph,
                                            const int write_rhs, const int e, const ElemCtx<P, T> &c,
                                            T r[3][nd_of(P)], const double *ctr = nullptr,
                                            const T *vxy = nullptr, const int vs = 0, const int dsub = 0) {
  constexpr int ND = nd_of(P);
  const Tab<T> &tb = ctab<T>(P);
  const int ne = m.ne;
  const T g = pc<T>(ph.g, ph.f.g);
  const T rx = c.rx, ry = c.ry, sx = c.sx, sy = c.sy, dJ = c.dJ;
  const T (&w)[3][ND] = c.w;
  const T (&hb)[3] = c.hb;
  const T idJ = rcp_t(dJ);
  T src1[3] = {0, 0, 0}, src2[3] = {0, 0, 0};  // per linear mode, for q_x and q_y
  {
    const T hbx = T(0.5) * (rx * (hb[1] - hb[0]) + sx * (hb[2] - hb[0]));
    const T hby = T(0.5) * (ry * (hb[1] - hb[0]) + sy * (hb[2] - hb[0]));
    const T fc = pc<T>(ph.fcor, ph.f.fcor);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      src1[k] = g * hbx * w[0][k] + fc * w[2][k];
      src2[k] = g * hby * w[0][k] - fc * w[1][k];
    }
    if (s.frc || s.frc_inline) {
      const int nn = m.nn;
      T t0, t1, t2, u0, u1, u2, p0, p1, p2;
      if (s.frc_inline) {
        // the centre once per element (or per block: ctr); vertex offsets in T (O(1e5) m
        // coordinates, float ulp ~1 cm)
        double cxd, cyd;
        if (ctr) {
          cxd = ctr[0];
          cyd = ctr[1];
        } else {
          storm_center(ph, stage_time(s.clk, s.tau, s.tide_t), cxd, cyd);
        }
        const T cx = from_d<T>(cxd), cy = from_d<T>(cyd);
        T x[3], y[3];
        if (vxy) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            x[a] = vxy[a * vs];
            y[a] = vxy[(3 + a) * vs];
          }
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int n = m.vnode[(size_t)a * ne + e];
            x[a] = from_d<T>(m.nodexy[n]);
            y[a] = from_d<T>(m.nodexy[nn + n]);
          }
        }
        vortex_at<T>(ph, x[0] - cx, y[0] - cy, t0, u0, p0);
        vortex_at<T>(ph, x[1] - cx, y[1] - cy, t1, u1, p1);
        vortex_at<T>(ph, x[2] - cx, y[2] - cy, t2, u2, p2);
      } else {
        const int n0 = m.vnode[e], n1 = m.vnode[ne + e], n2 = m.vnode[2 * (size_t)ne + e];
        const T *F = (const T *)s.frc;
        t0 = F[n0]; t1 = F[n1]; t2 = F[n2];
        u0 = F[nn + n0]; u1 = F[nn + n1]; u2 = F[nn + n2];
        p0 = F[2 * nn + n0]; p1 = F[2 * nn + n1]; p2 = F[2 * nn + n2];
      }
      const T pax = T(0.5) * (rx * (p1 - p0) + sx * (p2 - p0));
      const T pay = T(0.5) * (ry * (p1 - p0) + sy * (p2 - p0));
      // Dubiner linear modes of the interpolant through vertex values (a0, a1, a2)
      const T third = T(1) / T(3), sixth = T(1) / T(6);  // constants: no divide at run time
      const T hm[3] = {(hb[0] + hb[1] + hb[2]) * third, T(0.5) * (hb[1] - hb[0]),
                       (T(2) * hb[2] - hb[0] - hb[1]) * sixth};
      const T tm[3] = {(t0 + t1 + t2) * third, T(0.5) * (t1 - t0), (T(2) * t2 - t0 - t1) * sixth};
      const T um[3] = {(u0 + u1 + u2) * third, T(0.5) * (u1 - u0), (T(2) * u2 - u0 - u1) * sixth};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        src1[k] += tm[k] - pax * (w[0][k] + hm[k]);
        src2[k] += um[k] - pay * (w[0][k] + hm[k]);
      }
      if constexpr (P == 2) {
        // quadratic modes: only the zeta part of -H grad p_a remains
        for (int k = 3; k < ND; ++k) {
          r[1][k] -= dJ * tb.nrm[k] * pax * w[0][k];
          r[2][k] -= dJ * tb.nrm[k] * pay * w[0][k];
        }
      }
    }
    if constexpr (P == 2) {
      for (int k = 3; k < ND; ++k) {
        r[1][k] += dJ * tb.nrm[k] * (g * hbx * w[0][k] + fc * w[2][k]);
        r[2][k] += dJ * tb.nrm[k] * (g * hby * w[0][k] - fc * w[1][k]);
      }
    }
  }
  const double dt = s.clk.dt;
  const size_t base = (size_t)ne;
  bool bad = false;
  T minv[ND];  // inverse mass matrix diagonal: 1 / (|J| ||phi_k||^2)
#pragma unroll
  for (int k = 0; k < ND; ++k) minv[k] = idJ * tb.inrm[k];
  // the stage update of degree of freedom (v, k) with its right-hand side L
  auto update = [&](const int v, const int k, const T L) {
    const size_t ix = (size_t)(v * ND + k) * base + e;
    const double Ld = to_d<T>(L);
    double out;
    if (write_rhs) {
      out = Ld;
    } else if (s.rk_form == 0) {  // forward-Euler stage
      out = fma(s.rcdt, Ld, s.uin[ix]);
    } else if (s.rk_form == 1) {
      // u/2 + (u1 + dt L)/2 == (u + (u1 + dt L)) / 2 exactly (halving commutes with rounding)
      out = half_exact(s.un[ix] + (s.uin[ix] + dt * Ld));
    } else {
      out = fma(s.rcdt, Ld, s.ra * s.un[ix] + s.rb * s.uin[ix]);
    }
    bad |= !finite_bits(out);
    s.uout[ix] = out;
    if (k == 0) {
      if (s.mean) static_cast<MT *>(s.mean)[(size_t)v * ne + e] = from_d<MT>(out);
      if constexpr (sizeof(T) == sizeof(double))
        if (s.mean64) s.mean64[(size_t)v * ne + e] = out;
    }
  };
  const T rain = pc<T>(ph.rain, ph.f.rain);  // (phi_0, R) / (|J| ||phi_0||^2) = R
  if constexpr (DSTEP == 1) {
#pragma unroll
    for (int v = 0; v < 3; ++v) {
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        T L = r[v][k] * minv[k];
        if (k < 3) L += (v == 1) ? src1[k] : (v == 2 ? src2[k] : T(0));
        if (v == 0 && k == 0) L += rain;
        update(v, k, L);
      }
    }
  } else {
    for (int d = dsub; d < 3 * ND; d += DSTEP) {
      const int v = d / ND, k = d - v * ND;
      // the operands of d, picked with selects (a dynamic register index would go to memory)
      T rr = T(0), mk = T(0), sk = T(0);
#pragma unroll
      for (int vv = 0; vv < 3; ++vv)
#pragma unroll
        for (int kk = 0; kk < ND; ++kk) rr = (vv * ND + kk == d) ? r[vv][kk] : rr;
#pragma unroll
      for (int kk = 0; kk < ND; ++kk) mk = kk == k ? minv[kk] : mk;
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) sk = (kk == k) ? (v == 1 ? src1[kk] : (v == 2 ? src2[kk] : sk)) : sk;
      T L = rr * mk;
      if (k < 3) L += sk;
      if (d == 0) L += rain;
      update(v, k, L);
    }
  }
  if (bad) atomicOr(s.err, ERR_NONFINITE);
}

// ------------------------------------------------------------------------ wetting/drying front
// Float form with wetting/drying.  Near the shoreline the vertex depths sit within a float rounding
// of the dry threshold h0 (a surface elevation of metres carries a float ulp of ~1e-7 m, against
// the 1e-10 m tolerance of the depth tests), so a float evaluation there flips wet/dry decisions
// that the FP64 arithmetic takes the other way.  The elements at the wetting/drying front are
// therefore updated in double, from double statics (DevMesh geo_d / lima_d / hbq_d), with the same
// operations as the FP64 form: area, edge and source arithmetic, limiter and wet/dry.  An element
// is at the front, given the flags at the start of the stage, if it is
//  - partially wet;
//  - wet, with a face neighbour that is not wet;
//  - dry, with a face neighbour that is not dry, an open-ocean or river edge, or rain falling.
// A dry element whose neighbours are all dry is left to the float path: walls on every edge and no
// momentum keep its surface exactly unchanged in either arithmetic (and wet/dry then removes the
// float momentum and restores the flat depth).  The element kernels list the front elements, and
// two small kernels spread over all SMs update them (k_front) and limit them (k_limwd_front).
constexpr uint8_t NBC_LAND = 255;  // neighbour code across a land edge
constexpr uint8_t NBC_OPEN = 254;  // across an open-ocean or river edge

// fe: the element's flag; n0..n2: its neighbours' flags (0 wet, 1 partially wet, 2 dry) or NBC_*.
__device__ __forceinline__ bool is_front(uint8_t fe, uint8_t n0, uint8_t n1, uint8_t n2, bool rain) {
  if (fe == 1) return true;
  if (fe == 0) return (n0 == 1 || n0 == 2) || (n1 == 1 || n1 == 2) || (n2 == 1 || n2 == 2);
  return rain || (n0 != 2 && n0 != NBC_LAND) || (n1 != 2 && n1 != NBC_LAND) || (n2 != 2 && n2 != NBC_LAND);
}

// Append flat index id to the front list (called only by the threads whose element is at the
// front): one atomic per group of converged threads.
__device__ __forceinline__ void front_append(const StageArgs &s, int id) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(s.fcnt, (unsigned)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  s.flist[base + __popc(mask & ((1u << lane) - 1u))] = id;
}

// The element kernels of a stage reset the previous stage's list counter (all its readers ran).
__device__ __forceinline__ void front_reset_prev(const StageArgs &s) {
  if (s.fcnt_prev && blockIdx.x == 0 && threadIdx.x == 0) *s.fcnt_prev = 0u;
}

template <int P, typename T, bool SPLIT, typename MT = T>
__device__ __forceinline__ void element_body(const DevMesh &m, const StageArgs &s, const Phys &ph,
                                             const int write_rhs, const int e,
                                             const T (*s_phe)[nqe_of(P)][nd_of(P)]) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const Tab<T> &tb = ctab<T>(P);
  const int ne = m.ne;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (s.cls) {  // s.cls implies s.wd; the front elements are left to k_front
      uint8_t nf[3];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const int j = m.nbr[(size_t)l * ne + e];
        nf[l] = j >= 0 ? s.wd[j] : (j == NBR_LAND ? NBC_LAND : NBC_OPEN);
      }
      const bool front = is_front(s.wd[e], nf[0], nf[1], nf[2], ph.rain != 0.0);
      s.cls[e] = front ? 1 : 0;
      if (front) {
        front_append(s, s.fbase + e);
        return;
      }
    }
  }
  const T g = pc<T>(ph.g, ph.f.g), sqg = pc<T>(ph.sqrt_g, ph.f.sqrt_g);
  ElemCtx<P, T> c;
  elem_load<P, T>(m, s.uin, e, c);
  const T *geo = (const T *)m.geo;
  const T (&w)[3][ND] = c.w;
  const T (&hb)[3] = c.hb;
  const double (&hbd)[3] = c.hbd;
  T r[3][ND];
  elem_area<P, T>(c, ph, r, m, e);

  // ---------------- edge integrals (Alg. 2 + Alg. 3), gathered per element in a fixed order
  const uint8_t fe = s.wd ? s.wd[e] : 0;
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    const int j = m.nbr[(size_t)l * ne + e];
    const T hl = geo[(GEO_HL0 + l) * (size_t)ne + e];
    T Fh[NQE][3];
    bool weighted = false;  // Fh already carries hl * w_q (flux read from the edge kernel)
    bool have = false;      // Fh filled
    if constexpr (SPLIT) {
      if (j >= 0) {
        const int ed = m.eledge[(size_t)l * ne + e];
        const bool minus = ed < 0;
        const int id = ed & 0x7fffffff;
        if (s.emode[id]) {
          const T *F = (const T *)s.eflux;
#pragma unroll
          for (int q = 0; q < NQE; ++q) {
            const int qi = minus ? NQE - 1 - q : q;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
              const T f = F[(size_t)(v * NQE + qi) * m.nint + id];
              Fh[q][v] = minus ? -f : f;
            }
          }
          weighted = have = true;
        }
      }
    }
    if (!have) {
      // own traces at the edge Gauss points and h_b there (end nodes of local edge l, vertex
      // (l+1)%3 -> (l+2)%3, selected without dynamic register indexing)
      const T nx = geo[(GEO_NX0 + l) * (size_t)ne + e], ny = geo[(GEO_NY0 + l) * (size_t)ne + e];
      const T hbA = l == 0 ? hb[1] : (l == 1 ? hb[2] : hb[0]);
      const T hbB = l == 0 ? hb[2] : (l == 1 ? hb[0] : hb[1]);
      T wp[NQE][3], hbq[NQE];
#pragma unroll
      for (int q = 0; q < NQE; ++q) {
#pragma unroll
        for (int v = 0; v < 3; ++v) wp[q][v] = modal_value<ND, T>(w[v], s_phe[l][q]);
        hbq[q] = T(0.5) * ((T(1) - tb.se[q]) * hbA + (T(1) + tb.se[q]) * hbB);
      }
      bool flows = false;
      if (j >= 0 && !SPLIT) {
        const int lj = (m.nle[e] >> (2 * l)) & 3;
        const double hbAd = l == 0 ? hbd[1] : (l == 1 ? hbd[2] : hbd[0]);
        const double hbBd = l == 0 ? hbd[2] : (l == 1 ? hbd[0] : hbd[1]);
        flows = edge_flows<P>(ph, fe, s.wd ? s.wd[j] : 0, s.uin, ne, e, l, j, lj, hbAd, hbBd);
        if (flows) {
          T wn[3][ND];
          load_modes<P, T>(s.uin, ne, j, wn);
#pragma unroll
          for (int q = 0; q < NQE; ++q) {
            T wm[3];
#pragma unroll
            for (int v = 0; v < 3; ++v) wm[v] = modal_value<ND, T>(wn[v], s_phe[lj][NQE - 1 - q]);
            numflux(ph, g, sqg, wp[q], wm, hbq[q], nx, ny, Fh[q]);
          }
        }
      }
      if (j == NBR_RIVER) {
#pragma unroll
        for (int q = 0; q < NQE; ++q) river(ph, g, sqg, wp[q], hbq[q], nx, ny, Fh[q]);
      } else if (j == NBR_OPEN) {
        const double ts = stage_time(s.clk, s.tau, s.tide_t);
        const T zt = from_d<T>(ph.tide_amp * sin(ph.tide_omega * ts + ph.tide_phase));
#pragma unroll
        for (int q = 0; q < NQE; ++q) {
          const T wo[3] = {zt, wp[q][1], wp[q][2]};
          numflux(ph, g, sqg, wp[q], wo, hbq[q], nx, ny, Fh[q]);
        }
      } else if (!flows) {  // land boundary, or an interior edge closed by wetting/drying
#pragma unroll
        for (int q = 0; q < NQE; ++q) wall(ph, g, sqg, wp[q], hbq[q], nx, ny, Fh[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQE; ++q) {
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const T f = weighted ? Fh[q][v] : (hl * tb.we[q]) * Fh[q][v];
        r[v][0] -= f;  // psi_00 = 1
#pragma unroll
        for (int k = 1; k < ND; ++k) r[v][k] -= f * s_phe[l][q][k];
      }
    }
  }

  elem_finish<P, T, MT>(m, s, ph, write_rhs, e, c, r);
}

// List entry i -> block i mod gridDim.x, lane i / gridDim.x: consecutive entries (neighbouring
// front elements) go to different SMs, and an SM's few front elements share one warp, so the
// double work of a short list spreads over the whole GPU instead of a few SMs' FP64 pipes.
__device__ __forceinline__ unsigned front_entry0() { return blockIdx.x + gridDim.x * threadIdx.x; }
__device__ __forceinline__ unsigned front_stride() { return gridDim.x * blockDim.x; }

// Weighted numerical flux at Gauss point q of local edge l of element e (double, as element_body
// computes it without the split variant's edge slots): hl w_q Fhat.n, n outward from e.
template <int P>
__device__ __forceinline__ void front_edge_point(const DevMesh &md, const StageArgs &s, const Phys &ph,
                                                 const ElemCtx<P, double> &c, const int e, const int l, const int q,
                                                 double f[3]) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const Tab<double> &tb = c_td[P - 1];
  const int ne = md.ne;
  const double g = ph.g, sqg = ph.sqrt_g;
  const double *geo = md.geo_d;
  const int j = md.nbr[(size_t)l * ne + e];
  const double hl = geo[(GEO_HL0 + l) * (size_t)ne + e];
  const double nx = geo[(GEO_NX0 + l) * (size_t)ne + e], ny = geo[(GEO_NY0 + l) * (size_t)ne + e];
  const double hbA = l == 0 ? c.hb[1] : (l == 1 ? c.hb[2] : c.hb[0]);
  const double hbB = l == 0 ? c.hb[2] : (l == 1 ? c.hb[0] : c.hb[1]);
  double wp[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) wp[v] = modal_value<ND, double>(c.w[v], tb.phe[l][q]);
  const double hbq = 0.5 * ((1.0 - tb.se[q]) * hbA + (1.0 + tb.se[q]) * hbB);
  double F[3];
  bool flows = false;
  if (j >= 0) {
    const int lj = (md.nle[e] >> (2 * l)) & 3;
    flows = edge_flows<P>(ph, s.wd ? s.wd[e] : 0, s.wd ? s.wd[j] : 0, s.uin, ne, e, l, j, lj, hbA, hbB);
    if (flows) {
      double wm[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        double x = s.uin[(size_t)(v * ND) * ne + j];  // psi_00 = 1
#pragma unroll
        for (int k = 1; k < ND; ++k) x += s.uin[(size_t)(v * ND + k) * ne + j] * tb.phe[lj][NQE - 1 - q][k];
        wm[v] = x;
      }
      numflux(ph, g, sqg, wp, wm, hbq, nx, ny, F);
    }
  }
  if (j == NBR_RIVER) {
    river(ph, g, sqg, wp, hbq, nx, ny, F);
  } else if (j == NBR_OPEN) {
    const double ts = stage_time(s.clk, s.tau, s.tide_t);
    const double wo[3] = {ph.tide_amp * sin(ph.tide_omega * ts + ph.tide_phase), wp[1], wp[2]};
    numflux(ph, g, sqg, wp, wo, hbq, nx, ny, F);
  } else if (!flows) {  // land boundary, or an interior edge closed by wetting/drying
    wall(ph, g, sqg, wp, hbq, nx, ny, F);
  }
  const double wgt = hl * tb.we[q];
#pragma unroll
  for (int v = 0; v < 3; ++v) f[v] = wgt * F[v];
}

// Sum over the `width` lanes of an aligned lane group (width a power of two, at most 32).
template <int WIDTH>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
  for (int o = WIDTH / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Lanes per front element in the double update: a power of two at least as large as the number of
// area points (NQA) and of edge Gauss points (3 NQE), which are equal at p = 1 (6) and p = 2 (12).
template <int P>
__host__ __device__ constexpr int front_lanes() { return P == 1 ? 8 : 16; }

// The double update of front elements by groups of lanes.  One thread's double update is a latency
// chain of thousands of instructions on GB300's narrow FP64 pipe, and a warp instruction holds that
// pipe for the same time whatever the number of active lanes; so each element gets a group of
// LPE = front_lanes lanes (four elements per warp at p = 1, two at p = 2), and lane j < NQA of a
// group evaluates both area point j and edge Gauss point j (local edge j / NQE, point j % NQE):
// no lane waits while another kind of point is computed.  The group sums the contributions (every
// lane gets the totals); every lane closes the area integrals and adds the edge terms, and lane j
// applies the inverse mass matrix, the closed-form sources and the RK stage to the degrees of
// freedom j, j + LPE, ... (elem_finish): 2 rounds at p = 1 and p = 2 instead of 9 or 18 on one
// lane.  Every lane of the warp calls this (the sums shuffle across the whole warp); has: the
// group has an element.
template <int P>
__device__ __forceinline__ void front_update_group(const DevMesh &m, const StageArgs &s, const Phys &ph,
                                                   const int write_rhs, const bool has, const int e) {
  constexpr int ND = nd_of(P), NQA = nqa_of(P), NQE = nqe_of(P);
  constexpr int LPE = front_lanes<P>();
  static_assert(NQA == 3 * NQE && NQA <= LPE, "one area point and one edge point per lane");
  const int sub = threadIdx.x & (LPE - 1);
  DevMesh md = m;
  md.geo = m.geo_d;
  md.lima = m.lima_d;
  md.hbq = m.hbq_d;
  ElemCtx<P, double> c;
  double ra[3][ND], re[3][ND];
  AreaSums<P, double> a;
  area_zero<P, double>(ra, a);
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int k = 0; k < ND; ++k) re[v][k] = 0.0;
  if (has) {
    elem_load<P, double>(md, s.uin, e, c);
    if (sub < NQA) {
      area_point<P, double>(c, ph, ra, a, md, e, sub);
      const int l = sub / NQE, q = sub % NQE;
      double f[3];
      front_edge_point<P>(md, s, ph, c, e, l, q, f);
      const Tab<double> &tb = c_td[P - 1];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        re[v][0] = -f[v];  // psi_00 = 1
#pragma unroll
        for (int k = 1; k < ND; ++k) re[v][k] = -(f[v] * tb.phe[l][q][k]);
      }
      if constexpr (P == 2) {
        // area_close scales (r - friction) by |J| and the edge terms are added after it: fold
        // both into this lane's r (edge terms divided by |J|), so that one array is summed
        const double idJ = rcp_d(c.dJ);
#pragma unroll
        for (int k = 0; k < ND; ++k) {
          ra[0][k] = fma(re[0][k], idJ, ra[0][k]);
          ra[1][k] = fma(re[1][k], idJ, ra[1][k] - a.fr[0][k]);
          ra[2][k] = fma(re[2][k], idJ, ra[2][k] - a.fr[1][k]);
          a.fr[0][k] = a.fr[1][k] = 0.0;
        }
      }
    }
  }
  if constexpr (P == 2) {
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int k = 0; k < ND; ++k) ra[v][k] = group_sum<LPE>(ra[v][k]);
  } else {  // at P = 1 the area points add to a.G
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int k = 0; k < ND; ++k) re[v][k] = group_sum<LPE>(re[v][k]);
#pragma unroll
    for (int i = 0; i < 4; ++i) a.G[i] = group_sum<LPE>(a.G[i]);
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      a.fr[0][k] = group_sum<LPE>(a.fr[0][k]);
      a.fr[1][k] = group_sum<LPE>(a.fr[1][k]);
    }
  }
  if (has) {  // every lane of the group holds the sums: each finishes some degrees of freedom
    area_close<P, double>(c, ph, ra, a);
    if constexpr (P == 1) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < ND; ++k) ra[v][k] += re[v][k];
    }
    StageArgs sd = s;
    sd.cls = nullptr;
    elem_finish<P, double, float, LPE>(md, sd, ph, write_rhs, e, c, ra, nullptr, nullptr, 0, sub);
  }
}

// The listed front elements of one model (flat index = element): 32 / LPE consecutive entries per
// warp; warp w of the list is warp w / gridDim.x of block w % gridDim.x, so that a short list
// spreads over every SM (one busy warp per block) instead of filling the first blocks.
template <int P>
__global__ void __launch_bounds__(128) k_front(const DevMesh m, const StageArgs s, const Phys ph, const int write_rhs) {
  constexpr int EPW = 32 / front_lanes<P>();  // elements per warp
  const unsigned n = *s.fcnt;
  const unsigned w = blockIdx.x + gridDim.x * (threadIdx.x >> 5), nw = gridDim.x * (blockDim.x >> 5);
  const unsigned slot = (threadIdx.x & 31) / front_lanes<P>();
  for (unsigned i0 = w * EPW; i0 < n; i0 += nw * EPW) {  // the same trip count in every lane of a warp
    const unsigned i = i0 + slot;
    front_update_group<P>(m, s, ph, write_rhs, i < n, i < n ? s.flist[i] : 0);
  }
}

// The float form's bounds keep the register counts these kernels had before the out-of-line front
// path (whose needs would otherwise raise the whole kernel's allocation): 2 or 3 resident
// 256-thread blocks per SM.
template <int P, typename T, bool SPLIT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? ((P == 1 && SPLIT) ? 3 : 2) : 1)
    k_element(const DevMesh m, const StageArgs s, const Phys ph, const int write_rhs) {
  __shared__ T s_phe[3][nqe_of(P)][nd_of(P)];
  load_phe<P, T>(s_phe);
  __syncthreads();
  front_reset_prev(s);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.nact) return;  // own elements and the first ghost layer of a part
  element_body<P, T, SPLIT>(m, s, ph, write_rhs, e, s_phe);
}

// ------------------------------------------------------------------------ tiled element update
// One block per tile of `tl.tile` consecutive elements (Hilbert order keeps a tile compact).  The
// tile's states are staged in shared memory; the block's threads compute every edge touching the
// tile once (an edge between two tiles is computed identically by both) and leave the weighted
// flux of each (element, local edge, Gauss point) in shared memory; after one barrier each thread
// finishes its element (area integrals, gather in the fixed local-edge order, inverse mass, RK).
// Shared memory: state [3*ND][tile] and flux slots [3][NQE][3][tile] in T, wet/dry flags [tile],
// front codes [3][tile] (per local edge: the neighbour's flag or NBC_*).
// ef: the float form with the inline vortex adds TILE_EF rows of the element phase's inputs (J^-1,
// det J, vertex h_b, vertex x and y), copied asynchronously at the start of the tile.
constexpr int TILE_EF = 14;
template <int P, typename T>
__host__ __device__ constexpr size_t tile_smem_bytes(int tile, bool ef = false) {
  return sizeof(T) * 3 * nd_of(P) * tile + sizeof(T) * 9 * nqe_of(P) * tile +
         (ef && sizeof(T) == sizeof(float) ? sizeof(float) * TILE_EF * tile : 0) + 4 * tile;
}

// Asynchronous 4-byte global -> shared copy (cp.async, cached in L1) and its completion.
__device__ __forceinline__ void cp_async4(void *dst_shared, const void *src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
  asm volatile(
      "{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %1;\n\tcp.async.ca.shared.global [%0], [g], 4;\n\t}" ::"r"(d),
      "l"(src_global)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Modes of element e: from the tile's shared-memory copy (already in T) or, for a neighbour in
// another tile, from global memory.
template <int P, typename T>
__device__ __forceinline__ void tile_modes(const T *s_u, int B, const double *u, int ne, int e, bool local,
                                           int li, T w[3][nd_of(P)]) {
#pragma unroll
  for (int v = 0; v < 3; ++v)
#pragma unroll
    for (int k = 0; k < nd_of(P); ++k) {
      const int row = v * nd_of(P) + k;
      w[v][k] = local ? s_u[row * B + li] : from_d<T>(__ldg(&u[(size_t)row * ne + e]));
    }
}

template <int P, typename T>
__device__ __forceinline__ void tile_edge(const DevMesh &m, const DevTiles &tl, const StageArgs &s, const Phys &ph,
                                          const int x, const int e0, const T *s_ud, T *s_slot,
                                          const uint8_t *s_wd, uint8_t *s_fr,
                                          const T (*s_phe)[nqe_of(P)][nd_of(P)]) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const Tab<T> &tb = ctab<T>(P);
  const int B = tl.tile, ne = m.ne;
  const T g = pc<T>(ph.g, ph.f.g), sqg = pc<T>(ph.sqrt_g, ph.f.sqrt_g);
  const int a = tl.ea[x], b = tl.eb[x];
  const unsigned code = tl.code[x];
  const int la = code & 3u, lb = (code >> 2) & 3u;
  const bool ina = (code >> 4) & 1u, inb = (code >> 5) & 1u;
  const T *tg = (const T *)tl.geo;
  const T nx = tg[x], ny = tg[tl.n + x], hl = tg[2 * (size_t)tl.n + x];
  T wa[3][ND];
  tile_modes<P, T>(s_ud, B, s.uin, ne, a, ina, a - e0, wa);
  T ta[NQE][3], hbq[NQE];
#pragma unroll
  for (int q = 0; q < NQE; ++q) {
#pragma unroll
    for (int v = 0; v < 3; ++v) ta[q][v] = modal_value<ND, T>(wa[v], s_phe[la][q]);
    hbq[q] = ((const T *)tl.hbq)[(size_t)q * tl.n + x];  // h_b at the point, host-computed
  }
  // slot of (element li, local edge l, Gauss point q, variable v)
  auto slot = [&](int li, int l, int q, int v) -> T & { return s_slot[(size_t)((l * NQE + q) * 3 + v) * B + li]; };
  if (b >= 0) {
    const uint8_t fa = s.wd ? (ina ? s_wd[a - e0] : s.wd[a]) : 0;
    const uint8_t fb = s.wd ? (inb ? s_wd[b - e0] : s.wd[b]) : 0;
    // the edge's vertex depths decide only an edge with exactly one dry side
    const bool one_dry = (fa == 2) != (fb == 2);
    const double hAd = one_dry ? tl.hb[x] : 0.0, hBd = one_dry ? tl.hb[tl.n + x] : 0.0;
    const bool flows = edge_flows<P>(ph, fa, fb, s.uin, ne, a, la, b, lb, hAd, hBd);
    if (s.cls) {  // front test: each in-tile side records the other side's flag
      if (ina) s_fr[la * B + a - e0] = fb;
      if (inb) s_fr[lb * B + b - e0] = fa;
    }
    T wb[3][ND];
    tile_modes<P, T>(s_ud, B, s.uin, ne, b, inb, b - e0, wb);
#pragma unroll
    for (int q = 0; q < NQE; ++q) {
      T tbq[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) tbq[v] = modal_value<ND, T>(wb[v], s_phe[lb][NQE - 1 - q]);
      const T wgt = hl * tb.we[q];
      if (flows) {
        T f[3];
        numflux(ph, g, sqg, ta[q], tbq, hbq[q], nx, ny, f);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          if (ina) slot(a - e0, la, q, v) = wgt * f[v];
          if (inb) slot(b - e0, lb, NQE - 1 - q, v) = -(wgt * f[v]);
        }
      } else {  // closed by wetting/drying: each side sees a wall
        if (ina) {
          T f[3];
          wall(ph, g, sqg, ta[q], hbq[q], nx, ny, f);
#pragma unroll
          for (int v = 0; v < 3; ++v) slot(a - e0, la, q, v) = wgt * f[v];
        }
        if (inb) {
          T f[3];
          wall(ph, g, sqg, tbq, hbq[q], -nx, -ny, f);
#pragma unroll
          for (int v = 0; v < 3; ++v) slot(b - e0, lb, NQE - 1 - q, v) = wgt * f[v];
        }
      }
    }
  } else if (b == NBR_LAND || b == NBR_RIVER) {
    if (s.cls) s_fr[la * B + a - e0] = b == NBR_LAND ? NBC_LAND : NBC_OPEN;
#pragma unroll
    for (int q = 0; q < NQE; ++q) {
      T f[3];
      if (b == NBR_RIVER)
        river(ph, g, sqg, ta[q], hbq[q], nx, ny, f);
      else
        wall(ph, g, sqg, ta[q], hbq[q], nx, ny, f);
#pragma unroll
      for (int v = 0; v < 3; ++v) slot(a - e0, la, q, v) = hl * tb.we[q] * f[v];
    }
  } else {
    if (s.cls) s_fr[la * B + a - e0] = NBC_OPEN;
    const double ts = stage_time(s.clk, s.tau, s.tide_t);
    const T zt = from_d<T>(ph.tide_amp * sin(ph.tide_omega * ts + ph.tide_phase));
#pragma unroll
    for (int q = 0; q < NQE; ++q) {
      const T wo[3] = {zt, ta[q][1], ta[q][2]};
      T f[3];
      numflux(ph, g, sqg, ta[q], wo, hbq[q], nx, ny, f);
#pragma unroll
      for (int v = 0; v < 3; ++v) slot(a - e0, la, q, v) = hl * tb.we[q] * f[v];
    }
  }
}

// One tile: stage, edges, barrier, elements.  Called with the whole block (uses __syncthreads).
template <int P, typename T>
__device__ __forceinline__ void tile_body(const DevMesh &m, const DevTiles &tl, const StageArgs &s, const Phys &ph,
                                          const int write_rhs, const int tile, unsigned char *smem_raw,
                                          const T (*s_phe)[nqe_of(P)][nd_of(P)]) {
  constexpr int ND = nd_of(P), NQE = nqe_of(P);
  const int B = tl.tile, ne = m.ne;
  // float form with the inline vortex: the element phase's inputs are prefetched to shared memory
  // (the launch sized the dynamic shared memory with tile_smem_bytes(tile, true))
  const bool ef = sizeof(T) == sizeof(float) && s.frc_inline;
  T *s_ud = reinterpret_cast<T *>(smem_raw);
  T *s_slot = s_ud + (size_t)3 * ND * B;
  float *s_ef = reinterpret_cast<float *>(s_slot + (size_t)9 * NQE * B);
  uint8_t *s_wd = reinterpret_cast<uint8_t *>(s_ef + (ef ? (size_t)TILE_EF * B : 0));
  uint8_t *s_fr = s_wd + B;
  const int e0 = tile * B, i = threadIdx.x;
  const int nloc = min(B, m.nact - e0);  // the tiles cover the updated elements [0, nact)
  __shared__ double s_ctr[2];  // storm centre at the stage time, once per block (inline vortex)
  if (s.frc_inline && i == 0) storm_center(ph, stage_time(s.clk, s.tau, s.tide_t), s_ctr[0], s_ctr[1]);
  if (ef) {
    // in flight while the states are staged and the edges computed
    if (i < nloc) {
      const float *geo = (const float *)m.geo;
#pragma unroll
      for (int r = 0; r < 5; ++r) cp_async4(&s_ef[r * B + i], &geo[(size_t)(GEO_RX + r) * ne + e0 + i]);
#pragma unroll
      for (int r = 0; r < 9; ++r) cp_async4(&s_ef[(5 + r) * B + i], &m.elf[(size_t)r * ne + e0 + i]);
    }
    cp_async_commit();
  }
  if (i < nloc) {
#pragma unroll
    for (int r = 0; r < 3 * ND; ++r) s_ud[r * B + i] = from_d<T>(__ldg(&s.uin[(size_t)r * ne + e0 + i]));
    s_wd[i] = s.wd ? s.wd[e0 + i] : 0;
    s_fr[i] = s_fr[B + i] = s_fr[2 * B + i] = NBC_LAND;  // every slot is rewritten by its edge
  }
  __syncthreads();
  const int beg = tl.start[tile], end = tl.start[tile + 1];
  for (int x = beg + i; x < end; x += B) tile_edge<P, T>(m, tl, s, ph, x, e0, s_ud, s_slot, s_wd, s_fr, s_phe);
  if (ef) cp_async_wait_all();  // each thread reads only the rows it copied
  __syncthreads();
  bool front = false;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (s.cls && i < nloc) {  // the front elements are left to the front kernels
      front = is_front(s_wd[i], s_fr[i], s_fr[B + i], s_fr[2 * B + i], ph.rain != 0.0);
      s.cls[e0 + i] = front ? 1 : 0;
      if (front) front_append(s, s.fbase + e0 + i);
    }
  }
  if (i < nloc && !front) {
    const int e = e0 + i;
    ElemCtx<P, T> c;
    if (ef) {
      c.rx = s_ef[i];
      c.ry = s_ef[B + i];
      c.sx = s_ef[2 * B + i];
      c.sy = s_ef[3 * B + i];
      c.dJ = s_ef[4 * B + i];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        c.hb[a] = s_ef[(5 + a) * B + i];
        c.hbd[a] = 0.0;  // the double vertex depths serve the untiled variants only
      }
    } else {
      elem_load_geom<P, T>(m, e, c);
    }
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int k = 0; k < ND; ++k) c.w[v][k] = s_ud[(v * ND + k) * B + i];
    T r[3][ND];
    elem_area<P, T>(c, ph, r, m, e);
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int q = 0; q < NQE; ++q)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const T f = s_slot[(size_t)((l * NQE + q) * 3 + v) * B + i];
          r[v][0] -= f;  // psi_00 = 1
#pragma unroll
          for (int k = 1; k < ND; ++k) r[v][k] -= f * s_phe[l][q][k];
        }
    elem_finish<P, T>(m, s, ph, write_rhs, e, c, r, s_ctr, ef ? (const T *)&s_ef[8 * B + i] : nullptr, B);
  }
  __syncthreads();  // the shared-memory tile is reused by the block's next tile
}

// WIDE: the float form at p = 1 held to 48 registers (5 resident 256-thread blocks per SM instead
// of 4): more latency hiding on large meshes, a nearly empty second wave on small ones.
template <int P, typename T, bool WIDE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (P == 1 ? (WIDE ? 5 : 4) : 2) : 1)
    k_tile(const DevMesh m, const DevTiles tl, const StageArgs s, const Phys ph, const int write_rhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_phe[3][nqe_of(P)][nd_of(P)];
  load_phe<P, T>(s_phe);
  front_reset_prev(s);
  tile_body<P, T>(m, tl, s, ph, write_rhs, blockIdx.x, smem_raw, s_phe);
}

// ------------------------------------------------------------------------ SLOPELIM + WETDRY
__device__ __forceinline__ float minmod(float a, float b) {
  if (a > 0.f && b > 0.f) return a < b ? a : b;
  if (a < 0.f && b < 0.f) return a > b ? a : b;
  return 0.f;
}
// Double minmod from the bits (integer pipe): opposite signs (or a zero) give 0; otherwise the
// operand of smaller magnitude (b on a tie), as the comparisons of the float version select.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ma = (unsigned long long)ia << 1, mb = (unsigned long long)ib << 1;  // |a|, |b|
  if ((ia ^ ib) < 0 || ma == 0 || mb == 0) return 0.0;
  return ma < mb ? a : b;
}
// a != b as numbers for finite values (+0 equals -0), from the bits
__device__ __forceinline__ bool differs(float a, float b) { return a != b; }
__device__ __forceinline__ bool differs(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ia != ib && ((ia | ib) << 1) != 0;
}

constexpr double WD_TOL = 1e-10;  // m: depths within this of h0 count as "at h0"

// Cockburn-Shu minmod limiter on the linear modes of each variable (nu = 1.5), against
// neighbour means read from `mean` (written by the element kernel, so unaffected by this pass);
// then the wet/dry operator (double): vertex depths of the linear part, flatten if the mean depth
// <= h0 (dry), else lift vertices below h0 to h0 and rescale the others' excess (mean kept);
// momentum removed where dry, or partially wet with the mean surface below the highest bed of the
// vertices at h0; at p = 2 limited or non-wet elements drop their quadratic modes.
// Rare path of the limiter, kept out of line so that its divisions are not executed
// speculatively for every element: rescale the limited midpoint deviations so that they sum to
// zero (theta+/- rule) and rebuild the linear modes from the midpoints of local edges 0 and 1.
template <int P, typename T>
__device__ __noinline__ void limiter_rebuild(const T d0, const T d1, const T d2, double *u1, double *u2) {
  const Tab<T> &tb = ctab<T>(P);
  const T d[3] = {d0, d1, d2};
  if constexpr (sizeof(T) == sizeof(double)) {
    // the same arithmetic with the sign tests, the maxima with zero and the ordering of the two
    // non-negative sums taken from the bits (integer pipe)
    double dp[3], dn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const bool nonneg = __double_as_longlong(d[i]) >= 0;  // sign bit clear
      dp[i] = nonneg ? d[i] : 0.0;
      dn[i] = nonneg ? 0.0 : -d[i];
    }
    const double pos = dp[0] + dp[1] + dp[2], neg = dn[0] + dn[1] + dn[2];
    double tp = 0.0, tm = 0.0;
    const long long bp = __double_as_longlong(pos), bn = __double_as_longlong(neg);
    if (bp > 0 && bn > 0) {  // both positive
      if (bn <= bp) {
        tp = ratio_t(neg, pos);
        tm = 1.0;
      } else {
        tp = 1.0;
        tm = ratio_t(pos, neg);
      }
    }
    double dh[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) dh[i] = tp * dp[i] - tm * dn[i];
    // inverse of the midpoint map of limwd_body: dh0 = (u1 + u2)/2, dh1 = (u2 - u1)/2
    *u1 = dh[0] - dh[1];
    *u2 = dh[0] + dh[1];
    return;
  }
  T pos = 0, neg = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    pos += d[i] > T(0) ? d[i] : T(0);
    neg += d[i] < T(0) ? -d[i] : T(0);
  }
  T tp = T(0), tm = T(0);
  if (pos > T(0) && neg > T(0)) {
    if (neg <= pos) {
      tp = ratio_t(neg, pos);
      tm = T(1);
    } else {
      tp = T(1);
      tm = ratio_t(pos, neg);
    }
  }
  T dh[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) dh[i] = tp * (d[i] > T(0) ? d[i] : T(0)) - tm * (d[i] < T(0) ? -d[i] : T(0));
  *u1 = to_d<T>((dh[0] * tb.phm[1][2] - tb.phm[0][2] * dh[1]) * tb.lim_idet);
  *u2 = to_d<T>((tb.phm[0][1] * dh[1] - dh[0] * tb.phm[1][1]) * tb.lim_idet);
}

// The limiter's six decomposition weights of element e (rows of m.lima), loaded once for the three
// variables (the limiter writes the state through a pointer, so the compiler could not reuse them).
template <typename T>
__device__ __forceinline__ void limiter_weights(const DevMesh &m, const int e, T A[6]) {
  const T *L = (const T *)m.lima;
#pragma unroll
  for (int r = 0; r < 6; ++r) A[r] = L[(size_t)r * m.ne + e];
}

// Cockburn-Shu limiting of variable v of element e (see limwd_body); nb: the face neighbours, code:
// the limiter's neighbour pairs (m.limj[e]), A: its weights (limiter_weights).  Returns true when
// the linear modes were rebuilt.
template <int P, typename T, bool FILTER = true>
__device__ __forceinline__ bool limit_variable(const DevMesh &m, double *u, const T *mean, const int e, const int v,
                                               const int nb[3], const unsigned code, const uint8_t *fcls,
                                               const T A[6]) {
  constexpr int ND = nd_of(P);
  const int ne = m.ne;
  const Tab<T> &tb = ctab<T>(P);
  const T nu = T(1.5);
  const double d0 = u[(size_t)(v * ND) * ne + e];
  const double d1 = u[(size_t)(v * ND + 1) * ne + e];
  const double d2 = u[(size_t)(v * ND + 2) * ne + e];
  T db3[3];  // neighbour means (stored in T: the float form rounds them once, when written)
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (nb[j] < 0) {
      db3[j] = from_d<T>(d0);
    } else if (sizeof(T) == sizeof(double) && fcls && !fcls[nb[j]]) {
      db3[j] = (T)u[(size_t)(v * ND) * ne + nb[j]];
    } else {
      db3[j] = mean[(size_t)v * ne + nb[j]];
    }
  }
  if constexpr (sizeof(T) == sizeof(double) && FILTER) {
    // Filtered predicate (after Shewchuk's floating-point filters): a float evaluation with an
    // error margin well above its rounding proves, when it can, that minmod returns the midpoint
    // deviation at every edge, i.e. the limiter leaves this variable untouched; only the
    // undecided cases run the exact double test below.  Zero slopes are untouched exactly.
    if (((__double_as_longlong(d1) | __double_as_longlong(d2)) << 1) == 0) return false;  // both +-0
    const float f0 = d2f(d0), f1 = d2f(d1), f2 = d2f(d2);
    const Tab<float> &tf = ctab<float>(P);
    bool sure = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float p1 = tf.phm[i][1], p2 = tf.phm[i][2];
      const float ut = f1 * p1 + f2 * p2;
      const float eu = 1e-6f * (fabsf(f1 * p1) + fabsf(f2 * p2));
      const unsigned c = (code >> (4 * i)) & 15u;
      const int j1 = c & 3, j2 = c >> 2;
      float db = 0.f, ed = 0.f;
      if (j1 != 3) {
        const float a1 = d2f(A[2 * i]), a2 = d2f(A[2 * i + 1]);
        const float b1 = d2f(db3[j1]), b2 = d2f(db3[j2]);
        db = 1.5f * (a1 * (b1 - f0) + a2 * (b2 - f0));
        ed = 1e-6f * 1.5f * (fabsf(a1) * (fabsf(b1) + fabsf(f0)) + fabsf(a2) * (fabsf(b2) + fabsf(f0))) + 1e-30f;
      }
      const bool ok = (fabsf(ut) > eu) && (fabsf(db) > ed) && ((ut > 0.f) == (db > 0.f)) &&
                      (fabsf(ut) + eu < fabsf(db) - ed);
      sure = sure && ok;
    }
    if (sure) return false;
  }
  const T u0 = from_d<T>(d0);
  const T u1 = from_d<T>(d1);
  const T u2 = from_d<T>(d2);
  T dd[3];  // neighbour mean minus own mean
#pragma unroll
  for (int j = 0; j < 3; ++j) dd[j] = db3[j] - u0;
  // midpoint deviations of the linear part; in double from the linear Dubiner modes at the
  // edge midpoints, (1/2, 1/2), (-1/2, 1/2) and (0, -1) (Eq. dubiner): the same values as the
  // table products (halving is exact), from two additions
  T ut[3];
  if constexpr (sizeof(T) == sizeof(double)) {
    ut[0] = half_exact(u1 + u2);
    ut[1] = half_exact(u2 - u1);
    ut[2] = -u2;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) ut[i] = u1 * tb.phm[i][1] + u2 * tb.phm[i][2];
  }
  T d[3];
  bool act = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const unsigned c = (code >> (4 * i)) & 15u;
    const int j1 = c & 3, j2 = c >> 2;
    // select without dynamic register indexing (which would place dd in local memory)
    const T x1 = j1 == 0 ? dd[0] : (j1 == 1 ? dd[1] : dd[2]);
    const T x2 = j2 == 0 ? dd[0] : (j2 == 1 ? dd[1] : dd[2]);
    T db = T(0);
    if (j1 != 3) db = A[2 * i] * x1 + A[2 * i + 1] * x2;
    d[i] = minmod(ut[i], nu * db);
    act |= differs(d[i], ut[i]);
  }
  if (!act) return false;
  limiter_rebuild<P, T>(d[0], d[1], d[2], u + (size_t)(v * ND + 1) * ne + e, u + (size_t)(v * ND + 2) * ne + e);
  return true;
}

// fcls (float form, set when front elements exist): in the float path, skip the front elements
// (cls 1: the front kernels limit them); in the double path of a front element, read a neighbour's
// mean from `mean` (mean64) if it is at the front too, else from its updated state u (which the
// float limiter, running after the front kernels, has not yet changed).
template <int P, typename T, bool FILTER = true>
__device__ __forceinline__ void wetdry_elem(const DevMesh &m, double *u, uint8_t *wd, const Phys &ph, int *err,
                                            int do_wd, const int e);

// FILTER: decide the clear cases with float filters first (the bulk kernels); the front path,
// whose elements are rarely clear cases and whose FP64 pipe is otherwise idle, goes straight to
// the exact double tests (same results, a shorter dependency chain).
template <int P, typename T, bool FILTER = true>
__device__ __forceinline__ void limwd_body(const DevMesh &m, double *u, const T *mean, uint8_t *wd,
                                           const Phys &ph, int *err, int do_lim, int do_wd, const int e,
                                           const uint8_t *fcls = nullptr) {
  constexpr int ND = nd_of(P);
  const int ne = m.ne;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (fcls && fcls[e]) return;
  }
  if (do_lim) {
    int nb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nb[j] = m.nbr[(size_t)j * ne + e];
    const unsigned code = m.limj[e];
    T A[6];
    limiter_weights<T>(m, e, A);
    bool any = false;
#pragma unroll
    for (int v = 0; v < 3; ++v) any |= limit_variable<P, T, FILTER>(m, u, mean, e, v, nb, code, fcls, A);
    if constexpr (P == 2) {
      if (any)
        for (int v = 0; v < 3; ++v)
          for (int k = 3; k < ND; ++k) u[(size_t)(v * ND + k) * ne + e] = 0.0;
    }
  }
  if (do_wd) wetdry_elem<P, T, FILTER>(m, u, wd, ph, err, do_wd, e);
}

// The wetting/drying operator on element e (see above); do_wd 1: apply, 2: classify only.
template <int P, typename T, bool FILTER>
__device__ __forceinline__ void wetdry_elem(const DevMesh &m, double *u, uint8_t *wd, const Phys &ph, int *err,
                                            int do_wd, const int e) {
  constexpr int ND = nd_of(P);
  const int ne = m.ne;
  {  // do_wd 1: apply the operator, 2: classify only (flags from the current state)
    const bool write = do_wd == 1;
    const double h0 = ph.h0;
    const double z0 = u[e], z1 = u[(size_t)ne + e], z2 = u[2 * (size_t)ne + e];
    if constexpr (FILTER) {
      // Filtered predicate: a float evaluation decides the clearly wet elements (every vertex depth
      // exceeds h0 by far more than the float rounding of its terms), for which the double test
      // below would change nothing; only the rest are tested in double.
      const float fz0 = filter_f<T>(z0), fz1 = filter_f<T>(z1), fz2 = filter_f<T>(z2);
      float fh0, fh1, fh2;
      if constexpr (sizeof(T) == sizeof(float)) {  // the float form's copy: the same rounded values
        fh0 = m.elf[e];
        fh1 = m.elf[ne + e];
        fh2 = m.elf[2 * (size_t)ne + e];
      } else {
        fh0 = d2f(m.hbv[e]);
        fh1 = d2f(m.hbv[ne + e]);
        fh2 = d2f(m.hbv[2 * (size_t)ne + e]);
      }
      const float mag = fabsf(fz0) + fabsf(fz1) + 2.f * fabsf(fz2) + fmaxf(fabsf(fh0), fmaxf(fabsf(fh1), fabsf(fh2)));
      const float margin = 1e-6f * mag + 1e-6f;
      const float lo = fminf(fz0 - fz1 - fz2 + fh0, fminf(fz0 + fz1 - fz2 + fh1, fz0 + 2.f * fz2 + fh2));
      if (lo > ph.f.h0 + margin) {
        if (do_wd == 1 || do_wd == 2) wd[e] = 0;
        return;
      }
    }
    const double hbv[3] = {m.hbv[e], m.hbv[ne + e], m.hbv[2 * (size_t)ne + e]};
    // zeta at the reference vertices (-1,-1), (1,-1), (-1,1): psi_10 = (-1, 1, 0), psi_01 = (-1, -1, 2)
    double H[3] = {z0 - z1 - z2 + hbv[0], z0 + z1 - z2 + hbv[1], z0 + 2.0 * z2 + hbv[2]};
    const double Hs = H[0] + H[1] + H[2];  // 3 x mean depth
    int flag;
    bool changed = false;
    if (Hs <= 3.0 * (h0 + WD_TOL)) {
      const double Hm = Hs / 3.0;
      H[0] = H[1] = H[2] = Hm;
      flag = 2;
      changed = true;
    } else {
      const double hmin = fmin(H[0], fmin(H[1], H[2]));
      if (hmin < h0) {
        double ex = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (H[i] >= h0) ex += H[i] - h0;
        const double S = (Hs - 3.0 * h0) / ex;
#pragma unroll
        for (int i = 0; i < 3; ++i) H[i] = (H[i] < h0) ? h0 : h0 + (H[i] - h0) * S;
        changed = true;
      }
      flag = (H[0] > h0 + WD_TOL && H[1] > h0 + WD_TOL && H[2] > h0 + WD_TOL) ? 0 : 1;
    }
    if (changed && write) {
      const double zv0 = H[0] - hbv[0], zv1 = H[1] - hbv[1], zv2 = H[2] - hbv[2];
      u[(size_t)ne + e] = 0.5 * (zv1 - zv0);
      u[2 * (size_t)ne + e] = (2.0 * zv2 - zv0 - zv1) / 6.0;
    }
    bool zero_q = flag == 2;
    if (flag == 1) {
      double bed = -INFINITY;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (H[i] <= h0 + WD_TOL && -hbv[i] > bed) bed = -hbv[i];
      if (z0 < bed) zero_q = true;
    }
    if (zero_q && write)
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        u[(size_t)(ND + k) * ne + e] = 0.0;
        u[(size_t)(2 * ND + k) * ne + e] = 0.0;
      }
    if constexpr (P == 2) {
      if (flag != 0 && write)
        for (int v = 0; v < 3; ++v)
          for (int k = 3; k < ND; ++k) u[(size_t)(v * ND + k) * ne + e] = 0.0;
    }
    wd[e] = (uint8_t)flag;
    if (Hs < 0.0) atomicOr(err, ERR_NEGDEPTH);
  }
}

// Double limiter and wet/dry of a front element (float form): the double limiter weights, the
// front neighbours' means from mean64 and the others' from their updated states.
template <int P>
__device__ __forceinline__ void front_limwd_body(const DevMesh &m, double *u, const double *mean64,
                                                 const uint8_t *cls, uint8_t *wd, const Phys &ph, int *err,
                                                 int do_lim, int do_wd, int e) {
  DevMesh md = m;
  md.lima = m.lima_d;
  limwd_body<P, double, false>(md, u, mean64, wd, ph, err, do_lim, do_wd, e, cls);
}
// The listed front elements of one model, four lanes each: lanes 0-2 of a group limit one variable
// each (zeta, q_x, q_y), then lane 0 drops the quadratic modes of a limited element (p = 2) and
// applies the wetting/drying operator.  Group g of the list is group g / gridDim.x of block
// g % gridDim.x: a short list spreads over every SM, a few elements per busy warp.
template <int P>
__global__ void __launch_bounds__(128) k_limwd_front(const DevMesh m, double *u, const double *mean64,
                                                     const uint8_t *cls, uint8_t *wd, const Phys ph, int *err,
                                                     int do_lim, int do_wd, const int *flist,
                                                     const unsigned *fcnt) {
  constexpr int ND = nd_of(P);
  const unsigned n = *fcnt;
  const int lane = threadIdx.x & 31, sub = lane & 3;
  const unsigned gid = blockIdx.x + gridDim.x * (threadIdx.x >> 2), ng = (gridDim.x * blockDim.x) >> 2;
  DevMesh md = m;
  md.lima = m.lima_d;
  for (unsigned i0 = 0; i0 < n; i0 += ng) {  // the same trip count in every lane of a warp
    const unsigned i = i0 + gid;
    const int e = i < n ? flist[i] : -1;
    const bool own = e >= 0 && e < m.nown;
    bool acted = false;
    if (own && do_lim && sub < 3) {
      int nb[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) nb[j] = m.nbr[(size_t)j * m.ne + e];
      double A[6];
      limiter_weights<double>(md, e, A);
      acted = limit_variable<P, double, false>(md, u, mean64, e, sub, nb, m.limj[e], cls, A);
    }
    const unsigned b = __ballot_sync(0xffffffffu, acted);
    __syncwarp();  // the limited modes before the wet/dry lane reads them
    if (own && sub == 0) {
      if constexpr (P == 2) {
        if ((b >> lane) & 7u)
          for (int v = 0; v < 3; ++v)
            for (int k = 3; k < ND; ++k) u[(size_t)(v * ND + k) * m.ne + e] = 0.0;
      }
      if (do_wd) wetdry_elem<P, double, false>(md, u, wd, ph, err, do_wd, e);
    }
  }
}

// float form: held to 40 registers (6 resident 256-thread blocks per SM): the pass is bound by the
// latency of its gathers, and more resident warps measured faster despite a small spill (storm
// limiter 0.286 -> 0.241 ms per step against 56 registers)
template <int P, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 1) k_limwd(const DevMesh m, double *u, const T *mean,
                                               uint8_t *wd, const Phys ph, int *err, int do_lim,
                                               int do_wd, const uint8_t *cls) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.nown) return;  // a part limits only its own elements
  limwd_body<P, T>(m, u, mean, wd, ph, err, do_lim, do_wd, e, cls);
}

// ------------------------------------------------------------------------ ensemble
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch.  Thread 0 of each block arrives on a counter; the
// last arrival resets it and bumps the generation that the others wait on.  Every wait is bounded
// by a.timeout_ns: on expiry the block records ERR_TIMEOUT and the kernel returns instead of
// hanging.  `skip` (test hook) makes this block not arrive.  Returns false once a timeout is seen.
__device__ __forceinline__ bool grid_barrier(const EnsArgs &a, bool skip) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = a.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    bool last = false;
    if (!skip) {
      const unsigned arrived = atomicAdd(a.bar, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(a.bar, 0u);
        __threadfence();
        atomicAdd(a.bar + 1, 1u);
        last = true;
      }
    }
    if (!last) {
      const unsigned long long t0 = global_ns();
      while (*gen == g0) {
        if (global_ns() - t0 > a.timeout_ns) {
          atomicOr(a.err, ERR_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return (*(volatile int *)a.err & ERR_TIMEOUT) == 0;
}

// Buffers of stage i of s: stage 0 reads u^n (U0); intermediate stages alternate U1 / U2; the last
// stage writes u^(n+1) over U0 (each element reads only its own u^n there).
__device__ __forceinline__ void stage_buffers(int i, int s, double *U0, double *U1, double *U2, double *&in,
                                              double *&out) {
  in = i == 0 ? U0 : ((i - 1) % 2 == 0 ? U1 : U2);
  out = i == s - 1 ? U0 : (i % 2 == 0 ? U1 : U2);
}

// Stage arguments of member md (no edge scratch; the mixed form evaluates forcing inline).
template <typename T>
__device__ __forceinline__ StageArgs member_stage(const MemberDev &md, const EnsArgs &a, int stage) {
  StageArgs sa;
  double *in, *out;
  stage_buffers(stage, a.nstages, md.U0, md.U1, md.U2, in, out);
  sa.uin = in;
  sa.un = md.U0;
  sa.uout = out;
  sa.mean = md.ph.limiter ? md.mean : nullptr;
  sa.wd = md.ph.wetdry ? md.wd : nullptr;
  sa.eflux = nullptr;
  sa.emode = nullptr;
  // front list (float form with wetting/drying): flat indices tile * block + i over all members;
  // the previous stage's counter is reset in the element phase by block 0 (ens_phase)
  sa.cls = md.cls;
  sa.mean64 = md.mean64;
  sa.flist = a.flist;
  sa.fcnt = a.fcnt + stage;
  sa.fcnt_prev = nullptr;
  sa.fbase = md.etile0 * (int)blockDim.x;
  const bool inl = md.ph.hurricane && sizeof(T) == sizeof(float);
  sa.frc = (md.ph.hurricane && !inl) ? md.frc : nullptr;
  sa.frc_inline = inl ? 1 : 0;
  sa.clk = Clock{a.step, md.t0, md.dt};
  sa.tau = a.tau[stage];
  sa.ra = a.ra[stage];
  sa.rb = a.rb[stage];
  sa.rc = a.rc[stage];
  sa.rcdt = sa.rc * md.dt;
  sa.rk_form = a.form[stage];
  sa.err = a.err;
  sa.tide_t = 0.0;
  return sa;
}

// Copy a member descriptor into shared memory (all threads of the block work on one tile).
__device__ __forceinline__ void load_member(MemberDev *dst, const MemberDev *src) {
  __syncthreads();
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(MemberDev) / sizeof(int)); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// Ensemble phases 3 and 4 (float form with wetting/drying): the double update, then the double
// limiter and wet/dry, of the listed front elements of every member, one per thread.  Out of line,
// so that the float phases keep their registers.
template <int P, typename T>
__device__ __noinline__ void ens_front_phase(const EnsArgs &a, int phase, int stage, int t_begin, int t_step) {
  const unsigned n = *(volatile unsigned *)&a.fcnt[stage];
  const int B = blockDim.x;
  if (phase == 3) {  // lane groups per front element, as in k_front
    constexpr int EPW = 32 / front_lanes<P>();
    const unsigned w = (unsigned)t_begin + (unsigned)t_step * (threadIdx.x >> 5), nw = ((unsigned)t_step * B) >> 5;
    const unsigned slot = (threadIdx.x & 31) / front_lanes<P>();
    for (unsigned i0 = w * EPW; i0 < n; i0 += nw * EPW) {
      const unsigned i = i0 + slot;
      const int id = i < n ? a.flist[i] : a.flist[i0];
      const MemberDev &md = a.mem[a.etile[id / B]];
      front_update_group<P>(md.m, member_stage<T>(md, a, stage), md.ph, 0, i < n, id - md.etile0 * B);
    }
    return;
  }
  // entry i -> block i mod t_step, thread i / t_step (spread over the SMs)
  for (unsigned i = t_begin + (unsigned)t_step * threadIdx.x; i < n; i += (unsigned)t_step * B) {
    const int id = a.flist[i];
    const MemberDev &md = a.mem[a.etile[id / B]];
    const int e = id - md.etile0 * B;
    double *in, *out;
    stage_buffers(stage, a.nstages, md.U0, md.U1, md.U2, in, out);
    front_limwd_body<P>(md.m, out, md.mean64, md.cls, md.wd, md.ph, a.err, md.ph.limiter, md.ph.wetdry, e);
  }
}

// Work items of a phase: statically t_begin, t_begin + t_step, ... (one per block in the phased
// launches), or claimed dynamically from a counter (the persistent launch, where a static split
// leaves some blocks with the slow items: storm-core tiles take longer).  The counter of each
// (stage, phase) grows by n + gridDim.x per step (every block ends with one failed claim), so the
// step's claims start at base = steps done x (n + gridDim.x).
struct TileClaim {
  unsigned long long *ctr;  // null: static
  unsigned long long base;
  int *s_t;                 // shared slot for the claimed index
  int t_begin, t_step;
  __device__ __forceinline__ int first(int n) const { return ctr ? next(n) : t_begin; }
  __device__ __forceinline__ int next(int n, int t = 0) const {
    if (!ctr) return t + t_step;
    __syncthreads();  // every thread has read the previous index
    if (threadIdx.x == 0) *s_t = (int)(atomicAdd(ctr, 1ull) - base);
    __syncthreads();
    return *s_t;
  }
};

template <int P, typename T>
__device__ __forceinline__ void ens_phase(const EnsArgs &a, int phase, int stage, int t_begin, int t_step,
                                          MemberDev *sd, const T (*s_phe)[nqe_of(P)][nd_of(P)],
                                          unsigned char *smem_raw, const TileClaim *cl = nullptr) {
  const TileClaim st{nullptr, 0, nullptr, t_begin, t_step};
  const TileClaim &c = cl ? *cl : st;
  if (phase == 1) {  // element update, one shared-memory tile per work item
    if (a.any_front && blockIdx.x == 0 && threadIdx.x == 0) a.fcnt[(stage + a.nstages - 1) % a.nstages] = 0u;
    for (int t = c.first(a.n_etile); t < a.n_etile; t = c.next(a.n_etile, t)) {
      load_member(sd, &a.mem[a.etile[t]]);
      const StageArgs sa = member_stage<T>(*sd, a, stage);
      tile_body<P, T>(sd->m, sd->tl, sa, sd->ph, 0, t - sd->etile0, smem_raw, s_phe);
    }
    return;
  }
  if (phase == 3 || phase == 4) {  // the listed front elements (float form): out of line
    ens_front_phase<P, T>(a, phase, stage, t_begin, t_step);
    return;
  }
  if (phase == 0) {  // WIND at the nodes of members with a hurricane
    for (int t = c.first(a.n_ntile); t < a.n_ntile; t = c.next(a.n_ntile, t)) {
      load_member(sd, &a.mem[a.ntile[t]]);
      const int n = (t - sd->ntile0) * blockDim.x + threadIdx.x;
      if (n < sd->m.nn)
        forcing_body<T>(sd->m.nodexy, sd->m.nn, sd->ph, stage_time(Clock{a.step, sd->t0, sd->dt}, a.tau[stage], 0.0),
                        (T *)sd->frc, n);
    }
  } else {
    for (int t = c.first(a.n_etile); t < a.n_etile; t = c.next(a.n_etile, t)) {
      load_member(sd, &a.mem[a.etile[t]]);
      const int e = (t - sd->etile0) * blockDim.x + threadIdx.x;
      if (e >= sd->m.ne) continue;
      if (sd->ph.limiter || sd->ph.wetdry) {
        double *in, *out;
        stage_buffers(stage, a.nstages, sd->U0, sd->U1, sd->U2, in, out);
        limwd_body<P, T>(sd->m, out, static_cast<const T *>(sd->mean), sd->wd, sd->ph, a.err, sd->ph.limiter,
                         sd->ph.wetdry, e, sd->cls);
      }
    }
  }
}

// One time step of every member in one cooperative launch: per stage, WIND -> element update ->
// limiter/wet-dry over the flat tile lists, separated by bounded grid barriers.  The float form is
// held to 3 (p = 1) or 2 (p = 2) resident 256-thread blocks per SM: left free, the union of the
// phases takes more registers than any phase needs and only 2 blocks fit.
template <int P, typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? (P == 1 ? 5 : 2) : 1)) k_ens_persistent(const EnsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_phe[3][nqe_of(P)][nd_of(P)];
  __shared__ MemberDev sd;
  load_phe<P, T>(s_phe);
  __syncthreads();
  __shared__ int s_t;
  if (*(volatile int *)a.err & ERR_TIMEOUT) return;  // an earlier step already failed
  const bool skip = a.fault && blockIdx.x == gridDim.x - 1;
  // steps done, read by every block before the first grid barrier (block 0 bumps it after the last)
  const unsigned long long done = (unsigned long long)*(volatile long long *)a.step;
  auto claim = [&](int stage, int k, int n) {
    return TileClaim{a.work + stage * 3 + k, done * (unsigned long long)(n + gridDim.x), &s_t, 0, 0};
  };
  for (int stage = 0; stage < a.nstages; ++stage) {
    if (a.n_ntile > 0) {
      const TileClaim c0 = claim(stage, 0, a.n_ntile);
      ens_phase<P, T>(a, 0, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw, &c0);
      if (!grid_barrier(a, skip)) return;
    }
    const TileClaim c1 = claim(stage, 1, a.n_etile);
    ens_phase<P, T>(a, 1, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw, &c1);
    if (!grid_barrier(a, skip)) return;
    if (a.any_front) {  // front elements: double update, then double limiter and wet/dry
      ens_phase<P, T>(a, 3, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw);
      if (!grid_barrier(a, skip)) return;
      ens_phase<P, T>(a, 4, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw);
      if (!grid_barrier(a, skip)) return;
    }
    if (a.any_limwd) {
      const TileClaim c2 = claim(stage, 2, a.n_etile);
      ens_phase<P, T>(a, 2, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw, &c2);
      if (stage < a.nstages - 1 && !grid_barrier(a, skip)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.step += 1;
}

// The same phases as separate launches (one tile per block); the stream orders them.
template <int P, typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? (P == 1 ? 5 : 2) : 1)) k_ens_phase(const EnsArgs a, int phase, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T s_phe[3][nqe_of(P)][nd_of(P)];
  __shared__ MemberDev sd;
  load_phe<P, T>(s_phe);
  __syncthreads();
  ens_phase<P, T>(a, phase, stage, blockIdx.x, gridDim.x, &sd, s_phe, smem_raw);
}

// The limiter and wet/dry phase as its own launch (phased mode), without the element phase's
// shared memory and register needs: the float form runs 6 resident 256-thread blocks per SM, as
// the single-model limiter does (its gathers' latency wants the warps).
template <int P, typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 6 : 1)) k_ens_limwd(const EnsArgs a, int stage) {
  __shared__ MemberDev sd;
  ens_phase<P, T>(a, 2, stage, blockIdx.x, gridDim.x, &sd, nullptr, nullptr);
}

template <typename T>
cudaError_t launch_ensemble_t(int p, bool persistent, const EnsArgs &a, int block, int grid, cudaStream_t s) {
  if (persistent) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cfg.dynamicSmemBytes = p == 1 ? tile_smem_bytes<1, T>(block, a.any_inline) : tile_smem_bytes<2, T>(block, a.any_inline);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return p == 1 ? cudaLaunchKernelEx(&cfg, k_ens_persistent<1, T>, a)
                  : cudaLaunchKernelEx(&cfg, k_ens_persistent<2, T>, a);
  }
  const size_t sm = p == 1 ? tile_smem_bytes<1, T>(block, a.any_inline) : tile_smem_bytes<2, T>(block, a.any_inline);
  for (int stage = 0; stage < a.nstages; ++stage) {
    if (a.n_ntile > 0) {
      if (p == 1) k_ens_phase<1, T><<<a.n_ntile, block, sm, s>>>(a, 0, stage);
      else k_ens_phase<2, T><<<a.n_ntile, block, sm, s>>>(a, 0, stage);
    }
    if (p == 1) k_ens_phase<1, T><<<a.n_etile, block, sm, s>>>(a, 1, stage);
    else k_ens_phase<2, T><<<a.n_etile, block, sm, s>>>(a, 1, stage);
    if (a.any_front) {  // a fixed grid striding over the front list
      const int fb = std::min(a.n_etile, 304);
      for (int ph = 3; ph <= 4; ++ph) {
        if (p == 1) k_ens_phase<1, T><<<fb, block, sm, s>>>(a, ph, stage);
        else k_ens_phase<2, T><<<fb, block, sm, s>>>(a, ph, stage);
      }
    }
    if (a.any_limwd) {
      if (p == 1) k_ens_limwd<1, T><<<a.n_etile, block, 0, s>>>(a, stage);
      else k_ens_limwd<2, T><<<a.n_etile, block, 0, s>>>(a, stage);
    }
  }
  return cudaGetLastError();
}

template <typename T>
int ensemble_blocks_per_sm_t(int p, int block, bool ef) {
  int n = 0;
  if (p == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_persistent<1, T>, block, tile_smem_bytes<1, T>(block, ef));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_persistent<2, T>, block, tile_smem_bytes<2, T>(block, ef));
  return n;
}

// ------------------------------------------------------------------------ launchers
// Upload the double tables and their float rounding into this translation unit's constant memory.
static inline void upload_tables_tu(const Tab<double> td[2]) {
  Tab<float> tf[2];
  for (int p = 0; p < 2; ++p) {
    const double *src = reinterpret_cast<const double *>(&td[p]);
    float *dst = reinterpret_cast<float *>(&tf[p]);
    for (size_t i = 0; i < sizeof(Tab<double>) / sizeof(double); ++i) dst[i] = (float)src[i];
  }
  cudaMemcpyToSymbol(c_td, td, sizeof(Tab<double>) * 2);
  cudaMemcpyToSymbol(c_tf, tf, sizeof(Tab<float>) * 2);
}

inline int nblocks(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T>
void launch_forcing_t(const DevMesh &m, const Phys &ph, const Clock &clk, double tau, double tf, void *frc,
                      const LaunchCfg &c) {
  k_forcing<T><<<nblocks(m.nn, 256), 256, 0, c.stream>>>(m.nodexy, m.nn, ph, clk, tau, tf, (T *)frc);
}

template <typename T>
void launch_edge_t(int p, const DevMesh &m, const StageArgs &s, const Phys &ph, const LaunchCfg &c) {
  if (m.nint == 0) return;
  if (p == 1)
    k_edge<1, T><<<nblocks(m.nint, c.block), c.block, 0, c.stream>>>(m, s, ph);
  else
    k_edge<2, T><<<nblocks(m.nint, c.block), c.block, 0, c.stream>>>(m, s, ph);
}

template <typename T>
void launch_element_t(int p, bool split, bool write_rhs, const DevMesh &m, const StageArgs &s, const Phys &ph,
                      const LaunchCfg &c) {
  const int nb = nblocks(m.nact, c.block), wr = write_rhs ? 1 : 0;
  if (p == 1) {
    if (split)
      k_element<1, T, true><<<nb, c.block, 0, c.stream>>>(m, s, ph, wr);
    else
      k_element<1, T, false><<<nb, c.block, 0, c.stream>>>(m, s, ph, wr);
  } else {
    if (split)
      k_element<2, T, true><<<nb, c.block, 0, c.stream>>>(m, s, ph, wr);
    else
      k_element<2, T, false><<<nb, c.block, 0, c.stream>>>(m, s, ph, wr);
  }
}

template <typename T>
void launch_tile_t(int p, bool wide, bool write_rhs, const DevMesh &m, const DevTiles &tl, const StageArgs &s,
                   const Phys &ph, const LaunchCfg &c) {
  const int wr = write_rhs ? 1 : 0;
  if (p == 1) {
    const size_t sm = tile_smem_bytes<1, T>(tl.tile, s.frc_inline != 0);
    if constexpr (sizeof(T) == sizeof(float)) {
      if (wide) {
        k_tile<1, T, true><<<tl.ntiles, tl.tile, sm, c.stream>>>(m, tl, s, ph, wr);
        return;
      }
    }
    k_tile<1, T, false><<<tl.ntiles, tl.tile, sm, c.stream>>>(m, tl, s, ph, wr);
  } else {
    const size_t sm = tile_smem_bytes<2, T>(tl.tile, s.frc_inline != 0);
    k_tile<2, T, false><<<tl.ntiles, tl.tile, sm, c.stream>>>(m, tl, s, ph, wr);
  }
}

template <typename T>
void prepare_tile_t() {
  // allow the largest tile's dynamic shared memory (p = 2, 256 elements)
  cudaFuncSetAttribute(k_tile<1, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes<1, T>(256, true));
  if constexpr (sizeof(T) == sizeof(float))
    cudaFuncSetAttribute(k_tile<1, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_smem_bytes<1, T>(256, true));
  cudaFuncSetAttribute(k_tile<2, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes<2, T>(256, true));
  cudaFuncSetAttribute(k_ens_persistent<1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tile_smem_bytes<1, T>(256, true));
  cudaFuncSetAttribute(k_ens_persistent<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tile_smem_bytes<2, T>(256, true));
  cudaFuncSetAttribute(k_ens_phase<1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes<1, T>(256, true));
  cudaFuncSetAttribute(k_ens_phase<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem_bytes<2, T>(256, true));
}

// Element means of u into the limiter's mean array, rounded to T as the element kernels round them.
template <typename T>
__global__ void k_copy_means(int nd, int ne, const double *u, T *mean) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  for (int v = 0; v < 3; ++v) mean[(size_t)v * ne + e] = from_d<T>(u[(size_t)v * nd * ne + e]);
}
template <typename T>
void launch_copy_means_t(int p, int ne, const double *u, void *mean, cudaStream_t s) {
  k_copy_means<T><<<nblocks(ne, 256), 256, 0, s>>>(nd_of(p), ne, u, static_cast<T *>(mean));
}

template <typename T>
void launch_limwd_t(int p, bool do_lim, int do_wd, const DevMesh &m, double *u, const void *mean_v, uint8_t *wd,
                    const Phys &ph, int *err, const LaunchCfg &c, const uint8_t *cls) {
  const T *mean = static_cast<const T *>(mean_v);
  const int nb = nblocks(m.nown, c.block);
  if (p == 1)
    k_limwd<1, T><<<nb, c.block, 0, c.stream>>>(m, u, mean, wd, ph, err, do_lim, do_wd, cls);
  else
    k_limwd<2, T><<<nb, c.block, 0, c.stream>>>(m, u, mean, wd, ph, err, do_lim, do_wd, cls);
}

// The front kernels: a fixed grid (captured in the step graph; the list length is read on the
// device) of one 32-thread block per SM, striding over the list.
inline int front_blocks() {
  static int n = 0;
  if (!n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n = sms > 0 ? sms : 152;
  }
  return n;
}
inline void launch_front_t(int p, const DevMesh &m, const StageArgs &s, const Phys &ph, int write_rhs,
                           cudaStream_t st) {
  // 8 blocks of 4 warps per SM; the busy warps (32 / LPE list entries each) go one per block first
  if (p == 1)
    k_front<1><<<8 * front_blocks(), 128, 0, st>>>(m, s, ph, write_rhs);
  else
    k_front<2><<<8 * front_blocks(), 128, 0, st>>>(m, s, ph, write_rhs);
}
inline void launch_limwd_front_t(int p, bool do_lim, int do_wd, const DevMesh &m, double *u, const double *mean64,
                                 const uint8_t *cls, uint8_t *wd, const Phys &ph, int *err, const int *flist,
                                 const unsigned *fcnt, cudaStream_t st) {
  // 2 blocks of 32 four-lane groups per SM; the list's groups go one per block first
  if (p == 1)
    k_limwd_front<1><<<2 * front_blocks(), 128, 0, st>>>(m, u, mean64, cls, wd, ph, err, do_lim, do_wd, flist, fcnt);
  else
    k_limwd_front<2><<<2 * front_blocks(), 128, 0, st>>>(m, u, mean64, cls, wd, ph, err, do_lim, do_wd, flist, fcnt);
}

}  // namespace dg
