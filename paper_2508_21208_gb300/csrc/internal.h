// internal.h -- data structures shared by the host preprocessor, the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgswem.h"

namespace dg {

constexpr int MAXD = 6;   // modes per variable at p <= 2
constexpr int MAXQA = 12; // area quadrature points at p <= 2
constexpr int MAXQE = 4;  // edge quadrature points at p <= 2

__host__ __device__ constexpr int nd_of(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ constexpr int nqa_of(int p) { return p == 1 ? 6 : 12; }
__host__ __device__ constexpr int nqe_of(int p) { return p == 1 ? 2 : 4; }

// Per-element geometry rows (structure of arrays, one row of n_elems values each).
// J^{-1} = [[rx, ry], [sx, sy]] (d(xi,eta)/d(x,y)), det J = |Omega_e|/2, and for local edge l
// (vertex (l+1)%3 -> (l+2)%3) the outward unit normal (nx_l, ny_l) and half length hl_l.
enum {
  GEO_RX, GEO_RY, GEO_SX, GEO_SY, GEO_DETJ,
  GEO_NX0, GEO_NX1, GEO_NX2, GEO_NY0, GEO_NY1, GEO_NY2, GEO_HL0, GEO_HL1, GEO_HL2,
  NGEO
};

constexpr int NBR_LAND = -1;
constexpr int NBR_OPEN = -2;
constexpr int NBR_RIVER = -3;

// Mesh after preprocessing, elements in internal (locality) order.
struct HostMesh {
  int ne = 0, nn = 0, nint = 0, nbnd = 0;
  // part of a partitioned domain (Sec. 5.3): elements [0, nown) are this part's own, [nown, nact)
  // the first ghost layer (updated here too, redundantly), [nact, ne) the second ghost layer (read
  // only); without a partition nown = nact = ne
  int nown = 0, nact = 0;
  std::vector<int> perm;          // internal index -> caller index
  std::vector<int> iperm;         // caller index -> internal index
  std::vector<int> vnode;         // [3][ne] node ids
  std::vector<double> geo;        // [NGEO][ne]
  std::vector<double> hbv;        // [3][ne] vertex h_b
  std::vector<double> area;       // [ne]
  std::vector<double> inradius;   // [ne]
  std::vector<int> nbr;           // [3][ne] neighbour (internal id) or NBR_LAND / NBR_OPEN
  std::vector<uint8_t> nle;       // [ne] neighbour's local edge index, 2 bits per local edge
  std::vector<int> eledge;        // [3][ne] interior edge id, bit 31 = this element is the minus side; -1
  std::vector<double> lima;       // [3][2][ne] limiter weights
  std::vector<uint16_t> limj;     // [ne] limiter neighbour pairs, 4 bits per local edge (15 = none)
  std::vector<int> edel;          // [2][nint] (plus, minus) elements
  std::vector<uint8_t> edle;      // [nint] l+ | l- << 2
  std::vector<double> edgeo;      // [3][nint] nx, ny, half length (normal out of the plus side)
  std::vector<double> edhb;       // [2][nint] h_b at the edge's end nodes (plus side's order)
  std::vector<double> nodexy;     // [2][nn]
};

// Edges touching each tile of `tile` consecutive (internal-order) elements, for the tiled
// element kernel: an interior edge whose two elements lie in one tile is listed once there; an
// edge between two tiles is listed in both; a boundary edge in its element's tile.  Side A is the
// edge's plus side (the normal points out of A); B is the minus element or NBR_LAND / NBR_OPEN.
struct TileEdges {
  int tile = 0, ntiles = 0, n = 0;
  std::vector<int> start;     // [ntiles + 1]
  std::vector<int> ea, eb;    // [n] elements (or boundary code in eb)
  std::vector<uint8_t> code;  // [n] lA | lB << 2 | (A in tile) << 4 | (B in tile) << 5
  std::vector<double> geo;    // [3][n] nx, ny, half length
  std::vector<double> hb;     // [2][n] h_b at the edge's end nodes (A's counter-clockwise order)
};
void build_tile_edges(const HostMesh &H, int tile, TileEdges &out);
inline int max_tile_edges(const HostMesh &H) { return 2 * H.nint + H.nbnd; }

// Returns 0 or DGSWEM_EMESH / DGSWEM_EINVAL with a message.  elem_class (optional, caller order):
// 0 own, 1 first ghost layer, 2 second ghost layer; the internal order then puts the classes in
// that order (Hilbert order within each).
int preprocess_mesh(const dgswem_mesh &m, const double *bathy, bool hilbert, HostMesh &out,
                    std::string &msg, const int32_t *elem_class = nullptr);

// ------------------------------------------------------------------ device-side views
// Float copies of the constants the float form uses, rounded once on the host (a double -> float
// conversion in a kernel runs on GB300's FP64 pipe).
struct PhysF {
  float g, sqrt_g, h0, cf, gn2, fcor, rain, river_q;
  float dp, tx, ty;  // pn - pc; half the translation velocity (x, y)
  float rmax, hB, flat, hB_rho_air, rho_ratio, inv_rho_w;
};

struct Phys {
  double g, sqrt_g, h0, cf, gn2, fcor;
  double tide_amp, tide_omega, tide_phase;
  double pc, pn, rmax, hB, vt, x0, y0, heading, flat, rho_air, rho_w;
  double cos_h, sin_h;     // heading direction of the storm track
  double hB_rho_air, rho_ratio, inv_rho_w;  // B / rho_air, rho_air / rho_w, 1 / rho_w
  int friction, wetdry, limiter, hurricane, flux;
  int holland15;           // B = 1.5: (Rmax/r)^B = s sqrt(s)
  double rain, river_q;
  PhysF f;
};

// The stage update's form, chosen on the host from (a, b, c): 0 u_in + c dt L; 1 the exact average
// (u^n + u_in + dt L) / 2; 2 the general a u^n + b u_in + c dt L.
inline int rk_form_of(double a, double b, double c) {
  if (a == 0.0 && b == 1.0) return 0;
  if (a == 0.5 && b == 0.5 && c == 0.5) return 1;
  return 2;
}

struct DevMesh {
  int ne, nn, nint;
  int nown, nact;          // partitioned domain: own / updated element counts (HostMesh); else ne
  const void *geo;         // T [NGEO][ne]
  const double *hbv;       // [3][ne]
  const double *area;      // [ne]
  const double *inradius;  // [ne]
  const int *nbr;          // [3][ne]
  const uint8_t *nle;      // [ne]
  const int *vnode;        // [3][ne]
  const void *lima;        // T [6][ne]
  const uint16_t *limj;    // [ne]
  const int *eledge;       // [3][ne]
  const int *edel;         // [2][nint]
  const uint8_t *edle;     // [nint]
  const void *edgeo;       // T [3][nint]
  const double *edhb;      // [2][nint]
  const void *hbq;         // T [NQA][ne]: h_b at the area quadrature points
  const void *edhbq;       // T [NQE][nint]: h_b at the interior edges' Gauss points
  const double *nodexy;    // [2][nn]
  const float *elf;        // float form: [9][ne] vertex h_b (3), vertex x (3), vertex y (3), rounded
                           // once on the host like the kernels' double -> float conversion
  // float form only: double copies of geo ([NGEO][ne]), lima ([6][ne]) and hbq ([NQA][ne]) for
  // the elements at the wetting/drying front, whose update runs in double (null in the FP64 form)
  const double *geo_d, *lima_d, *hbq_d;
};


struct Clock {
  const long long *step;   // device counter of completed steps
  double t0, dt;           // stage time = t0 + (step + tau) * dt
};

constexpr int MAX_STAGES = 8;
// Two-register Shu-Osher stage table: u_i = a_i u^n + b_i u_(i-1) + c_i dt L(u_(i-1)); stage i
// evaluates L at tau_(i-1).  Returns the stage count (0 if the parameters name no valid scheme).
int rk_stage_table(const dgswem_params &p, double a[MAX_STAGES], double b[MAX_STAGES], double c[MAX_STAGES],
                   double tau[MAX_STAGES]);

struct StageArgs {
  const double *uin;       // u^(s): [3][ND][ne]
  const double *un;        // u^n (second stage only)
  double *uout;            // u^(s+1)
  void *mean;              // T [3][ne] element means of u^(s+1), read by the limiter
  const uint8_t *wd;       // wet/dry flags
  void *eflux;             // T [3][NQE][nint] weighted interior-edge fluxes (split variant)
  uint8_t *emode;          // [nint] 1 = the edge flux in eflux applies, 0 = both sides see a wall
  const void *frc;         // T [3][nn] nodal forcing at the stage time, or nullptr
  int frc_inline;          // 1: evaluate the forcing at the element's vertices (mixed form)
  Clock clk;
  double tau;              // stage time = clk.t0 + (step + tau) * clk.dt
  double ra, rb, rc;       // u_out = ra u^n + rb u_in + rc dt L(u_in)
  double rcdt;             // rc * dt
  int rk_form;             // rk_form_of(ra, rb, rc)
  int *err;
  double tide_t;           // stage time when clk.step is null (single operator calls)
  // Float form with wetting/drying (null otherwise): the element kernels mark each element at the
  // wetting/drying front with cls[e] = 1 (0 elsewhere), skip it, and append its flat index
  // fbase + e to flist, counting in *fcnt; the front kernels then update the listed elements in
  // double and write their means in double to mean64.  *fcnt_prev, the previous stage's counter,
  // is reset by the element kernels (its readers have finished).
  uint8_t *cls;
  double *mean64;
  int *flist;
  unsigned *fcnt, *fcnt_prev;
  int fbase;
};

struct DevTiles {
  int tile, ntiles;
  const int *start;        // [ntiles + 1]
  const int *ea, *eb;      // [n]
  const uint8_t *code;     // [n]
  const void *geo;         // T [3][n]
  const double *hb;        // [2][n]
  const void *hbq;         // T [NQE][n]: h_b at the Gauss points
  int n;
};

// One ensemble member (scenario) as the ensemble kernels see it.
struct MemberDev {
  DevMesh m;               // the member's mesh statics (shared with members on the same mesh)
  DevTiles tl;             // the mesh's tile edge lists for the ensemble's tile size
  Phys ph;
  double *U0, *U1, *U2;    // its own state (U2 only for three or more stages)
  void *mean;              // T [3][ne] element means for the limiter
  uint8_t *wd;
  void *frc;               // T [3][nn]
  uint8_t *cls;            // float form with wetting/drying: front class per element (StageArgs)
  double *mean64;          // float form with wetting/drying: the front elements' means in double
  double t0, dt;           // stage time = t0 + (step + stage) * dt (its own dt)
  int etile0, ntile0;      // first element / node tile of this member in the flat tile lists
};

struct EnsArgs {
  int nstages;
  double ra[MAX_STAGES], rb[MAX_STAGES], rc[MAX_STAGES], tau[MAX_STAGES];
  int form[MAX_STAGES];    // rk_form_of per stage
  const MemberDev *mem;
  const int *etile;        // element tile -> member
  const int *ntile;        // node tile -> member (members with a hurricane)
  int n_etile, n_ntile;
  long long *step;         // shared step counter
  unsigned *bar;           // grid barrier: [0] arrivals, [1] generation
  int *err;
  int fault;               // test hook: the last block never arrives at a barrier
  int any_limwd;
  int any_inline;          // some member evaluates the vortex inline (float form): tile_smem_bytes(, true)
  int any_front;           // some member has front elements to list (float form with wetting/drying)
  int *flist;              // the front list of every member (flat element indices: tile * block + i)
  unsigned *fcnt;          // its counter per stage
  unsigned long long *work;  // persistent launch: work-item claim counters, [stage][phase 0, 1, 2]
  unsigned long long timeout_ns;
};

// error word bits
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_NEGDEPTH = 2;
constexpr int ERR_TIMEOUT = 4;

// reference tables (product-side restatement of the basis and quadrature)
template <typename T>
struct Tab {
  T wq[MAXQA];             // area weights on the reference triangle (area 2)
  T iwq[MAXQA];            // their inverses
  T phq[MAXQA][MAXD];      // basis at area points
  T dxq[MAXQA][MAXD];      // d basis / d xi
  T dyq[MAXQA][MAXD];      // d basis / d eta
  T nq[MAXQA][3];          // linear vertex shape functions at area points
  T we[MAXQE];             // edge weights on [-1, 1]
  T se[MAXQE];             // edge points on [-1, 1] (ascending, mirror symmetric)
  T phe[3][MAXQE][MAXD];   // basis on local edge l at its own parameter s_g
  T nrm[MAXD];             // squared reference norms
  T inrm[MAXD];            // their inverses
  T phm[3][3];             // linear modes at the three edge midpoints
  T phv[3][MAXD];          // basis at the three vertices
  T lim_idet;              // 1 / (phm[0][1] phm[1][2] - phm[0][2] phm[1][1]): linear modes from midpoints 0, 1
};

void build_tables(int p, Tab<double> &t);
// h_b at the area quadrature points of every element ([NQA][ne]) and at the Gauss points of n
// edges from their end values hA, hB ([NQE][n]), with the reference tables of degree p.  Computed
// once on the host (in the FP64 form, an interpolation per point and stage costs more FP64 issue
// than reading the value).
void area_point_hb(int p, const HostMesh &H, std::vector<double> &out);
void edge_point_hb(int p, const double *hA, const double *hB, int n, std::vector<double> &out);

// launchers (kernels_f64.cu: T = double; kernels_f32.cu: T = float)
struct LaunchCfg {
  int block;
  cudaStream_t stream;
};
#define DG_DECLARE_LAUNCHERS(SUF)                                                                 \
  void upload_tables_##SUF(const Tab<double> td[2]);                                             \
  void launch_forcing_##SUF(const DevMesh &m, const Phys &ph, const Clock &clk, double tau,      \
                            double t_fixed, void *frc, const LaunchCfg &c);                      \
  void launch_edge_##SUF(int p, const DevMesh &m, const StageArgs &s, const Phys &ph,            \
                         const LaunchCfg &c);                                                    \
  void launch_element_##SUF(int p, bool split, bool write_rhs, const DevMesh &m,                 \
                            const StageArgs &s, const Phys &ph, const LaunchCfg &c);             \
  void launch_limwd_##SUF(int p, bool do_lim, int do_wd, const DevMesh &m, double *u,            \
                          const void *mean, uint8_t *wd, const Phys &ph, int *err,               \
                          const LaunchCfg &c, const uint8_t *cls);                              \
  void launch_tile_##SUF(int p, bool wide, bool write_rhs, const DevMesh &m, const DevTiles &tl,   \
                         const StageArgs &s, const Phys &ph, const LaunchCfg &c);                 \
  void prepare_tile_##SUF();                                                                      \
  cudaError_t launch_ensemble_##SUF(int p, bool persistent, const EnsArgs &a, int block, int grid, \
                                    cudaStream_t s);                                             \
  int ensemble_blocks_per_sm_##SUF(int p, int block, bool ef);                                  \
  void launch_copy_means_##SUF(int p, int ne, const double *u, void *mean, cudaStream_t s);
DG_DECLARE_LAUNCHERS(f64)
DG_DECLARE_LAUNCHERS(f32)
#undef DG_DECLARE_LAUNCHERS

inline void launch_forcing(bool mixed, const DevMesh &m, const Phys &ph, const Clock &clk, double tau,
                           double t_fixed, void *frc, const LaunchCfg &c) {
  mixed ? launch_forcing_f32(m, ph, clk, tau, t_fixed, frc, c)
        : launch_forcing_f64(m, ph, clk, tau, t_fixed, frc, c);
}
inline void launch_edge(bool mixed, int p, const DevMesh &m, const StageArgs &s, const Phys &ph,
                        const LaunchCfg &c) {
  mixed ? launch_edge_f32(p, m, s, ph, c) : launch_edge_f64(p, m, s, ph, c);
}
inline void launch_element(bool mixed, int p, bool split, bool write_rhs, const DevMesh &m,
                           const StageArgs &s, const Phys &ph, const LaunchCfg &c) {
  mixed ? launch_element_f32(p, split, write_rhs, m, s, ph, c)
        : launch_element_f64(p, split, write_rhs, m, s, ph, c);
}
// cls (float form only): elements with cls[e] = 1 are skipped (the front kernels handle them);
// null: every element.
inline void launch_limwd(bool mixed, int p, bool do_lim, int do_wd, const DevMesh &m, double *u,
                         const void *mean, uint8_t *wd, const Phys &ph, int *err,
                         const LaunchCfg &c, const uint8_t *cls = nullptr) {
  mixed ? launch_limwd_f32(p, do_lim, do_wd, m, u, mean, wd, ph, err, c, cls)
        : launch_limwd_f64(p, do_lim, do_wd, m, u, mean, wd, ph, err, c, nullptr);
}
// Float form with wetting/drying: the double update of the listed front elements (s.flist,
// *s.fcnt), then their double limiter and wet/dry.  kernels_f32.cu.
void launch_front(int p, const DevMesh &m, const StageArgs &s, const Phys &ph, int write_rhs, cudaStream_t st);
void launch_limwd_front(int p, bool do_lim, int do_wd, const DevMesh &m, double *u, const double *mean64,
                        const uint8_t *cls, uint8_t *wd, const Phys &ph, int *err, const int *flist,
                        const unsigned *fcnt, cudaStream_t st);
inline void launch_tile(bool mixed, int p, bool wide, bool write_rhs, const DevMesh &m, const DevTiles &tl,
                        const StageArgs &s, const Phys &ph, const LaunchCfg &c) {
  mixed ? launch_tile_f32(p, wide, write_rhs, m, tl, s, ph, c) : launch_tile_f64(p, wide, write_rhs, m, tl, s, ph, c);
}
inline cudaError_t launch_ensemble(bool mixed, int p, bool persistent, const EnsArgs &a, int block, int grid,
                                   cudaStream_t s) {
  return mixed ? launch_ensemble_f32(p, persistent, a, block, grid, s)
               : launch_ensemble_f64(p, persistent, a, block, grid, s);
}
// element means of u into the limiter's mean array (T [3][ne])
inline void launch_copy_means(bool mixed, int p, int ne, const double *u, void *mean, cudaStream_t s) {
  mixed ? launch_copy_means_f32(p, ne, u, mean, s) : launch_copy_means_f64(p, ne, u, mean, s);
}
inline int ensemble_blocks_per_sm(bool mixed, int p, int block, bool ef) {
  return mixed ? ensemble_blocks_per_sm_f32(p, block, ef) : ensemble_blocks_per_sm_f64(p, block, ef);
}
void upload_common_tables(const Tab<double> td[2]);

// precision-independent kernels (common_kernels.cu)
void launch_init_nodal(int p, const DevMesh &m, const double *nodal, double *u, cudaStream_t s);
void launch_dt(int p, const DevMesh &m, const double *u, const Phys &ph, unsigned long long *best,
               cudaStream_t s);
void launch_mass(int p, const DevMesh &m, const double *u, double *partial, double *result,
                 cudaStream_t s);
void launch_permute(const double *src, double *dst, const int *map, int rows, int ne,
                    cudaStream_t s);
void launch_permute_u8(const uint8_t *src, uint8_t *dst, const int *map, int ne, cudaStream_t s);
void launch_advance(long long *step, cudaStream_t s);
// pack / unpack the halo records (state rows and wet/dry flag) of the elements idx[0..n)
void launch_halo_pack(int nd, int ne, const double *u, const uint8_t *wd, const int *idx, int n, double *buf,
                      cudaStream_t s);
void launch_halo_unpack(int nd, int ne, double *u, uint8_t *wd, const int *idx, int n, const double *buf,
                        cudaStream_t s);
int mass_partial_count(int ne);

}  // namespace dg
