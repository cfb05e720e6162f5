// api.cu -- the C ABI declared in include/dgswem.h: context life cycle, workspace layout,
// uploads, the captured step graph, state I/O, single-operator entry points and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace dg;

namespace {
constexpr size_t kAlign = 256;
}  // namespace

// ------------------------------------------------------------------ helpers shared with ensemble.cu
int ctx_fail(dgswem_ctx *c, int code, const std::string &msg) {
  if (c && c->sticky == 0) {
    c->sticky = code;
    c->errmsg = msg;
  }
  return code;
}

// A query the context's current mode cannot answer: reported, but not sticky.
static int ctx_refuse(dgswem_ctx *c, int code, const std::string &msg) {
  if (c && c->sticky == 0) c->errmsg = msg;
  return code;
}

int ctx_cuda(dgswem_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return 0;
  return ctx_fail(c, DGSWEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_params(const dgswem_params *p, std::string &msg) {
  if (!p) { msg = "params: null"; return DGSWEM_EINVAL; }
  if (p->p != 1 && p->p != 2) { msg = "params: p must be 1 or 2"; return DGSWEM_EINVAL; }
  if (p->precision != DGSWEM_FP64 && p->precision != DGSWEM_FP32_MIXED) {
    msg = "params: unknown precision"; return DGSWEM_EINVAL;
  }
  if (!(p->g > 0) || !std::isfinite(p->g)) { msg = "params: g must be positive"; return DGSWEM_EINVAL; }
  {
    const double f[] = {p->g, p->cfl, p->dt, p->h0, p->manning_n, p->cf, p->coriolis_lat_deg, p->tide_amp,
                        p->tide_period, p->tide_phase, p->pc_hpa, p->pn_hpa, p->rmax_m, p->holland_b, p->vt_ms,
                        p->track_x0, p->track_y0, p->track_heading, p->rho_air, p->rho_water, p->rain_rate,
                        p->river_q};
    for (double x : f)
      if (!std::isfinite(x)) { msg = "params: non-finite value"; return DGSWEM_EINVAL; }
  }
  if (p->dt < 0) { msg = "params: dt must be >= 0 (0: from cfl)"; return DGSWEM_EINVAL; }
  if (!(p->dt > 0) && !(p->cfl > 0)) { msg = "params: need dt > 0 or cfl > 0"; return DGSWEM_EINVAL; }
  if (p->h0 < 0 || !std::isfinite(p->h0)) { msg = "params: h0 must be >= 0"; return DGSWEM_EINVAL; }
  if (p->friction < 0 || p->friction > 2) { msg = "params: unknown friction law"; return DGSWEM_EINVAL; }
  if (p->friction == DGSWEM_FRICTION_QUADRATIC && !(p->cf >= 0)) { msg = "params: cf < 0"; return DGSWEM_EINVAL; }
  if (p->friction == DGSWEM_FRICTION_MANNING && !(p->manning_n >= 0)) { msg = "params: manning_n < 0"; return DGSWEM_EINVAL; }
  if (p->tide_amp != 0.0 && !(p->tide_period > 0)) { msg = "params: tide_period must be > 0"; return DGSWEM_EINVAL; }
  if (p->hurricane) {
    if (!(p->rho_air > 0) || !(p->rho_water > 0) || !(p->rmax_m > 0) || !(p->holland_b > 0)) {
      msg = "params: hurricane needs rho_air, rho_water, rmax_m, holland_b > 0"; return DGSWEM_EINVAL;
    }
  }
  if (p->flux != DGSWEM_FLUX_LLF && p->flux != DGSWEM_FLUX_ROE) { msg = "params: unknown numerical flux"; return DGSWEM_EINVAL; }
  if (!std::isfinite(p->rain_rate) || !std::isfinite(p->river_q)) { msg = "params: non-finite rain or river rate"; return DGSWEM_EINVAL; }
  double a[MAX_STAGES], b[MAX_STAGES], c[MAX_STAGES], tau[MAX_STAGES];
  if (rk_stage_table(*p, a, b, c, tau) < 2) { msg = "params: unknown Runge-Kutta scheme or bad table"; return DGSWEM_EINVAL; }
  return 0;
}

Phys make_phys(const dgswem_params &p) {
  Phys ph{};
  ph.g = p.g;
  ph.sqrt_g = std::sqrt(p.g);
  ph.h0 = p.h0;
  ph.cf = p.cf;
  ph.gn2 = p.g * p.manning_n * p.manning_n;
  const double omega = 7.2921e-5, deg = 3.14159265358979323846 / 180.0;
  ph.flat = 2.0 * omega * std::sin(p.coriolis_lat_deg * deg);
  ph.fcor = p.coriolis ? ph.flat : 0.0;
  ph.tide_amp = p.tide_amp;
  ph.tide_omega = p.tide_period > 0 ? 2.0 * 3.14159265358979323846 / p.tide_period : 0.0;
  ph.tide_phase = p.tide_phase;
  ph.pc = 100.0 * p.pc_hpa;
  ph.pn = 100.0 * p.pn_hpa;
  ph.rmax = p.rmax_m;
  ph.hB = p.holland_b;
  ph.vt = p.vt_ms;
  ph.x0 = p.track_x0;
  ph.y0 = p.track_y0;
  ph.heading = p.track_heading;
  ph.cos_h = std::cos(p.track_heading);
  ph.sin_h = std::sin(p.track_heading);
  ph.hB_rho_air = p.rho_air > 0 ? p.holland_b / p.rho_air : 0.0;
  ph.rho_ratio = p.rho_water > 0 ? p.rho_air / p.rho_water : 0.0;
  ph.inv_rho_w = p.rho_water > 0 ? 1.0 / p.rho_water : 0.0;
  ph.rho_air = p.rho_air;
  ph.rho_w = p.rho_water;
  ph.friction = p.friction;
  ph.wetdry = p.h0 > 0.0 ? 1 : 0;
  ph.limiter = p.limiter ? 1 : 0;
  ph.hurricane = p.hurricane ? 1 : 0;
  ph.flux = p.flux;
  ph.holland15 = p.holland_b == 1.5 ? 1 : 0;
  ph.rain = p.rain_rate;
  ph.river_q = p.river_q;
  PhysF &f = ph.f;
  f.g = (float)ph.g;
  f.sqrt_g = (float)ph.sqrt_g;
  f.h0 = (float)ph.h0;
  f.cf = (float)ph.cf;
  f.gn2 = (float)ph.gn2;
  f.fcor = (float)ph.fcor;
  f.rain = (float)ph.rain;
  f.river_q = (float)ph.river_q;
  f.dp = (float)(ph.pn - ph.pc);
  f.tx = 0.5f * (float)(ph.vt * ph.cos_h);
  f.ty = 0.5f * (float)(ph.vt * ph.sin_h);
  f.rmax = (float)ph.rmax;
  f.hB = (float)ph.hB;
  f.flat = (float)ph.flat;
  f.hB_rho_air = (float)ph.hB_rho_air;
  f.rho_ratio = (float)ph.rho_ratio;
  f.inv_rho_w = (float)ph.inv_rho_w;
  return ph;
}

void upload_all_tables() {
  Tab<double> td[2];
  build_tables(1, td[0]);
  build_tables(2, td[1]);
  upload_tables_f64(td);
  upload_tables_f32(td);
  upload_common_tables(td);
  prepare_tile_f64();
  prepare_tile_f32();
}

// Convert a double vector to the arithmetic type of the form (float for the mixed form).
static std::vector<char> typed(const std::vector<double> &v, bool mixed) {
  std::vector<char> out(v.size() * (mixed ? sizeof(float) : sizeof(double)));
  if (mixed) {
    float *f = reinterpret_cast<float *>(out.data());
    for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
  } else {
    std::memcpy(out.data(), v.data(), v.size() * sizeof(double));
  }
  return out;
}

// double -> float as the kernels convert (round to nearest even; magnitudes below float's normal
// range give a signed zero), so that a value rounded here equals the one a kernel would compute.
static float device_float(double x) {
  if (std::fabs(x) < (double)FLT_MIN) return std::signbit(x) ? -0.0f : 0.0f;
  return (float)x;
}

// The float form's per-element vertex data: h_b, x and y at the three vertices ([9][ne]).
static std::vector<char> element_floats(const HostMesh &H) {
  const size_t ne = H.ne, nn = H.nn;
  std::vector<char> out(9 * ne * sizeof(float));
  float *f = reinterpret_cast<float *>(out.data());
  for (size_t e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) {
      const size_t n = (size_t)H.vnode[a * ne + e];
      f[a * ne + e] = device_float(H.hbv[a * ne + e]);
      f[(3 + a) * ne + e] = device_float(H.nodexy[n]);
      f[(6 + a) * ne + e] = device_float(H.nodexy[nn + n]);
    }
  return out;
}

// ------------------------------------------------------------------ workspace layout
void carve_mesh(Carver &k, const HostMesh &H, int p, bool mixed, DevMesh &m, int **perm, int **iperm) {
  const int ne = H.ne, nn = H.nn, nint = H.nint;
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  m.ne = ne;
  m.nn = nn;
  m.nown = H.nown;
  m.nact = H.nact;
  m.nint = nint;
  m.geo = k.take<char>(tsz * NGEO * ne);
  m.hbv = k.take<double>(3 * (size_t)ne);
  m.area = k.take<double>(ne);
  m.inradius = k.take<double>(ne);
  m.nbr = k.take<int>(3 * (size_t)ne);
  m.nle = k.take<uint8_t>(ne);
  m.vnode = k.take<int>(3 * (size_t)ne);
  m.lima = k.take<char>(tsz * 6 * ne);
  m.limj = k.take<uint16_t>(ne);
  m.eledge = k.take<int>(3 * (size_t)ne);
  m.edel = k.take<int>(2 * (size_t)nint);
  m.edle = k.take<uint8_t>(nint);
  m.edgeo = k.take<char>(tsz * 3 * nint);
  m.edhb = k.take<double>(2 * (size_t)nint);
  // h_b at quadrature points: the area points for the FP64 form, the edge Gauss points for both
  m.hbq = mixed ? nullptr : k.take<char>(tsz * nqa_of(p) * ne);
  m.edhbq = k.take<char>(tsz * nqe_of(p) * nint);
  m.nodexy = k.take<double>(2 * (size_t)nn);
  m.elf = mixed ? k.take<float>(9 * (size_t)ne) : nullptr;
  // the float form's double statics for the elements at the wetting/drying front
  m.geo_d = mixed ? k.take<double>(NGEO * (size_t)ne) : nullptr;
  m.lima_d = mixed ? k.take<double>(6 * (size_t)ne) : nullptr;
  m.hbq_d = mixed ? k.take<double>((size_t)nqa_of(p) * ne) : nullptr;
  *perm = k.take<int>(ne);
  *iperm = k.take<int>(ne);
}

static void layout(dgswem_ctx *c, char *base, size_t *bytes) {
  const HostMesh &H = c->hm;
  const int ne = H.ne, nn = H.nn, nint = H.nint, ND = c->ND, NQE = nqe_of(c->P);
  const size_t tsz = c->mixed ? sizeof(float) : sizeof(double);
  Carver k{base};
  carve_mesh(k, H, c->P, c->mixed, c->dm, &c->d_perm, &c->d_iperm);
  const size_t nu = 3 * (size_t)ND * ne;
  c->U0 = k.take<double>(nu);
  c->U1 = k.take<double>(nu);
  c->U2 = c->nst >= 3 ? k.take<double>(nu) : nullptr;
  c->mean = k.take<char>(tsz * 3 * ne);
  c->cls = k.take<uint8_t>(ne);
  c->mean64 = c->mixed ? k.take<double>(3 * (size_t)ne) : nullptr;
  c->flist = k.take<int>(ne);
  c->fcnt = k.take<unsigned>(MAX_STAGES);
  c->d_send_idx = k.take<int>(c->halo_send.size());
  c->d_recv_idx = k.take<int>(c->halo_recv.size());
  c->wd = k.take<uint8_t>(ne);
  c->wd_stage = k.take<uint8_t>(ne);
  c->eflux = k.take<char>(tsz * 3 * NQE * nint);
  c->emode = k.take<uint8_t>(nint);
  c->frc = k.take<char>(tsz * 3 * nn);
  c->partial = k.take<double>(4 * (size_t)mass_partial_count(ne));
  c->result = k.take<double>(2);
  c->staging = k.take<double>(std::max(nu, 3 * (size_t)nn));
  c->step = k.take<long long>(1);
  c->err = k.take<int>(1);
  c->dtbits = k.take<unsigned long long>(1);
  // tile edge lists, sized for the smallest tile (64) and the worst case of the edge count
  const int mt = max_tile_edges(H);
  DevTiles &T = c->tiles;
  T.start = k.take<int>((ne + 63) / 64 + 1);
  T.ea = k.take<int>(mt);
  T.eb = k.take<int>(mt);
  T.code = k.take<uint8_t>(mt);
  T.geo = k.take<char>(tsz * 3 * mt);
  T.hb = k.take<double>(2 * (size_t)mt);
  T.hbq = k.take<char>(tsz * NQE * mt);
  *bytes = k.off;
}

// Build and upload the tile edge lists for tile size `tile` (outside any stream capture).
static int prepare_tiles(dgswem_ctx *c, int tile) {
  if (c->tiles.tile == tile) return 0;
  TileEdges &H = c->htiles;
  build_tile_edges(c->hm, tile, H);
  DevTiles &T = c->tiles;
  const int mt = max_tile_edges(c->hm);
  if (H.n > mt) return ctx_fail(c, DGSWEM_EINVAL, "tile edge list larger than its buffer");
  c->host_keep.push_back(typed(H.geo, c->mixed));
  std::vector<double> hbq;
  edge_point_hb(c->P, H.hb.data(), H.hb.data() + H.n, H.n, hbq);
  c->host_keep.push_back(typed(hbq, c->mixed));
  cudaStream_t s = c->st;
  int r = 0;
  if (T.hbq)
    r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<void *>(T.hbq), c->host_keep.back().data(),
                                     c->host_keep.back().size(), cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(T.start), H.start.data(), H.start.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(T.ea), H.ea.data(), H.n * sizeof(int), cudaMemcpyHostToDevice, s),
                "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(T.eb), H.eb.data(), H.n * sizeof(int), cudaMemcpyHostToDevice, s),
                "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<uint8_t *>(T.code), H.code.data(), H.n, cudaMemcpyHostToDevice, s),
                "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<void *>(T.geo), c->host_keep[c->host_keep.size() - 2].data(),
                                   c->host_keep[c->host_keep.size() - 2].size(), cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<double *>(T.hb), H.hb.data(), H.hb.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, s), "tiles");
  if (r) return c->sticky;
  if (int e = ctx_cuda(c, cudaStreamSynchronize(s), "tiles sync")) return e;
  T.tile = tile;
  T.ntiles = H.ntiles;
  T.n = H.n;
  return 0;
}

// The mesh view whose every element counts as own and updated: the initial and single-operator
// wet/dry and limiter calls apply to the ghost elements of a part as well.
static DevMesh whole(const DevMesh &m) {
  DevMesh a = m;
  a.nown = a.nact = a.ne;
  return a;
}

// ------------------------------------------------------------------ one step
static const char *kname_forcing = "forcing";
static const char *kname_edge = "edge_flux";
static const char *kname_element = "element_update";
static const char *kname_limwd = "limiter_wetdry";
static const char *kname_front = "front_update";
static const char *kname_limwd_front = "front_limiter_wetdry";
static const char *kname_advance = "advance";

static void mark(dgswem_ctx *c, const char *name, std::vector<const char *> *names, int *ev_i) {
  if (!names) return;
  cudaEventRecordWithFlags(c->ev[*ev_i], c->st, cudaEventRecordExternal);
  names->push_back(name);
  ++*ev_i;
}

// State buffer that stage `stage` writes: intermediate stages alternate U1 / U2, the last one
// writes u^(n+1) over U0 (each element reads only its own u^n there).
static double *stage_out(dgswem_ctx *c, int stage) {
  return stage == c->nst - 1 ? c->U0 : (stage % 2 == 0 ? c->U1 : c->U2);
}

// Issue the kernels of one stage on the context stream (ev_i: next kernel-timing event).
static void enqueue_stage(dgswem_ctx *c, int variant, int block, int stage, std::vector<const char *> *names,
                          int *ev_i) {
  const bool split = variant == DGSWEM_VARIANT_SPLIT;
  const LaunchCfg cfg{block, c->st};
  const Phys &ph = c->ph;
  {
    // stage 0 reads u^n (U0); intermediate stages alternate U1 / U2; the last writes over U0
    double *uin = stage == 0 ? c->U0 : ((stage - 1) % 2 == 0 ? c->U1 : c->U2);
    double *out = stage_out(c, stage);
    const Clock clk{c->step, c->t0, c->dt};
    const bool inline_frc = ph.hurricane && c->mixed;  // mixed form: vortex evaluated per element vertex
    if (ph.hurricane && !inline_frc) {
      mark(c, kname_forcing, names, ev_i);
      launch_forcing(c->mixed, c->dm, ph, clk, c->rtau[stage], 0.0, c->frc, cfg);
    }
    StageArgs sa{};
    sa.uin = uin;
    sa.un = c->U0;
    sa.uout = out;
    sa.mean = ph.limiter ? c->mean : nullptr;
    sa.wd = ph.wetdry ? c->wd : nullptr;
    sa.eflux = c->eflux;
    sa.emode = c->emode;
    sa.frc = (ph.hurricane && !inline_frc) ? c->frc : nullptr;
    sa.frc_inline = inline_frc ? 1 : 0;
    sa.clk = clk;
    sa.tau = c->rtau[stage];
    sa.ra = c->ra[stage];
    sa.rb = c->rb[stage];
    sa.rc = c->rc[stage];
    sa.rcdt = sa.rc * c->dt;
    sa.rk_form = rk_form_of(sa.ra, sa.rb, sa.rc);
    sa.err = c->err;
    // float form with wetting/drying: the element kernels list the front elements, which the front
    // kernels update in double
    const bool front = c->mixed && ph.wetdry;
    sa.cls = front ? c->cls : nullptr;
    sa.mean64 = front ? c->mean64 : nullptr;
    sa.flist = c->flist;
    sa.fcnt = c->fcnt + stage;
    sa.fcnt_prev = front ? c->fcnt + (stage + c->nst - 1) % c->nst : nullptr;
    sa.fbase = 0;
    if (variant == DGSWEM_VARIANT_TILED || variant == DGSWEM_VARIANT_TILED_WIDE) {
      mark(c, kname_element, names, ev_i);
      launch_tile(c->mixed, c->P, variant == DGSWEM_VARIANT_TILED_WIDE, false, c->dm, c->tiles, sa, ph, cfg);
    } else {
      if (split && c->dm.nint > 0) {
        mark(c, kname_edge, names, ev_i);
        launch_edge(c->mixed, c->P, c->dm, sa, ph, cfg);
      }
      mark(c, kname_element, names, ev_i);
      launch_element(c->mixed, c->P, split, false, c->dm, sa, ph, cfg);
    }
    if (front) {
      mark(c, kname_front, names, ev_i);
      launch_front(c->P, c->dm, sa, ph, 0, c->st);
    }
    if (ph.limiter || ph.wetdry) {
      if (front) {  // before the float limiter, which changes the non-front states they read
        mark(c, kname_limwd_front, names, ev_i);
        launch_limwd_front(c->P, ph.limiter, ph.wetdry, c->dm, out, c->mean64, c->cls, c->wd, ph, c->err, c->flist,
                           sa.fcnt, c->st);
      }
      mark(c, kname_limwd, names, ev_i);
      launch_limwd(c->mixed, c->P, ph.limiter, ph.wetdry, c->dm, out, c->mean, c->wd, ph, c->err, cfg, sa.cls);
    }
  }
}

// Issue the kernels of one time step (the scheme's stages) on the context stream.
static int enqueue_step(dgswem_ctx *c, int variant, int block, std::vector<const char *> *names) {
  int ev_i = 0;
  for (int stage = 0; stage < c->nst; ++stage) enqueue_stage(c, variant, block, stage, names, &ev_i);
  mark(c, kname_advance, names, &ev_i);
  launch_advance(c->step, c->st);
  if (names) {
    cudaEventRecordWithFlags(c->ev[ev_i], c->st, cudaEventRecordExternal);
  }
  return 0;
}

static int kernels_in_step(const dgswem_ctx *c, int variant) {
  const int per_stage = 1 + ((c->ph.hurricane && !c->mixed) ? 1 : 0) + ((variant == DGSWEM_VARIANT_SPLIT && c->dm.nint > 0) ? 1 : 0) +
                  ((c->ph.limiter || c->ph.wetdry) ? 1 : 0) + ((c->mixed && c->ph.wetdry) ? 2 : 0);
  return c->nst * per_stage + 1;
}

static void destroy_alt(dgswem_ctx *c) {
  if (c->exec_alt) cudaGraphExecDestroy(c->exec_alt);
  if (c->graph_alt) cudaGraphDestroy(c->graph_alt);
  c->exec_alt = nullptr;
  c->graph_alt = nullptr;
}

static void destroy_graph(dgswem_ctx *c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  destroy_alt(c);
}

// Capture one step for (variant, block) with or without the kernel-timing event nodes, as the
// active graph (the caller has released the previous one).
static int capture_one(dgswem_ctx *c, int variant, int block, bool timing) {
  if (!c->ensemble && (variant == DGSWEM_VARIANT_TILED || variant == DGSWEM_VARIANT_TILED_WIDE))
    if (int r = prepare_tiles(c, block)) return r;
  std::vector<const char *> names;
  if (timing) {
    const int need = kernels_in_step(c, variant) + 1;
    while ((int)c->ev.size() < need) {
      cudaEvent_t e;
      if (int r = ctx_cuda(c, cudaEventCreate(&e), "cudaEventCreate")) return r;
      c->ev.push_back(e);
    }
  }
  if (int r = ctx_cuda(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "begin capture")) return r;
  if (c->ensemble)
    ensemble_enqueue_step(c, timing ? &names : nullptr);
  else
    enqueue_step(c, variant, block, timing ? &names : nullptr);
  cudaError_t e = cudaStreamEndCapture(c->st, &c->graph);
  if (int r = ctx_cuda(c, e, "end capture")) return r;
  if (int r = ctx_cuda(c, cudaGraphInstantiate(&c->exec, c->graph, 0), "graph instantiate")) return r;
  c->graph_t0 = c->t0;
  c->variant = variant;
  c->block = block;
  c->timing = timing;
  if (timing) c->knames = names;
  c->kernels_per_step = c->ensemble ? c->kernels_per_step : kernels_in_step(c, variant);
  return 0;
}

int capture_graph(dgswem_ctx *c, int variant, int block, bool timing) {
  destroy_graph(c);
  return capture_one(c, variant, block, timing);
}

int read_error_word(dgswem_ctx *c) {
  if (int r = ctx_cuda(c, cudaMemcpyAsync(c->h_err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "read error word"))
    return r;
  if (int r = ctx_cuda(c, cudaStreamSynchronize(c->st), "stream sync")) return r;
  const int w = *c->h_err;
  if (w & ERR_TIMEOUT) return ctx_fail(c, DGSWEM_ETIMEOUT, "a device-side grid barrier wait timed out");
  if (w & ERR_NONFINITE) return ctx_fail(c, DGSWEM_ENONFINITE, "non-finite value in the state");
  if (w & ERR_NEGDEPTH) return ctx_fail(c, DGSWEM_ENEGDEPTH, "negative element mean depth after wetting/drying");
  return 0;
}

int attach_common(dgswem_ctx *c, void *d_workspace, size_t bytes, void *stream) {
  if (c->attached) return ctx_fail(c, DGSWEM_ESTATE, "already attached");
  if (!d_workspace || bytes < c->need) return ctx_fail(c, DGSWEM_ENOMEM, "workspace smaller than dgswem_workspace_size");
  if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign)
    return ctx_fail(c, DGSWEM_EINVAL, "workspace must be 256-byte aligned");
  if (stream) {
    c->st = (cudaStream_t)stream;
  } else {
    if (int r = ctx_cuda(c, cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking), "stream create")) return r;
    c->st = c->own_stream;
  }
  if (int r = ctx_cuda(c, cudaMallocHost(&c->h_pinned, 64), "pinned scratch")) return r;
  c->h_err = reinterpret_cast<int *>(c->h_pinned);
  c->h_res = reinterpret_cast<double *>(static_cast<char *>(c->h_pinned) + 16);
  c->ws = static_cast<char *>(d_workspace);
  c->ws_bytes = bytes;
  upload_all_tables();
  return ctx_cuda(c, cudaGetLastError(), "table upload");
}

int upload_mesh(dgswem_ctx *c, const HostMesh &H, const DevMesh &m, int *perm, int *iperm) {
  cudaStream_t s = c->st;
  auto put = [&](const void *dst, const void *src, size_t n) -> int {
    if (n == 0) return 0;
    return ctx_cuda(c, cudaMemcpyAsync(const_cast<void *>(dst), src, n, cudaMemcpyHostToDevice, s), "upload");
  };
  const size_t base = c->host_keep.size();
  c->host_keep.push_back(typed(H.geo, c->mixed));
  c->host_keep.push_back(typed(H.lima, c->mixed));
  c->host_keep.push_back(typed(H.edgeo, c->mixed));
  {
    std::vector<double> v;
    area_point_hb(c->P, H, v);
    c->host_keep.push_back(typed(v, c->mixed));
    if (m.hbq_d) c->host_keep.push_back(typed(v, false));
    edge_point_hb(c->P, H.edhb.data(), H.edhb.data() + H.nint, H.nint, v);
    c->host_keep.push_back(typed(v, c->mixed));
  }
  const size_t ihbq = base + 3, iedhbq = base + (m.hbq_d ? 5 : 4);
  int r = 0;
  r |= put(m.geo, c->host_keep[base].data(), c->host_keep[base].size());
  r |= put(m.hbv, H.hbv.data(), H.hbv.size() * sizeof(double));
  r |= put(m.area, H.area.data(), H.area.size() * sizeof(double));
  r |= put(m.inradius, H.inradius.data(), H.inradius.size() * sizeof(double));
  r |= put(m.nbr, H.nbr.data(), H.nbr.size() * sizeof(int));
  r |= put(m.nle, H.nle.data(), H.nle.size());
  r |= put(m.vnode, H.vnode.data(), H.vnode.size() * sizeof(int));
  r |= put(m.lima, c->host_keep[base + 1].data(), c->host_keep[base + 1].size());
  r |= put(m.limj, H.limj.data(), H.limj.size() * sizeof(uint16_t));
  r |= put(m.eledge, H.eledge.data(), H.eledge.size() * sizeof(int));
  r |= put(m.edel, H.edel.data(), H.edel.size() * sizeof(int));
  r |= put(m.edle, H.edle.data(), H.edle.size());
  r |= put(m.edgeo, c->host_keep[base + 2].data(), c->host_keep[base + 2].size());
  r |= put(m.edhb, H.edhb.data(), H.edhb.size() * sizeof(double));
  if (m.hbq) r |= put(m.hbq, c->host_keep[ihbq].data(), c->host_keep[ihbq].size());
  if (m.edhbq) r |= put(m.edhbq, c->host_keep[iedhbq].data(), c->host_keep[iedhbq].size());
  if (m.geo_d) r |= put(m.geo_d, H.geo.data(), H.geo.size() * sizeof(double));
  if (m.lima_d) r |= put(m.lima_d, H.lima.data(), H.lima.size() * sizeof(double));
  if (m.hbq_d) r |= put(m.hbq_d, c->host_keep[base + 4].data(), c->host_keep[base + 4].size());
  r |= put(m.nodexy, H.nodexy.data(), H.nodexy.size() * sizeof(double));
  if (m.elf) {
    c->host_keep.push_back(element_floats(H));
    r |= put(m.elf, c->host_keep.back().data(), c->host_keep.back().size());
  }
  r |= put(perm, H.perm.data(), H.perm.size() * sizeof(int));
  r |= put(iperm, H.iperm.data(), H.iperm.size() * sizeof(int));
  return r ? c->sticky : 0;
}

// ------------------------------------------------------------------ C ABI

// dgswem_create, and dgswem_create_part when part is set.
static int create_common(const dgswem_mesh *mesh, const double *bathy, const dgswem_params *params,
                         const dgswem_init *init, const dgswem_tuning *tuning, const dgswem_part *part,
                         dgswem_ctx **out) {
  if (!out) return DGSWEM_EINVAL;
  *out = nullptr;
  if (!mesh || !bathy) return DGSWEM_EINVAL;
  std::string msg;
  if (check_params(params, msg)) return DGSWEM_EINVAL;
  if (part) {  // a part runs with the global time step, fixed by the caller
    if (!(params->dt > 0) || !part->elem_class || part->n_send < 0 || part->n_recv < 0 ||
        (part->n_send > 0 && !part->send_elems) || (part->n_recv > 0 && !part->recv_elems))
      return DGSWEM_EINVAL;
  }
  dgswem_ctx *c = new dgswem_ctx();
  c->prm = *params;
  if (tuning) c->tun = *tuning;
  if (c->tun.variant < 0 || c->tun.variant > DGSWEM_VARIANT_TILED_WIDE || (c->tun.block != 0 && c->tun.block != 64 && c->tun.block != 128 &&
                                                    c->tun.block != 256) ||
      c->tun.reorder < 0 || c->tun.reorder > 2) {
    delete c;
    return DGSWEM_EINVAL;
  }
  c->P = params->p;
  c->ND = nd_of(c->P);
  c->mixed = params->precision == DGSWEM_FP32_MIXED;
  c->nst = rk_stage_table(*params, c->ra, c->rb, c->rc, c->rtau);
  int r = preprocess_mesh(*mesh, bathy, c->tun.reorder != 2, c->hm, msg, part ? part->elem_class : nullptr);
  if (r) {
    delete c;
    return r;
  }
  if (part) {
    // send: own elements; receive: ghost elements (caller indices, checked against the classes)
    c->part = true;
    for (int i = 0; i < part->n_send; ++i) {
      const int e = part->send_elems[i];
      if (e < 0 || e >= c->hm.ne || part->elem_class[e] != 0) { delete c; return DGSWEM_EINVAL; }
      c->halo_send.push_back(c->hm.iperm[e]);
    }
    for (int i = 0; i < part->n_recv; ++i) {
      const int e = part->recv_elems[i];
      if (e < 0 || e >= c->hm.ne || part->elem_class[e] == 0) { delete c; return DGSWEM_EINVAL; }
      c->halo_recv.push_back(c->hm.iperm[e]);
    }
  }
  c->ph = make_phys(*params);
  c->t0 = init ? init->t0 : 0.0;
  if (!std::isfinite(c->t0)) { delete c; return DGSWEM_EINVAL; }
  const int ne = c->hm.ne, nn = c->hm.nn, ND = c->ND;
  if (init && init->modal) {
    c->init_kind = 1;
    c->init_modal.resize(3 * (size_t)ND * ne);
    for (size_t row = 0; row < 3 * (size_t)ND; ++row)
      for (int i = 0; i < ne; ++i) {
        const double v = init->modal[row * ne + c->hm.perm[i]];
        if (!std::isfinite(v)) { delete c; return DGSWEM_EINVAL; }
        c->init_modal[row * ne + i] = v;
      }
  } else if (init && init->nodal) {
    c->init_kind = 2;
    c->init_nodal.assign(init->nodal, init->nodal + 3 * (size_t)nn);
    for (double v : c->init_nodal)
      if (!std::isfinite(v)) { delete c; return DGSWEM_EINVAL; }
  }
  layout(c, nullptr, &c->need);
  *out = c;
  return 0;
}

extern "C" {

int dgswem_create(const dgswem_mesh *mesh, const double *bathy, const dgswem_params *params,
                  const dgswem_init *init, const dgswem_tuning *tuning, dgswem_ctx **out) {
  return create_common(mesh, bathy, params, init, tuning, nullptr, out);
}

int dgswem_create_part(const dgswem_mesh *mesh, const double *bathy, const dgswem_params *params,
                       const dgswem_init *init, const dgswem_tuning *tuning, const dgswem_part *part,
                       dgswem_ctx **out) {
  if (!part) {
    if (out) *out = nullptr;
    return DGSWEM_EINVAL;
  }
  return create_common(mesh, bathy, params, init, tuning, part, out);
}

int dgswem_workspace_size(const dgswem_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return DGSWEM_EINVAL;
  *bytes = ctx->need;
  return 0;
}

static int upload_static(dgswem_ctx *c) {
  c->host_keep.clear();
  return upload_mesh(c, c->hm, c->dm, c->d_perm, c->d_iperm);
}

static int autotune(dgswem_ctx *c, int *best_variant, int *best_block) {
  std::vector<int> variants, blocks;
  if (c->tun.variant == DGSWEM_VARIANT_AUTO) {
    variants = {DGSWEM_VARIANT_SPLIT, DGSWEM_VARIANT_FUSED, DGSWEM_VARIANT_TILED};
    // the wider register bound differs only for the float form at p = 1
    if (c->mixed && c->P == 1) variants.push_back(DGSWEM_VARIANT_TILED_WIDE);
  } else {
    variants = {c->tun.variant};
  }
  if (c->tun.block == 0)
    blocks = {64, 128, 256};
  else
    blocks = {c->tun.block};
  *best_variant = variants[0];
  *best_block = blocks[0];
  if (variants.size() * blocks.size() == 1) return 0;
  const size_t nu = 3 * (size_t)c->ND * c->hm.ne;
  cudaStream_t s = c->st;
  // save the state, the flags and the step counter; every trial restores them
  std::vector<double> save_u(nu);
  std::vector<uint8_t> save_wd(c->hm.ne);
  if (int r = ctx_cuda(c, cudaMemcpyAsync(save_u.data(), c->U0, nu * sizeof(double), cudaMemcpyDeviceToHost, s), "tune save")) return r;
  if (int r = ctx_cuda(c, cudaMemcpyAsync(save_wd.data(), c->wd, c->hm.ne, cudaMemcpyDeviceToHost, s), "tune save")) return r;
  if (int r = ctx_cuda(c, cudaStreamSynchronize(s), "tune sync")) return r;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Per candidate: one replay to estimate the step time, then the best of three batches sized to
  // about 1 ms each (short single samples cannot separate candidates a few percent apart).  The
  // first candidate is also replayed for ~5 ms beforehand so that every trial sees warm clocks.
  auto timed = [&](int n, float *ms) -> int {
    cudaEventRecord(e0, s);
    for (int i = 0; i < n; ++i) cudaGraphLaunch(c->exec, s);
    cudaEventRecord(e1, s);
    if (int r = ctx_cuda(c, cudaEventSynchronize(e1), "tune timing")) return r;
    cudaEventElapsedTime(ms, e0, e1);
    return 0;
  };
  auto restore = [&]() {
    cudaMemcpyAsync(c->U0, save_u.data(), nu * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(c->wd, save_wd.data(), c->hm.ne, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(c->step, 0, sizeof(long long), s);
    cudaMemsetAsync(c->err, 0, sizeof(int), s);
    cudaMemsetAsync(c->fcnt, 0, MAX_STAGES * sizeof(unsigned), s);
  };
  float best = INFINITY;
  bool warmed = false;
  for (int v : variants)
    for (int b : blocks) {
      if (int r = capture_graph(c, v, b, false)) return r;
      float t1 = 0, ms = 0;
      if (int r = timed(1, &t1)) return r;
      const int reps = std::min(200, std::max(3, (int)std::ceil(1.0f / std::max(t1, 1e-3f))));
      if (!warmed) {
        if (int r = timed(std::min(1000, 5 * reps), &ms)) return r;
        warmed = true;
      }
      float per = INFINITY;
      for (int k = 0; k < 3; ++k) {
        if (int r = timed(reps, &ms)) return r;
        per = std::min(per, ms / reps);
      }
      c->tune_log.push_back({v, b, per});
      if (per < best) {
        best = per;
        *best_variant = v;
        *best_block = b;
      }
      restore();
    }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ctx_cuda(c, cudaGetLastError(), "autotune");
}

int dgswem_attach(dgswem_ctx *c, void *d_workspace, size_t bytes, void *stream) {
  if (!c) return DGSWEM_EINVAL;
  if (c->ensemble) return ensemble_attach(c, d_workspace, bytes, stream);
  if (int r = attach_common(c, d_workspace, bytes, stream)) return r;
  size_t sz = 0;
  layout(c, c->ws, &sz);
  cudaStream_t s = c->st;
  if (int r = upload_static(c)) return r;
  if (c->part) {
    if (!c->halo_send.empty())
      cudaMemcpyAsync(c->d_send_idx, c->halo_send.data(), c->halo_send.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (!c->halo_recv.empty())
      cudaMemcpyAsync(c->d_recv_idx, c->halo_recv.data(), c->halo_recv.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  }
  c->tiles.tile = 0;
  const size_t nu = 3 * (size_t)c->ND * c->hm.ne;
  cudaMemsetAsync(c->step, 0, sizeof(long long), s);
  cudaMemsetAsync(c->err, 0, sizeof(int), s);
  cudaMemsetAsync(c->wd, 0, c->hm.ne, s);
  cudaMemsetAsync(c->fcnt, 0, MAX_STAGES * sizeof(unsigned), s);
  cudaMemsetAsync(c->U1, 0, nu * sizeof(double), s);
  if (c->init_kind == 1) {
    cudaMemcpyAsync(c->U0, c->init_modal.data(), nu * sizeof(double), cudaMemcpyHostToDevice, s);
  } else if (c->init_kind == 2) {
    cudaMemcpyAsync(c->staging, c->init_nodal.data(), c->init_nodal.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    launch_init_nodal(c->P, c->dm, c->staging, c->U0, s);
  } else {
    cudaMemsetAsync(c->U0, 0, nu * sizeof(double), s);
  }
  const LaunchCfg cfg{128, s};
  if (c->ph.wetdry) launch_limwd(c->mixed, c->P, false, 1, whole(c->dm), c->U0, c->mean, c->wd, c->ph, c->err, cfg);
  if (c->prm.dt > 0) {
    c->dt = c->prm.dt;
  } else {
    launch_dt(c->P, c->dm, c->U0, c->ph, c->dtbits, s);
    unsigned long long bits = 0;
    if (int r = ctx_cuda(c, cudaMemcpyAsync(c->h_res, c->dtbits, 8, cudaMemcpyDeviceToHost, s), "dt readback")) return r;
    if (int r = ctx_cuda(c, cudaStreamSynchronize(s), "attach sync")) return r;
    std::memcpy(&bits, c->h_res, 8);
    double best;
    std::memcpy(&best, &bits, 8);
    if (!(best > 0) || !std::isfinite(best)) return ctx_fail(c, DGSWEM_EINVAL, "no element with a positive wave speed: dt undefined");
    c->dt = c->prm.cfl * 3.0 / (2.0 * c->P + 1.0) * best;
  }
  if (int r = ctx_cuda(c, cudaStreamSynchronize(s), "attach sync")) return r;
  if (int r = ctx_cuda(c, cudaGetLastError(), "attach")) return r;
  c->attached = true;
  int v = c->tun.variant, b = c->tun.block;
  if (int r = autotune(c, &v, &b)) return r;
  if (int r = capture_graph(c, v, b, false)) return r;
  return read_error_word(c);
}

int dgswem_step(dgswem_ctx *c, int32_t n) {
  if (!c) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "step before attach");
  if (n < 0) return DGSWEM_EINVAL;
  if (c->part) return ctx_fail(c, DGSWEM_ESTATE, "a part steps with dgswem_stage_compute / dgswem_stage_finish");
  for (int i = 0; i < n; ++i) {
    cudaError_t e = cudaGraphLaunch(c->exec, c->st);
    if (e != cudaSuccess) return ctx_cuda(c, e, "graph launch");
    c->steps_done++;
  }
  return 0;
}

int dgswem_sync(dgswem_ctx *c) {
  if (!c) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  return read_error_word(c);
}

int dgswem_get_state(dgswem_ctx *c, double *hz, double *hqx, double *hqy) {
  if (!c) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "use dgswem_ensemble_get_state");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  const int ne = c->hm.ne, ND = c->ND;
  launch_permute(c->U0, c->staging, c->d_iperm, 3 * ND, ne, c->st);
  double *dst[3] = {hz, hqx, hqy};
  for (int v = 0; v < 3; ++v)
    if (dst[v])
      if (int r = ctx_cuda(c, cudaMemcpyAsync(dst[v], c->staging + (size_t)v * ND * ne, (size_t)ND * ne * sizeof(double),
                                              cudaMemcpyDeviceToHost, c->st), "state readback"))
        return r;
  return read_error_word(c);
}

int dgswem_set_state(dgswem_ctx *c, const double *hz, const double *hqx, const double *hqy, double t) {
  if (!c || !hz || !hqx || !hqy || !std::isfinite(t)) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  const int ne = c->hm.ne, ND = c->ND;
  const double *src[3] = {hz, hqx, hqy};
  for (int v = 0; v < 3; ++v)
    if (int r = ctx_cuda(c, cudaMemcpyAsync(c->staging + (size_t)v * ND * ne, src[v], (size_t)ND * ne * sizeof(double),
                                            cudaMemcpyHostToDevice, c->st), "state upload"))
      return r;
  launch_permute(c->staging, c->U0, c->d_perm, 3 * ND, ne, c->st);
  cudaMemsetAsync(c->step, 0, sizeof(long long), c->st);
  c->t0 = t;
  c->steps_done = 0;
  if (c->ph.wetdry)  // recompute the flags only; the state is not modified
    launch_limwd(c->mixed, c->P, false, 2, whole(c->dm), c->U0, c->mean, c->wd, c->ph, c->err, LaunchCfg{128, c->st});
  if (int r = ctx_cuda(c, cudaGetLastError(), "set_state")) return r;
  // the captured graph bakes t0 into its kernel parameters (the step count comes from the device
  // counter reset above): recapture only for another t0
  if (c->exec && c->graph_t0 == t) return 0;
  return capture_graph(c, c->variant, c->block, c->timing);
}

int dgswem_mass(dgswem_ctx *c, double *mz, double *vol) {
  if (!c || !mz || !vol) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  launch_mass(c->P, c->dm, c->U0, c->partial, c->result, c->st);
  if (int r = ctx_cuda(c, cudaMemcpyAsync(c->h_res, c->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "mass readback"))
    return r;
  if (int r = read_error_word(c)) return r;
  *mz = c->h_res[0];
  *vol = c->h_res[1];
  return 0;
}

int dgswem_info(dgswem_ctx *c, double *dt, double *t, int64_t *steps) {
  if (!c) return DGSWEM_EINVAL;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (dt) *dt = c->dt;
  if (t) *t = c->t0 + (double)c->steps_done * c->dt;
  if (steps) *steps = c->steps_done;
  return 0;
}

int dgswem_get_flags(dgswem_ctx *c, uint8_t *h) {
  if (!c || !h) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  launch_permute_u8(c->wd, c->wd_stage, c->d_iperm, c->hm.ne, c->st);
  if (int r = ctx_cuda(c, cudaMemcpyAsync(h, c->wd_stage, c->hm.ne, cudaMemcpyDeviceToHost, c->st), "flags readback"))
    return r;
  return read_error_word(c);
}

void dgswem_destroy(dgswem_ctx *c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  destroy_graph(c);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  ensemble_release(c);
  delete c;
}

const char *dgswem_last_error(const dgswem_ctx *c) {
  if (!c) return "null context";
  return c->errmsg.c_str();
}

// ---- single operators
int dgswem_eval_rhs(dgswem_ctx *c, double t, double *h_out) {
  if (!c || !h_out || !std::isfinite(t)) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  const LaunchCfg cfg{c->block, c->st};
  const bool inline_frc = c->ph.hurricane && c->mixed;
  if (c->ph.hurricane && !inline_frc) launch_forcing(c->mixed, c->dm, c->ph, Clock{nullptr, 0, 0}, 0.0, t, c->frc, cfg);
  StageArgs sa{};
  sa.uin = c->U0;
  sa.un = c->U0;
  sa.uout = c->U1;
  sa.mean = nullptr;
  sa.wd = c->ph.wetdry ? c->wd : nullptr;
  sa.eflux = c->eflux;
  sa.emode = c->emode;
  sa.frc = (c->ph.hurricane && !inline_frc) ? c->frc : nullptr;
  sa.frc_inline = inline_frc ? 1 : 0;
  sa.clk = Clock{nullptr, 0.0, c->dt};
  sa.tau = 0.0;
  sa.ra = 0.0;
  sa.rb = 1.0;
  sa.rc = 1.0;
  sa.rcdt = c->dt;
  sa.rk_form = 0;
  sa.err = c->err;
  sa.tide_t = t;
  // float form with wetting/drying: the front elements take the double path, as in a step
  const bool front = c->mixed && c->ph.wetdry;
  sa.cls = front ? c->cls : nullptr;
  sa.mean64 = nullptr;
  sa.flist = c->flist;
  sa.fcnt = c->fcnt;
  sa.fcnt_prev = nullptr;
  sa.fbase = 0;
  if (front) cudaMemsetAsync(c->fcnt, 0, sizeof(unsigned), c->st);
  const bool split = c->variant == DGSWEM_VARIANT_SPLIT;
  if (c->variant == DGSWEM_VARIANT_TILED || c->variant == DGSWEM_VARIANT_TILED_WIDE) {
    launch_tile(c->mixed, c->P, c->variant == DGSWEM_VARIANT_TILED_WIDE, true, c->dm, c->tiles, sa, c->ph, cfg);
  } else {
    if (split) launch_edge(c->mixed, c->P, c->dm, sa, c->ph, cfg);
    launch_element(c->mixed, c->P, split, true, c->dm, sa, c->ph, cfg);
  }
  if (front) {
    launch_front(c->P, c->dm, sa, c->ph, 1, c->st);
    cudaMemsetAsync(c->fcnt, 0, sizeof(unsigned), c->st);  // the step graph expects zero counters
  }
  const int ne = c->hm.ne, ND = c->ND;
  launch_permute(c->U1, c->staging, c->d_iperm, 3 * ND, ne, c->st);
  if (int r = ctx_cuda(c, cudaMemcpyAsync(h_out, c->staging, 3 * (size_t)ND * ne * sizeof(double), cudaMemcpyDeviceToHost,
                                          c->st), "rhs readback"))
    return r;
  return read_error_word(c);
}

int dgswem_apply_limiter(dgswem_ctx *c) {
  if (!c) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  launch_copy_means(c->mixed, c->P, c->hm.ne, c->U0, c->mean, c->st);
  launch_limwd(c->mixed, c->P, true, 0, whole(c->dm), c->U0, c->mean, c->wd, c->ph, c->err, LaunchCfg{c->block, c->st});
  if (int r = ctx_cuda(c, cudaGetLastError(), "limiter")) return r;
  return read_error_word(c);
}

int dgswem_apply_wetdry(dgswem_ctx *c) {
  if (!c) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  Phys ph = c->ph;
  if (!(ph.h0 > 0)) return ctx_fail(c, DGSWEM_EINVAL, "wetting/drying is off (h0 = 0)");
  launch_limwd(c->mixed, c->P, false, 1, whole(c->dm), c->U0, c->mean, c->wd, ph, c->err, LaunchCfg{c->block, c->st});
  if (int r = ctx_cuda(c, cudaGetLastError(), "wetdry")) return r;
  return read_error_word(c);
}

int dgswem_eval_forcing(dgswem_ctx *c, double t, double *h_out) {
  if (!c || !h_out || !std::isfinite(t)) return DGSWEM_EINVAL;
  if (c->ensemble) return ctx_fail(c, DGSWEM_EINVAL, "not available for an ensemble");
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (!c->ph.hurricane) return ctx_fail(c, DGSWEM_EINVAL, "no hurricane forcing configured");
  launch_forcing(c->mixed, c->dm, c->ph, Clock{nullptr, 0, 0}, 0.0, t, c->frc, LaunchCfg{256, c->st});
  const size_t n = 3 * (size_t)c->hm.nn;
  std::vector<char> buf(n * (c->mixed ? 4 : 8));
  if (int r = ctx_cuda(c, cudaMemcpyAsync(buf.data(), c->frc, buf.size(), cudaMemcpyDeviceToHost, c->st), "forcing readback"))
    return r;
  if (int r = read_error_word(c)) return r;
  for (size_t i = 0; i < n; ++i)
    h_out[i] = c->mixed ? (double)reinterpret_cast<float *>(buf.data())[i] : reinterpret_cast<double *>(buf.data())[i];
  return 0;
}

// ---- kernel timing
int dgswem_set_kernel_timing(dgswem_ctx *c, int32_t on) {
  if (!c) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (int r = ctx_cuda(c, cudaStreamSynchronize(c->st), "sync")) return r;
  const bool want = on != 0;
  if (want == c->timing && c->exec) return 0;
  if (c->exec_alt && c->alt_timing == want) {  // the other mode is already captured: swap
    std::swap(c->graph, c->graph_alt);
    std::swap(c->exec, c->exec_alt);
    c->alt_timing = c->timing;
    c->timing = want;
    return 0;
  }
  // keep the active graph as the alternative and capture the requested mode
  destroy_alt(c);
  c->graph_alt = c->graph;
  c->exec_alt = c->exec;
  c->alt_timing = c->timing;
  c->graph = nullptr;
  c->exec = nullptr;
  return capture_one(c, c->variant, c->block, want);
}

int dgswem_kernel_times(dgswem_ctx *c, float *ms, const char **names, int32_t cap, int32_t *n) {
  if (!c || !n) return DGSWEM_EINVAL;
  if (!c->timing) return ctx_refuse(c, DGSWEM_ESTATE, "kernel timing is off");
  if (int r = ctx_cuda(c, cudaStreamSynchronize(c->st), "sync")) return r;
  const int k = (int)c->knames.size();
  *n = k;
  for (int i = 0; i < k && i < cap; ++i) {
    float t = 0;
    cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]);
    if (ms) ms[i] = t;
    if (names) names[i] = c->knames[i];
  }
  return ctx_cuda(c, cudaGetLastError(), "kernel times");
}

int dgswem_tune_log(dgswem_ctx *c, int32_t *variant, int32_t *block, float *ms, int32_t cap, int32_t *n) {
  if (!c || !n) return DGSWEM_EINVAL;
  const std::vector<TuneEntry> &log = c->ensemble ? ensemble_tune_log(c) : c->tune_log;
  *n = (int32_t)log.size();
  for (int32_t i = 0; i < *n && i < cap; ++i) {
    if (variant) variant[i] = log[i].variant;
    if (block) block[i] = log[i].block;
    if (ms) ms[i] = log[i].ms_per_step;
  }
  return 0;
}

// ---- a part of a partitioned domain
int dgswem_halo_sizes(dgswem_ctx *c, size_t *send_bytes, size_t *recv_bytes) {
  if (!c || !send_bytes || !recv_bytes) return DGSWEM_EINVAL;
  if (!c->part) return ctx_fail(c, DGSWEM_EINVAL, "not a part (dgswem_create_part)");
  const size_t rec = (3 * (size_t)c->ND + 1) * sizeof(double);
  *send_bytes = c->halo_send.size() * rec;
  *recv_bytes = c->halo_recv.size() * rec;
  return 0;
}

int dgswem_halo_attach(dgswem_ctx *c, void *d_send, void *d_recv) {
  if (!c) return DGSWEM_EINVAL;
  if (!c->part) return ctx_fail(c, DGSWEM_EINVAL, "not a part (dgswem_create_part)");
  if ((!c->halo_send.empty() && !d_send) || (!c->halo_recv.empty() && !d_recv) ||
      reinterpret_cast<uintptr_t>(d_send) % 8 || reinterpret_cast<uintptr_t>(d_recv) % 8)
    return ctx_fail(c, DGSWEM_EINVAL, "halo buffers: null or not 8-byte aligned");
  c->d_send_buf = static_cast<double *>(d_send);
  c->d_recv_buf = static_cast<double *>(d_recv);
  return 0;
}

int dgswem_stage_compute(dgswem_ctx *c) {
  if (!c) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (!c->part) return ctx_fail(c, DGSWEM_EINVAL, "not a part (dgswem_create_part)");
  if (c->stage_open) return ctx_fail(c, DGSWEM_ESTATE, "dgswem_stage_finish first");
  if ((!c->halo_send.empty() && !c->d_send_buf) || (!c->halo_recv.empty() && !c->d_recv_buf))
    return ctx_fail(c, DGSWEM_ESTATE, "dgswem_halo_attach first");
  int ev_i = 0;
  enqueue_stage(c, c->variant, c->block, c->stage_i, nullptr, &ev_i);
  launch_halo_pack(c->ND, c->hm.ne, stage_out(c, c->stage_i), c->wd, c->d_send_idx, (int)c->halo_send.size(),
                   c->d_send_buf, c->st);
  c->stage_open = true;
  return ctx_cuda(c, cudaGetLastError(), "stage compute");
}

int dgswem_stage_finish(dgswem_ctx *c) {
  if (!c) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->stage_open) return ctx_fail(c, DGSWEM_ESTATE, "dgswem_stage_compute first");
  launch_halo_unpack(c->ND, c->hm.ne, stage_out(c, c->stage_i), c->wd, c->d_recv_idx, (int)c->halo_recv.size(),
                     c->d_recv_buf, c->st);
  c->stage_open = false;
  if (++c->stage_i == c->nst) {
    c->stage_i = 0;
    launch_advance(c->step, c->st);
    c->steps_done++;
  }
  return ctx_cuda(c, cudaGetLastError(), "stage finish");
}

int dgswem_graph_info(dgswem_ctx *c, int32_t *kps, int32_t *variant, int32_t *block) {
  if (!c) return DGSWEM_EINVAL;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (kps) *kps = c->kernels_per_step;
  if (variant) *variant = c->variant;
  if (block) *block = c->block;
  return 0;
}

}  // extern "C"
