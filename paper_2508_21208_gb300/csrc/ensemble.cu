// ensemble.cu -- batched storm ensemble: several scenarios (members) on meshes of uneven size,
// advanced together.  Members that pass the same mesh and bathymetry pointers share one copy of
// the mesh statics; each member has its own state, forcing, time step and clock.  A step is one
// persistent cooperative launch (phases separated by bounded grid barriers) or, as the
// autotuner's alternative, one launch per phase; either way it is captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace dg;

struct EnsMember {
  int mesh = 0;
  dgswem_params prm{};
  Phys ph{};
  int init_kind = 0;
  std::vector<double> init_modal, init_nodal;
  double t0 = 0.0, dt = 0.0;
  double *U0 = nullptr, *U1 = nullptr, *U2 = nullptr;
  void *mean = nullptr;  // T [3][ne]
  uint8_t *cls = nullptr;    // [ne] wetting/drying front class (float form)
  double *mean64 = nullptr;  // [3][ne] the front elements' means in double (float form)
  uint8_t *wd = nullptr;
  void *frc = nullptr;
};

struct EnsMesh {
  HostMesh hm;
  DevMesh dm{};
  DevTiles dt{};   // tile edge lists on the device (tile size dt.tile)
  TileEdges ht;
  int *perm = nullptr, *iperm = nullptr;
  const dgswem_mesh *key_mesh = nullptr;
  const double *key_bathy = nullptr;
};

struct EnsembleState {
  std::vector<EnsMesh> meshes;
  std::vector<EnsMember> mem;
  MemberDev *d_mem = nullptr;
  int *d_etile = nullptr, *d_ntile = nullptr;
  unsigned *bar = nullptr;
  unsigned long long *dtbits = nullptr;
  int max_etile = 0, max_ntile = 0, n_etile = 0, n_ntile = 0;
  std::vector<int> h_etile, h_ntile;
  std::vector<MemberDev> h_mem;
  bool persistent = true;
  int block = 128, grid = 0, fault = 0, any_limwd = 0, any_inline = 0, any_front = 0;
  int *flist = nullptr;       // front list of all members (float form with wetting/drying)
  unsigned *fcnt = nullptr;   // its counter per stage
  unsigned long long *work = nullptr;  // persistent launch: work-item claim counters
  unsigned long long timeout_ns = 1000000000ull;  // 1 s per grid-barrier wait
  std::vector<TuneEntry> tune;
};

static void ens_layout(dgswem_ctx *c, char *base, size_t *bytes) {
  EnsembleState &E = *c->ens;
  const int ND = c->ND;
  const size_t tsz = c->mixed ? sizeof(float) : sizeof(double);
  Carver k{base};
  for (EnsMesh &m : E.meshes) {
    carve_mesh(k, m.hm, c->P, c->mixed, m.dm, &m.perm, &m.iperm);
    const int mt = max_tile_edges(m.hm);
    m.dt.start = k.take<int>((m.hm.ne + 63) / 64 + 1);
    m.dt.ea = k.take<int>(mt);
    m.dt.eb = k.take<int>(mt);
    m.dt.code = k.take<uint8_t>(mt);
    m.dt.geo = k.take<char>(tsz * 3 * mt);
    m.dt.hb = k.take<double>(2 * (size_t)mt);
    m.dt.hbq = k.take<char>(tsz * nqe_of(c->P) * mt);
  }
  size_t stage = 0;
  for (EnsMember &mb : E.mem) {
    const HostMesh &H = E.meshes[mb.mesh].hm;
    const size_t nu = 3 * (size_t)ND * H.ne;
    mb.U0 = k.take<double>(nu);
    mb.U1 = k.take<double>(nu);
    mb.U2 = c->nst >= 3 ? k.take<double>(nu) : nullptr;
    mb.mean = k.take<char>(tsz * 3 * (size_t)H.ne);
    mb.cls = k.take<uint8_t>(H.ne);
    mb.mean64 = c->mixed ? k.take<double>(3 * (size_t)H.ne) : nullptr;
    mb.wd = k.take<uint8_t>(H.ne);
    mb.frc = k.take<char>(tsz * 3 * H.nn);
    stage = std::max(stage, std::max(nu, 3 * (size_t)H.nn));
  }
  size_t ne_all = 0;
  for (EnsMember &mb : E.mem) ne_all += E.meshes[mb.mesh].hm.ne;
  E.flist = k.take<int>(ne_all);
  E.fcnt = k.take<unsigned>(MAX_STAGES);
  E.work = k.take<unsigned long long>(3 * MAX_STAGES);
  E.d_mem = k.take<MemberDev>(E.mem.size());
  E.d_etile = k.take<int>(E.max_etile);
  E.d_ntile = k.take<int>(E.max_ntile);
  E.bar = k.take<unsigned>(2);
  E.dtbits = k.take<unsigned long long>(E.mem.size());
  c->staging = k.take<double>(stage);
  c->step = k.take<long long>(1);
  c->err = k.take<int>(1);
  *bytes = k.off;
}

// Flat tile lists for a tile (block) size: element tiles of every member, then node tiles of the
// members with hurricane forcing.
static void build_tiles(dgswem_ctx *c, int block) {
  EnsembleState &E = *c->ens;
  E.h_etile.clear();
  E.h_ntile.clear();
  E.h_mem.assign(E.mem.size(), MemberDev{});
  E.any_limwd = 0;
  E.any_inline = 0;
  E.any_front = 0;
  for (size_t i = 0; i < E.mem.size(); ++i) {
    EnsMember &mb = E.mem[i];
    const EnsMesh &M = E.meshes[mb.mesh];
    MemberDev &d = E.h_mem[i];
    d.m = M.dm;
    d.tl = M.dt;
    d.ph = mb.ph;
    d.U0 = mb.U0;
    d.U1 = mb.U1;
    d.U2 = mb.U2;
    d.mean = mb.mean;
    d.wd = mb.wd;
    d.frc = mb.frc;
    // float form with wetting/drying: the front elements take the double path
    d.cls = (c->mixed && mb.ph.wetdry) ? mb.cls : nullptr;
    d.mean64 = d.cls ? mb.mean64 : nullptr;
    E.any_front |= d.cls ? 1 : 0;
    d.t0 = mb.t0;
    d.dt = mb.dt;
    d.etile0 = (int)E.h_etile.size();
    const int nt = (M.hm.ne + block - 1) / block;
    for (int t = 0; t < nt; ++t) E.h_etile.push_back((int)i);
    E.any_limwd |= (mb.ph.limiter || mb.ph.wetdry) ? 1 : 0;
    E.any_inline |= (mb.ph.hurricane && c->mixed) ? 1 : 0;
  }
  for (size_t i = 0; i < E.mem.size(); ++i) {
    EnsMember &mb = E.mem[i];
    if (!mb.ph.hurricane || c->mixed) continue;  // the mixed form evaluates the vortex per element vertex
    const EnsMesh &M = E.meshes[mb.mesh];
    E.h_mem[i].ntile0 = (int)E.h_ntile.size();
    const int nt = (M.hm.nn + block - 1) / block;
    for (int t = 0; t < nt; ++t) E.h_ntile.push_back((int)i);
  }
  E.n_etile = (int)E.h_etile.size();
  E.n_ntile = (int)E.h_ntile.size();
}

static int upload_tiles(dgswem_ctx *c) {
  EnsembleState &E = *c->ens;
  int r = 0;
  r |= ctx_cuda(c, cudaMemcpyAsync(E.d_mem, E.h_mem.data(), E.h_mem.size() * sizeof(MemberDev),
                                   cudaMemcpyHostToDevice, c->st), "member upload");
  r |= ctx_cuda(c, cudaMemcpyAsync(E.d_etile, E.h_etile.data(), E.h_etile.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, c->st), "tile upload");
  if (!E.h_ntile.empty())
    r |= ctx_cuda(c, cudaMemcpyAsync(E.d_ntile, E.h_ntile.data(), E.h_ntile.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, c->st), "tile upload");
  if (r) return c->sticky;
  return ctx_cuda(c, cudaStreamSynchronize(c->st), "tile upload sync");
}

// (Re)initialise every member's state: modal / nodal / rest, then the wet/dry operator.
static int init_states(dgswem_ctx *c) {
  EnsembleState &E = *c->ens;
  cudaStream_t s = c->st;
  for (EnsMember &mb : E.mem) {
    const EnsMesh &M = E.meshes[mb.mesh];
    const size_t nu = 3 * (size_t)c->ND * M.hm.ne;
    cudaMemsetAsync(mb.U1, 0, nu * sizeof(double), s);
    cudaMemsetAsync(mb.wd, 0, M.hm.ne, s);
    if (mb.init_kind == 1) {
      cudaMemcpyAsync(mb.U0, mb.init_modal.data(), nu * sizeof(double), cudaMemcpyHostToDevice, s);
    } else if (mb.init_kind == 2) {
      cudaMemcpyAsync(c->staging, mb.init_nodal.data(), mb.init_nodal.size() * sizeof(double),
                      cudaMemcpyHostToDevice, s);
      launch_init_nodal(c->P, M.dm, c->staging, mb.U0, s);
    } else {
      cudaMemsetAsync(mb.U0, 0, nu * sizeof(double), s);
    }
    if (mb.ph.wetdry)
      launch_limwd(c->mixed, c->P, false, 1, M.dm, mb.U0, mb.mean, mb.wd, mb.ph, c->err, LaunchCfg{128, s});
    // the nodal staging buffer is reused by the next member: finish this one first
    if (int r = ctx_cuda(c, cudaStreamSynchronize(s), "ensemble init")) return r;
  }
  cudaMemsetAsync(c->step, 0, sizeof(long long), s);
  cudaMemsetAsync(E.bar, 0, 2 * sizeof(unsigned), s);
  cudaMemsetAsync(E.fcnt, 0, MAX_STAGES * sizeof(unsigned), s);
  cudaMemsetAsync(E.work, 0, 3 * MAX_STAGES * sizeof(unsigned long long), s);
  if (int r = ctx_cuda(c, cudaStreamSynchronize(s), "ensemble init")) return r;
  return ctx_cuda(c, cudaGetLastError(), "ensemble init");
}

static int grid_for(dgswem_ctx *c, int block) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = ensemble_blocks_per_sm(c->mixed, c->P, block, c->ens->any_inline != 0);
  return std::min(c->ens->n_etile, per_sm * sms);
}

void ensemble_enqueue_step(dgswem_ctx *c, std::vector<const char *> *names) {
  EnsembleState &E = *c->ens;
  EnsArgs a{};
  a.nstages = c->nst;
  for (int i = 0; i < c->nst; ++i) {
    a.ra[i] = c->ra[i];
    a.rb[i] = c->rb[i];
    a.rc[i] = c->rc[i];
    a.tau[i] = c->rtau[i];
    a.form[i] = rk_form_of(c->ra[i], c->rb[i], c->rc[i]);
  }
  a.mem = E.d_mem;
  a.etile = E.d_etile;
  a.ntile = E.d_ntile;
  a.n_etile = E.n_etile;
  a.n_ntile = E.n_ntile;
  a.step = c->step;
  a.bar = E.bar;
  a.err = c->err;
  a.fault = E.fault;
  a.any_limwd = E.any_limwd;
  a.any_inline = E.any_inline;
  a.any_front = E.any_front;
  a.flist = E.flist;
  a.fcnt = E.fcnt;
  a.work = E.work;
  a.timeout_ns = E.timeout_ns;
  if (names) {
    cudaEventRecordWithFlags(c->ev[0], c->st, cudaEventRecordExternal);
    names->push_back(E.persistent ? "ensemble_persistent_step" : "ensemble_phases");
  }
  cudaError_t e = launch_ensemble(c->mixed, c->P, E.persistent, a, E.block, E.grid, c->st);
  if (e != cudaSuccess) ctx_cuda(c, e, "ensemble launch");
  if (!E.persistent) launch_advance(c->step, c->st);
  if (names) cudaEventRecordWithFlags(c->ev[1], c->st, cudaEventRecordExternal);
  c->kernels_per_step = E.persistent ? 1 : c->nst * ((E.n_ntile > 0) + 1 + E.any_limwd + 2 * E.any_front) + 1;
}

static int upload_mesh_tiles(dgswem_ctx *c, EnsMesh &M, int tile) {
  if (M.dt.tile == tile) return 0;
  build_tile_edges(M.hm, tile, M.ht);
  if (M.ht.n > max_tile_edges(M.hm)) return ctx_fail(c, DGSWEM_EINVAL, "tile list larger than its buffer");
  auto typed = [&](const std::vector<double> &v) {
    std::vector<char> out(v.size() * (c->mixed ? 4 : 8));
    for (size_t i = 0; i < v.size(); ++i) {
      if (c->mixed) reinterpret_cast<float *>(out.data())[i] = (float)v[i];
      else reinterpret_cast<double *>(out.data())[i] = v[i];
    }
    return out;
  };
  const std::vector<char> geo = typed(M.ht.geo);
  std::vector<double> hbq_d;
  edge_point_hb(c->P, M.ht.hb.data(), M.ht.hb.data() + M.ht.n, M.ht.n, hbq_d);
  const std::vector<char> hbq = typed(hbq_d);
  cudaStream_t s = c->st;
  int r = 0;
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(M.dt.start), M.ht.start.data(), M.ht.start.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(M.dt.ea), M.ht.ea.data(), M.ht.n * sizeof(int), cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<int *>(M.dt.eb), M.ht.eb.data(), M.ht.n * sizeof(int), cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<uint8_t *>(M.dt.code), M.ht.code.data(), M.ht.n, cudaMemcpyHostToDevice, s), "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<void *>(M.dt.geo), geo.data(), geo.size(), cudaMemcpyHostToDevice, s), "tiles");
  if (M.dt.hbq)
    r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<void *>(M.dt.hbq), hbq.data(), hbq.size(), cudaMemcpyHostToDevice, s),
                  "tiles");
  r |= ctx_cuda(c, cudaMemcpyAsync(const_cast<double *>(M.dt.hb), M.ht.hb.data(), M.ht.hb.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, s), "tiles");
  if (r) return c->sticky;
  if (int e = ctx_cuda(c, cudaStreamSynchronize(s), "tiles sync")) return e;
  M.dt.tile = tile;
  M.dt.ntiles = M.ht.ntiles;
  M.dt.n = M.ht.n;
  return 0;
}

static int configure(dgswem_ctx *c, bool persistent, int block) {
  EnsembleState &E = *c->ens;
  for (EnsMesh &M : E.meshes)
    if (int r = upload_mesh_tiles(c, M, block)) return r;
  build_tiles(c, block);
  E.persistent = persistent;
  E.block = block;
  E.grid = persistent ? grid_for(c, block) : E.n_etile;
  if (persistent && E.grid < 1) return ctx_fail(c, DGSWEM_ECUDA, "ensemble kernel cannot be resident");
  if (int r = upload_tiles(c)) return r;
  return capture_graph(c, persistent ? 1 : 2, block, c->timing);
}

int ensemble_attach(dgswem_ctx *c, void *d_workspace, size_t bytes, void *stream) {
  if (int r = attach_common(c, d_workspace, bytes, stream)) return r;
  EnsembleState &E = *c->ens;
  size_t sz = 0;
  ens_layout(c, c->ws, &sz);
  for (EnsMesh &m : E.meshes) m.dt.tile = 0;
  c->host_keep.clear();
  for (EnsMesh &m : E.meshes)
    if (int r = upload_mesh(c, m.hm, m.dm, m.perm, m.iperm)) return r;
  cudaMemsetAsync(c->err, 0, sizeof(int), c->st);
  if (int r = init_states(c)) return r;
  // per-member time step from its own initial state (after wet/dry)
  for (size_t i = 0; i < E.mem.size(); ++i) {
    EnsMember &mb = E.mem[i];
    if (mb.prm.dt > 0) {
      mb.dt = mb.prm.dt;
      continue;
    }
    launch_dt(c->P, E.meshes[mb.mesh].dm, mb.U0, mb.ph, E.dtbits + i, c->st);
  }
  std::vector<unsigned long long> bits(E.mem.size());
  if (int r = ctx_cuda(c, cudaMemcpyAsync(bits.data(), E.dtbits, bits.size() * 8, cudaMemcpyDeviceToHost, c->st),
                       "dt readback"))
    return r;
  if (int r = ctx_cuda(c, cudaStreamSynchronize(c->st), "dt sync")) return r;
  for (size_t i = 0; i < E.mem.size(); ++i) {
    EnsMember &mb = E.mem[i];
    if (mb.prm.dt > 0) continue;
    double best;
    std::memcpy(&best, &bits[i], 8);
    if (!(best > 0) || !std::isfinite(best)) return ctx_fail(c, DGSWEM_EINVAL, "member without a positive wave speed");
    mb.dt = mb.prm.cfl * 3.0 / (2.0 * c->P + 1.0) * best;
  }
  c->dt = E.mem[0].dt;
  c->attached = true;
  // autotune: one persistent launch vs one launch per phase, and the element tile (block) size
  std::vector<int> blocks = c->tun.block ? std::vector<int>{c->tun.block} : std::vector<int>{64, 128, 256};
  std::vector<bool> modes;
  if (c->tun.variant == DGSWEM_ENSEMBLE_PERSISTENT) modes = {true};
  else if (c->tun.variant == DGSWEM_ENSEMBLE_PHASED) modes = {false};
  else modes = {true, false};
  bool best_mode = modes[0];
  int best_block = blocks[0];
  if (modes.size() * blocks.size() > 1) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = INFINITY;
    for (bool mode : modes)
      for (int b : blocks) {
        if (int r = configure(c, mode, b)) return r;
        cudaGraphLaunch(c->exec, c->st);
        // best of two batches of three steps (a step of a large ensemble is milliseconds long)
        const int reps = 3;
        float ms = INFINITY;
        for (int k = 0; k < 2; ++k) {
          cudaEventRecord(e0, c->st);
          for (int i = 0; i < reps; ++i) cudaGraphLaunch(c->exec, c->st);
          cudaEventRecord(e1, c->st);
          if (int r = ctx_cuda(c, cudaEventSynchronize(e1), "ensemble tune")) return r;
          float t = 0;
          cudaEventElapsedTime(&t, e0, e1);
          ms = std::min(ms, t);
        }
        E.tune.push_back({mode ? 1 : 2, b, ms / reps});
        if (ms < best) {
          best = ms;
          best_mode = mode;
          best_block = b;
        }
        if (int r = read_error_word(c)) return r;
        if (int r = init_states(c)) return r;
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (int r = configure(c, best_mode, best_block)) return r;
  if (int r = init_states(c)) return r;
  return read_error_word(c);
}

const std::vector<TuneEntry> &ensemble_tune_log(dgswem_ctx *c) { return c->ens->tune; }

void ensemble_release(dgswem_ctx *c) {
  delete c->ens;
  c->ens = nullptr;
}

extern "C" {

int dgswem_ensemble_create(int32_t n, const dgswem_mesh *const *meshes, const double *const *bathy,
                           const dgswem_params *params, const dgswem_init *inits, const dgswem_tuning *tuning,
                           dgswem_ctx **out) {
  if (!out) return DGSWEM_EINVAL;
  *out = nullptr;
  if (n < 1 || !meshes || !bathy || !params) return DGSWEM_EINVAL;
  std::string msg;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i] || !bathy[i]) return DGSWEM_EINVAL;
    if (check_params(&params[i], msg)) return DGSWEM_EINVAL;
    if (params[i].p != params[0].p || params[i].precision != params[0].precision) return DGSWEM_EINVAL;
    if (params[i].rk_scheme != params[0].rk_scheme) return DGSWEM_EINVAL;
    if (params[i].rk_scheme == DGSWEM_RK_CUSTOM &&
        (params[i].rk_stages != params[0].rk_stages ||
         std::memcmp(params[i].rk_coeffs, params[0].rk_coeffs, sizeof(params[0].rk_coeffs)) != 0))
      return DGSWEM_EINVAL;
  }
  dgswem_ctx *c = new dgswem_ctx();
  c->ensemble = true;
  c->prm = params[0];
  if (tuning) c->tun = *tuning;
  if ((c->tun.block != 0 && c->tun.block != 64 && c->tun.block != 128 && c->tun.block != 256) ||
      c->tun.variant < 0 || c->tun.variant > 2) {
    delete c;
    return DGSWEM_EINVAL;
  }
  c->P = params[0].p;
  c->ND = nd_of(c->P);
  c->mixed = params[0].precision == DGSWEM_FP32_MIXED;
  c->nst = rk_stage_table(params[0], c->ra, c->rb, c->rc, c->rtau);
  c->ens = new EnsembleState();
  EnsembleState &E = *c->ens;
  for (int i = 0; i < n; ++i) {
    int mi = -1;
    for (size_t j = 0; j < E.meshes.size(); ++j)
      if (E.meshes[j].key_mesh == meshes[i] && E.meshes[j].key_bathy == bathy[i]) mi = (int)j;
    if (mi < 0) {
      EnsMesh M;
      M.key_mesh = meshes[i];
      M.key_bathy = bathy[i];
      const int r = preprocess_mesh(*meshes[i], bathy[i], c->tun.reorder != 2, M.hm, msg);
      if (r) {
        delete c->ens;
        delete c;
        return r;
      }
      E.meshes.push_back(std::move(M));
      mi = (int)E.meshes.size() - 1;
    }
    EnsMember mb;
    mb.mesh = mi;
    mb.prm = params[i];
    mb.ph = make_phys(params[i]);
    const HostMesh &H = E.meshes[mi].hm;
    const dgswem_init *ini = inits ? &inits[i] : nullptr;
    mb.t0 = ini ? ini->t0 : 0.0;
    if (ini && ini->modal) {
      mb.init_kind = 1;
      const size_t rows = 3 * (size_t)c->ND;
      mb.init_modal.resize(rows * H.ne);
      for (size_t row = 0; row < rows; ++row)
        for (int e = 0; e < H.ne; ++e) mb.init_modal[row * H.ne + e] = ini->modal[row * H.ne + H.perm[e]];
    } else if (ini && ini->nodal) {
      mb.init_kind = 2;
      mb.init_nodal.assign(ini->nodal, ini->nodal + 3 * (size_t)H.nn);
    }
    E.mem.push_back(std::move(mb));
  }
  // tile lists are sized for the smallest tile (64)
  E.max_etile = E.max_ntile = 0;
  for (const EnsMember &mb : E.mem) {
    const HostMesh &H = E.meshes[mb.mesh].hm;
    E.max_etile += (H.ne + 63) / 64;
    if (mb.ph.hurricane) E.max_ntile += (H.nn + 63) / 64;
  }
  ens_layout(c, nullptr, &c->need);
  *out = c;
  return 0;
}

int dgswem_ensemble_step(dgswem_ctx *c, int32_t n) {
  if (!c || !c->ensemble) return DGSWEM_EINVAL;
  return dgswem_step(c, n);
}

int dgswem_ensemble_get_state(dgswem_ctx *c, int32_t member, double *hz, double *hqx, double *hqy) {
  if (!c || !c->ensemble) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  EnsembleState &E = *c->ens;
  if (member < 0 || member >= (int)E.mem.size()) return DGSWEM_EINVAL;
  const EnsMember &mb = E.mem[member];
  const EnsMesh &M = E.meshes[mb.mesh];
  const int ne = M.hm.ne, ND = c->ND;
  launch_permute(mb.U0, c->staging, M.iperm, 3 * ND, ne, c->st);
  double *dst[3] = {hz, hqx, hqy};
  for (int v = 0; v < 3; ++v)
    if (dst[v])
      if (int r = ctx_cuda(c, cudaMemcpyAsync(dst[v], c->staging + (size_t)v * ND * ne, (size_t)ND * ne * sizeof(double),
                                              cudaMemcpyDeviceToHost, c->st), "member readback"))
        return r;
  return read_error_word(c);
}

int dgswem_ensemble_get_flags(dgswem_ctx *c, int32_t member, uint8_t *h) {
  if (!c || !c->ensemble || !h) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  EnsembleState &E = *c->ens;
  if (member < 0 || member >= (int)E.mem.size()) return DGSWEM_EINVAL;
  const EnsMember &mb = E.mem[member];
  const EnsMesh &M = E.meshes[mb.mesh];
  uint8_t *stage = reinterpret_cast<uint8_t *>(c->staging);  // at least ne bytes
  launch_permute_u8(mb.wd, stage, M.iperm, M.hm.ne, c->st);
  if (int r = ctx_cuda(c, cudaMemcpyAsync(h, stage, M.hm.ne, cudaMemcpyDeviceToHost, c->st), "member flags readback"))
    return r;
  return read_error_word(c);
}

int dgswem_ensemble_info(dgswem_ctx *c, int32_t member, double *dt, double *t, int64_t *steps) {
  if (!c || !c->ensemble) return DGSWEM_EINVAL;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  EnsembleState &E = *c->ens;
  if (member < 0 || member >= (int)E.mem.size()) return DGSWEM_EINVAL;
  const EnsMember &mb = E.mem[member];
  if (dt) *dt = mb.dt;
  if (t) *t = mb.t0 + (double)c->steps_done * mb.dt;
  if (steps) *steps = c->steps_done;
  return 0;
}

int dgswem_ensemble_set_fault(dgswem_ctx *c, int32_t skip_arrival) {
  if (!c || !c->ensemble) return DGSWEM_EINVAL;
  if (c->sticky) return c->sticky;
  if (!c->attached) return ctx_fail(c, DGSWEM_ESTATE, "not attached");
  if (int r = ctx_cuda(c, cudaStreamSynchronize(c->st), "sync")) return r;
  c->ens->fault = skip_arrival ? 1 : 0;
  if (skip_arrival && !c->ens->persistent)
    return ctx_fail(c, DGSWEM_EINVAL, "the fault hook needs the persistent launch (no barriers otherwise)");
  return capture_graph(c, c->ens->persistent ? 1 : 2, c->ens->block, c->timing);
}

}  // extern "C"
