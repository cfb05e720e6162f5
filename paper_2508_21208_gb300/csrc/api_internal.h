// api_internal.h -- the context behind the opaque dgswem_ctx handle.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

struct TuneEntry {
  int variant, block;
  float ms_per_step;
};

struct EnsembleState;  // ensemble.cu

// Carves aligned sub-buffers out of one workspace (or only measures, when base is null).
struct Carver {
  char *base;
  size_t off = 0;
  template <class X>
  X *take(size_t count) {
    off = (off + 255) / 256 * 256;
    X *p = base ? reinterpret_cast<X *>(base + off) : nullptr;
    off += (count > 0 ? count : 1) * sizeof(X);
    return p;
  }
};

struct dgswem_ctx {
  bool ensemble = false;
  dgswem_params prm{};
  dgswem_tuning tun{};
  int P = 1, ND = 3;
  bool mixed = false;
  dg::HostMesh hm;
  int init_kind = 0;  // 0 rest, 1 modal, 2 nodal
  std::vector<double> init_modal, init_nodal;
  double t0 = 0.0, dt = 0.0;
  double graph_t0 = 0.0;  // the t0 baked into the captured step graph
  int64_t steps_done = 0;
  int nst = 2;  // Runge-Kutta stages
  double ra[dg::MAX_STAGES] = {}, rb[dg::MAX_STAGES] = {}, rc[dg::MAX_STAGES] = {}, rtau[dg::MAX_STAGES] = {};
  // device side
  size_t need = 0, ws_bytes = 0;
  char *ws = nullptr;
  cudaStream_t st = nullptr, own_stream = nullptr;
  bool attached = false;
  dg::DevMesh dm{};
  dg::DevTiles tiles{};     // tile edge lists of the tiled variant (tile size tiles.tile, 0 = none)
  dg::TileEdges htiles;
  dg::Phys ph{};
  int *d_perm = nullptr, *d_iperm = nullptr;
  double *U0 = nullptr, *U1 = nullptr, *U2 = nullptr, *partial = nullptr, *result = nullptr, *staging = nullptr;
  void *mean = nullptr;  // T [3][ne] element means for the limiter
  uint8_t *cls = nullptr;     // [ne] wetting/drying front class (float form)
  double *mean64 = nullptr;   // [3][ne] the front elements' means in double (float form)
  int *flist = nullptr;       // [ne] front list (float form)
  unsigned *fcnt = nullptr;   // [MAX_STAGES] front list counters, one per stage
  uint8_t *wd = nullptr, *wd_stage = nullptr, *emode = nullptr;
  void *eflux = nullptr, *frc = nullptr;
  long long *step = nullptr;
  int *err = nullptr;
  unsigned long long *dtbits = nullptr;
  void *h_pinned = nullptr;
  int *h_err = nullptr;
  double *h_res = nullptr;
  std::vector<std::vector<char>> host_keep;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_step = 0, variant = 0, block = 128;
  bool timing = false;
  // the same configuration captured in the other timing mode, kept so that switching is free
  cudaGraph_t graph_alt = nullptr;
  cudaGraphExec_t exec_alt = nullptr;
  bool alt_timing = false;
  std::vector<cudaEvent_t> ev;
  std::vector<const char *> knames;
  std::vector<TuneEntry> tune_log;
  // a part of a partitioned domain (dgswem_create_part): halo lists in internal element order,
  // their device copies, the caller's packed buffers and the stage in progress
  bool part = false;
  std::vector<int> halo_send, halo_recv;
  int *d_send_idx = nullptr, *d_recv_idx = nullptr;
  double *d_send_buf = nullptr, *d_recv_buf = nullptr;
  int stage_i = 0;
  bool stage_open = false;
  // errors
  int sticky = 0;
  std::string errmsg;
  // ensemble
  EnsembleState *ens = nullptr;
};

int ctx_fail(dgswem_ctx *c, int code, const std::string &msg);
int ctx_cuda(dgswem_ctx *c, cudaError_t e, const char *what);
int check_params(const dgswem_params *p, std::string &msg);
dg::Phys make_phys(const dgswem_params &p);
void upload_all_tables();
int read_error_word(dgswem_ctx *c);
int attach_common(dgswem_ctx *c, void *d_workspace, size_t bytes, void *stream);
int capture_graph(dgswem_ctx *c, int variant, int block, bool timing);
void carve_mesh(Carver &k, const dg::HostMesh &H, int p, bool mixed, dg::DevMesh &m, int **perm,
                int **iperm);
int upload_mesh(dgswem_ctx *c, const dg::HostMesh &H, const dg::DevMesh &m, int *perm, int *iperm);
// ensemble.cu
int ensemble_attach(dgswem_ctx *c, void *d_workspace, size_t bytes, void *stream);
void ensemble_enqueue_step(dgswem_ctx *c, std::vector<const char *> *names);
void ensemble_release(dgswem_ctx *c);
const std::vector<TuneEntry> &ensemble_tune_log(dgswem_ctx *c);
