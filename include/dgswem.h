/*
 * dgswem.h -- C ABI of the GB300 DG-SWEM hot path (libdgswem.so).
 *
 * The library advances the p-th order modal discontinuous Galerkin discretisation of the 2D
 * shallow water equations (Wichitrnithed et al., arXiv 2508.21208, Sec. 2.1 Eq. SWE and
 * Sec. 2.2 Eq. elem_weak_form / Eq. RKSSP) on an unstructured triangle mesh on one GPU:
 * area integrals of flux and sources (Alg. 1), interior, land, open-ocean and river edge fluxes
 * (Alg. 2, Alg. 3; LLF or Roe), the inverse (diagonal) mass matrix and the SSP-RK stage update
 * (SSP-RK2 by default), the slope
 * limiter and the wetting/drying treatment (Sec. 5.2.3 SLOPELIM, WETDRY), and nodal wind /
 * pressure forcing (Sec. 5.2.3 WIND).  Every step runs in CUDA kernels built for sm_103a; there
 * is no CPU fallback.  Host code only preprocesses the mesh (edge list, neighbour maps, limiter
 * geometry, locality reordering) and marshals arguments.
 *
 * Conventions (all entry points):
 *  - Return 0 on success or a negative DGSWEM_E* code.  Errors are sticky per context; the text
 *    of the first one is available from dgswem_last_error().  The exception is a query the
 *    context's mode cannot answer (dgswem_kernel_times with timing off): DGSWEM_ESTATE, not
 *    sticky.
 *  - Pointers named h_* / plain const pointers are HOST memory owned by the caller and only read
 *    during the call (create deep-copies them).  The one device buffer the library uses is the
 *    workspace the caller attaches (dgswem_attach); the library allocates no device memory.
 *  - Modal state arrays are [ndof][n_elems] per variable (zeta, q_x = H u_x, q_y = H u_y),
 *    modes in the order (0,0), (1,0), (0,1), (2,0), (1,1), (0,2) of the Dubiner basis
 *    (Sec. 2.2, Eq. dubiner), elements in the caller's original order.  Mode (0,0) is the
 *    element mean.  ndof = 3 at p = 1 and 6 at p = 2.
 *  - Work is issued asynchronously on the CUDA stream given to dgswem_attach; calls that return
 *    data to the host synchronise that stream.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef DGSWEM_H
#define DGSWEM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DGSWEM_API __attribute__((visibility("default")))
#else
#define DGSWEM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DGSWEM_OK 0
#define DGSWEM_EINVAL -1     /* bad argument or parameter value */
#define DGSWEM_EMESH -2      /* invalid mesh: index out of range, clockwise or degenerate
                                triangle, edge shared by more than two triangles or by two
                                triangles with the same orientation, boundary edge list entry
                                that is not a boundary edge */
#define DGSWEM_ECUDA -3      /* a CUDA runtime call failed */
#define DGSWEM_ENONFINITE -4 /* a NaN or Inf appeared in the state */
#define DGSWEM_ENEGDEPTH -5  /* an element mean depth became negative after wetting/drying */
#define DGSWEM_ETIMEOUT -6   /* a bounded device-side wait gave up (ensemble grid barrier) */
#define DGSWEM_ENOMEM -7     /* the attached workspace is smaller than dgswem_workspace_size */
#define DGSWEM_ESTATE -8     /* call out of order (e.g. step before attach) */
#define DGSWEM_ETOOBIG -9    /* input larger than a fixed-size library buffer allows */

/* boundary edge types (Sec. 2.1: Gamma_land, Gamma_ocean) */
#define DGSWEM_BC_LAND 0 /* no normal flow: mirror ghost state */
#define DGSWEM_BC_OPEN 1 /* elevation-specified (tidal) boundary, momentum from the interior */
#define DGSWEM_BC_RIVER 2 /* river inflow (Gamma_river): the land mirror ghost shifted so that the
                             mean normal discharge of the two traces is -river_q (inflow) */

/* arithmetic forms */
#define DGSWEM_FP64 0       /* every step in IEEE double */
#define DGSWEM_FP32_MIXED 1 /* volume, edge and source arithmetic in float; RK state, the RK
                               update, the mass sum and the wet/dry depth tests in double */

/* bottom friction tau_b (Eq. SWE) */
#define DGSWEM_FRICTION_NONE 0
#define DGSWEM_FRICTION_MANNING 1   /* tau_b = g n^2 |q| / H^(7/3) */
#define DGSWEM_FRICTION_QUADRATIC 2 /* tau_b = C_f |q| / H^2 */

/* kernel organisation of one RK stage (chosen by the autotuner when 0) */
#define DGSWEM_VARIANT_AUTO 0
#define DGSWEM_VARIANT_SPLIT 1 /* edge kernel stores each interior edge flux once, the element
                                  kernel gathers it (the paper's Alg. 2 + Alg. 3 organisation,
                                  atomic-free) */
#define DGSWEM_VARIANT_FUSED 2 /* one element kernel computes its own edge fluxes from its
                                  neighbours' states (no flux scratch, edge work done twice) */
#define DGSWEM_VARIANT_TILED 3 /* one block per tile of consecutive elements: the tile's states
                                  are staged in shared memory, every edge touching the tile is
                                  computed once by the block (edges between tiles by both), then
                                  each thread finishes its element (no flux scratch in HBM) */
#define DGSWEM_VARIANT_TILED_WIDE 4 /* TILED with a tighter register bound in the FP32-mixed form
                                       at p = 1 (5 instead of 4 resident 256-thread blocks per
                                       SM): better on large meshes; identical to TILED otherwise */

typedef struct dgswem_ctx dgswem_ctx; /* opaque, library-owned */

/* Triangle mesh.  xy: [n_nodes][2] metres; tri: [n_elems][3] node indices, counter-clockwise,
 * 0-based; bedge: [n_bedges][2] node pairs of boundary edges with bedge_type[n_bedges]
 * (DGSWEM_BC_*).  Boundary edges absent from bedge are land. */
typedef struct {
  int32_t n_nodes, n_elems, n_bedges;
  const double *xy;
  const int32_t *tri;
  const int32_t *bedge;
  const int32_t *bedge_type;
} dgswem_mesh;

/* Model and numerics parameters (SI units). */
typedef struct {
  int32_t p;         /* polynomial degree: 1 or 2 (Sec. 2.2, Eq. dubiner) */
  int32_t precision; /* DGSWEM_FP64 or DGSWEM_FP32_MIXED */
  double g;          /* gravity */
  double cfl;        /* dt = cfl * 3/(2p+1) * min_e r_e / lambda_e (r_e inradius) unless dt > 0 */
  double dt;         /* > 0: fixed time step overriding cfl; 0: from cfl; < 0: DGSWEM_EINVAL */
  double h0;         /* wetting/drying minimum depth; 0 disables wetting/drying */
  int32_t friction;  /* DGSWEM_FRICTION_* */
  double manning_n, cf;
  int32_t limiter;   /* 1: Cockburn-Shu minmod slope limiter after each stage */
  int32_t coriolis;  /* 1: f = 2 Omega sin(latitude) Coriolis source */
  double coriolis_lat_deg;
  double tide_amp, tide_period, tide_phase; /* open boundary zeta = A sin(2 pi t / T + phase) */
  int32_t hurricane; /* 1: Holland vortex wind stress and pressure gradient */
  double pc_hpa, pn_hpa, rmax_m, holland_b, vt_ms, track_x0, track_y0, track_heading;
  double rho_air, rho_water;
  int32_t rk_scheme;     /* DGSWEM_RK_* (0 = SSP(2,2)) */
  int32_t rk_stages;     /* DGSWEM_RK_CUSTOM: number of stages s, 2 <= s <= 8 */
  double rk_coeffs[24];  /* DGSWEM_RK_CUSTOM: (a_i, b_i, c_i) for i = 1..s, see below */
  int32_t flux;          /* numerical flux F^ of Eq. elem_weak_form: DGSWEM_FLUX_LLF or _ROE */
  double rain_rate;      /* R of Eq. SWE: uniform rain rate (m/s) */
  double river_q;        /* inflow discharge per unit width on DGSWEM_BC_RIVER edges (m^2/s) */
} dgswem_params;

/* numerical fluxes (Sec. 2.2 names local Lax-Friedrichs and Roe as choices for F^) */
#define DGSWEM_FLUX_LLF 0 /* local Lax-Friedrichs, lambda = max(|u.n| + sqrt(gH)) of the two traces */
#define DGSWEM_FLUX_ROE 1 /* Roe (1981): Roe-averaged |A| in the edge frame, Harten entropy fix
                             (delta = c~/10) on the two acoustic waves */

/* SSP Runge-Kutta schemes in the two-register Shu-Osher form (Sec. 2.2: the paper uses SSPRK
 * schemes optimised for DG, Kubatko et al. 2014): u^(0) = u^n,
 * u^(i) = a_i u^n + b_i u^(i-1) + c_i dt L(u^(i-1)), i = 1..s, u^(n+1) = u^(s); the limiter and
 * wet/dry run after every stage; stage i sees boundary data and forcing at t_n + tau_(i-1) dt with
 * tau_0 = 0, tau_i = b_i tau_(i-1) + c_i.  Any scheme of this form (e.g. DG-optimised
 * coefficients) can be given as DGSWEM_RK_CUSTOM.  The CFL number is not rescaled: choose cfl
 * (or dt) for the scheme's stability region. */
#define DGSWEM_RK_SSP22 0  /* Shu-Osher SSP(2,2) */
#define DGSWEM_RK_SSP33 1  /* Shu-Osher SSP(3,3) */
#define DGSWEM_RK_SSP32 2  /* SSP(3,2): s-1 Euler steps of dt/(s-1), then the average (Ketcheson 2008) */
#define DGSWEM_RK_SSP42 3  /* SSP(4,2), same family */
#define DGSWEM_RK_SSP52 4  /* SSP(5,2), same family */
#define DGSWEM_RK_SSP43 5  /* SSP(4,3) (Spiteri & Ruuth 2002) */
#define DGSWEM_RK_CUSTOM 6

/* Tuning knobs; pass NULL to dgswem_create for the defaults (all zero = automatic). */
typedef struct {
  int32_t variant;   /* DGSWEM_VARIANT_* */
  int32_t block;     /* threads per block of the element kernels (= elements per tile for the
                        tiled variant): 0 (auto), 64, 128, 256 */
  int32_t reorder;   /* 0: auto (Hilbert order on), 1: Hilbert curve order, 2: keep caller order */
  int32_t autotune;  /* 1: time the candidate variants / block sizes at attach and keep the best */
} dgswem_tuning;

/* Initial state: modal ([3][ndof][n_elems], caller order) or nodal ([3][n_nodes]: the linear
 * interpolant in each element); both NULL = lake at rest (zeta = q = 0).  t0 is the start time. */
typedef struct {
  const double *modal;
  const double *nodal;
  double t0;
} dgswem_init;

/* Validate the mesh and parameters, preprocess the mesh on the host (edge list, neighbour and
 * element-to-edge maps, boundary tags, limiter geometry, Hilbert-order relabelling) and keep a
 * private copy of everything.  No device work happens here.  bathy: [n_nodes] h_b, positive
 * downward (Sec. 2.1), linear within each element.  tuning may be NULL.
 * Errors: DGSWEM_EINVAL, DGSWEM_EMESH; *out is set to NULL on error. */
DGSWEM_API int dgswem_create(const dgswem_mesh *mesh, const double *bathy, const dgswem_params *params,
                  const dgswem_init *init, const dgswem_tuning *tuning, dgswem_ctx **out);

/* Bytes of device workspace (256-byte aligned) that dgswem_attach needs.  No paper passage: the
 * paper keeps its arrays in unified memory (Sec. 5.1); this library instead lets the caller
 * provide one explicit device buffer.  Errors: DGSWEM_EINVAL (null argument). */
DGSWEM_API int dgswem_workspace_size(const dgswem_ctx *ctx, size_t *bytes);

/* Bind a caller-owned device buffer of at least dgswem_workspace_size bytes (the caller keeps
 * ownership and must keep it alive until dgswem_destroy) and a CUDA stream (cudaStream_t passed
 * as void*; NULL = a private non-blocking stream the library creates).  Uploads the static mesh
 * data and the initial state,
 * applies the wetting/drying operator to the initial state, computes dt when params->dt <= 0,
 * autotunes if asked, and captures one time step as a CUDA graph.  Synchronises the stream.
 * Replaces the paper's unified-memory placement and prefetching (Sec. 5.1, Sec. 5.2.4) with one
 * upload; the time step follows Sec. 6.1, which runs a fixed dt for the whole simulation.
 * Errors: DGSWEM_ENOMEM (buffer null or smaller than dgswem_workspace_size, checked before any
 * device work), DGSWEM_EINVAL (buffer not 256-byte aligned), DGSWEM_ECUDA, DGSWEM_ESTATE (already
 * attached). */
DGSWEM_API int dgswem_attach(dgswem_ctx *ctx, void *d_workspace, size_t bytes, void *stream);

/* Advance n_steps time steps of the chosen SSP-RK scheme (Sec. 2.2 Eq. RKSSP; SSP-RK2 by
 * default) by replaying the captured graph.  Asynchronous: device-side errors (DGSWEM_ENONFINITE, DGSWEM_ENEGDEPTH) are
 * reported by the next synchronising call. */
DGSWEM_API int dgswem_step(dgswem_ctx *ctx, int32_t n_steps);

/* Copy the modal state to caller-owned host arrays, each [ndof][n_elems] in the caller's
 * element order: the Dubiner coefficients of zeta, q_x and q_y (Sec. 2.2, Eq. dubiner; the
 * unknowns of the weak form Eq. elem_weak_form).  Any of the three pointers may be NULL.
 * Synchronises.  Errors: DGSWEM_ESTATE (not attached), DGSWEM_ECUDA, or a sticky device error. */
DGSWEM_API int dgswem_get_state(dgswem_ctx *ctx, double *h_zeta, double *h_qx, double *h_qy);

/* Replace the modal state (caller order, same layout as dgswem_get_state: the Dubiner
 * coefficients of Sec. 2.2, Eq. dubiner) and set the time to t (the step counter restarts at 0).
 * Wet/dry flags are recomputed from the new state (classification of Sec. 5.2.3 WETDRY, state
 * unchanged).  The copies are asynchronous; the host arrays must stay valid until the next
 * synchronising call.  Errors: DGSWEM_EINVAL (null pointer, non-finite t), DGSWEM_ESTATE. */
DGSWEM_API int dgswem_set_state(dgswem_ctx *ctx, const double *h_zeta, const double *h_qx,
                     const double *h_qy, double t);

/* Total surface anomaly volume sum_e |Omega_e| zeta_e,00 and water volume
 * sum_e |Omega_e| (zeta_e,00 + mean h_b), each a compensated (Neumaier) double sum in a fixed
 * block order, hence bitwise reproducible.  No paper passage defines it: it is this library's
 * conservation diagnostic for the continuity equation of Eq. SWE (with mode (0,0) the element
 * mean, the discrete volume is exactly this sum).  Synchronises.  Errors: DGSWEM_EINVAL (null
 * pointer), DGSWEM_ESTATE, DGSWEM_ECUDA, or a sticky device error. */
DGSWEM_API int dgswem_mass(dgswem_ctx *ctx, double *mass_zeta, double *volume);

/* Time step, current time t0 + steps*dt, and steps done since create / set_state.  The step is
 * fixed for the run, as the paper's runs use one fixed dt (Sec. 6.1).  Any pointer may be NULL.
 * Errors: DGSWEM_ESTATE (not attached). */
DGSWEM_API int dgswem_info(dgswem_ctx *ctx, double *dt, double *t, int64_t *steps_done);

/* Wait for the stream and surface any device-side error (no paper passage: the host-side
 * counterpart of the paper's `!$acc wait`, Sec. 5.3).  Errors: the sticky error, DGSWEM_ESTATE. */
DGSWEM_API int dgswem_sync(dgswem_ctx *ctx);

/* Per-element wet/dry flags (0 wet, 1 partially wet, 2 dry), caller order: the element states of
 * the wetting/drying treatment (Sec. 5.2.3 WETDRY).  Synchronises.  Errors: DGSWEM_EINVAL (null
 * pointer or an ensemble context: see dgswem_ensemble_get_flags), DGSWEM_ESTATE. */
DGSWEM_API int dgswem_get_flags(dgswem_ctx *ctx, uint8_t *h_flags);

/* Release the context (after synchronising its stream).  The caller's workspace and stream stay
 * the caller's.  No paper passage. */
DGSWEM_API void dgswem_destroy(dgswem_ctx *ctx);
/* Text of the context's first error ("" if none; "null context" for NULL).  No paper passage. */
DGSWEM_API const char *dgswem_last_error(const dgswem_ctx *ctx);

/* ---- single operators, for checking each step of the path against a reference ----
 * Each runs the named kernel(s) once on the current state, on the context's stream, then
 * synchronises. */

/* L_h(u) of Eq. RKSSP at time t (area integrals of Alg. 1, edge fluxes of Alg. 2 gathered as in
 * Alg. 3, inverse mass matrix; no limiter, no wet/dry), written to h_out as [3][ndof][n_elems] in
 * caller order.  In the FP32-mixed form the elements at the wetting/drying front take the double
 * path, as in a step. */
DGSWEM_API int dgswem_eval_rhs(dgswem_ctx *ctx, double t, double *h_out);
/* Apply the slope limiter (Sec. 2.2, where limiting is optional; kernel SLOPELIM of Sec. 5.2.3) to
 * the current state in place, every element in the form's own arithmetic. */
DGSWEM_API int dgswem_apply_limiter(dgswem_ctx *ctx);
/* Apply the wetting/drying operator (kernel WETDRY of Sec. 5.2.3) to the current state in place.
 * DGSWEM_EINVAL when wetting/drying is off (h0 = 0). */
DGSWEM_API int dgswem_apply_wetdry(dgswem_ctx *ctx);
/* Nodal forcing (WIND) at time t: h_out [3][n_nodes] = (tau_x/rho_w, tau_y/rho_w,
 * (p_a - p_n)/rho_w); the pressure anomaly, since only its gradient enters Eq. SWE. */
DGSWEM_API int dgswem_eval_forcing(dgswem_ctx *ctx, double t, double *h_out);

/* ---- kernel timing (no paper passage: the per-kernel times behind Sec. 6.2's breakdown) ----
 * With timing on, dgswem_step replays a graph of the same step with event-record nodes between
 * its kernels (captured on first use; both graphs are kept, so switching back and forth costs a
 * stream synchronisation only).  dgswem_kernel_times then returns, for the last replayed step,
 * each kernel's duration in milliseconds and its name (static strings), in launch order;
 * n_kernels gets the count.  The event nodes lengthen a step by a few microseconds, so a caller
 * timing whole steps turns timing on only for the steps whose kernel times it reads. */
DGSWEM_API int dgswem_set_kernel_timing(dgswem_ctx *ctx, int32_t on);
DGSWEM_API int dgswem_kernel_times(dgswem_ctx *ctx, float *ms, const char **names, int32_t capacity,
                        int32_t *n_kernels);
/* Kernel launches per time step in the captured graph, and the chosen variant / block size (no
 * paper passage).  Any pointer may be NULL.  Errors: DGSWEM_ESTATE (not attached). */
DGSWEM_API int dgswem_graph_info(dgswem_ctx *ctx, int32_t *kernels_per_step, int32_t *variant,
                      int32_t *block);

/* No paper passage.  The autotuner's measurements at attach: for each timed candidate its variant (single model:
 * DGSWEM_VARIANT_*; ensemble: DGSWEM_ENSEMBLE_*), block / tile size and milliseconds per step.
 * n_entries gets the count (0 when a fixed configuration was requested). */
DGSWEM_API int dgswem_tune_log(dgswem_ctx *ctx, int32_t *variant, int32_t *block, float *ms_per_step,
                               int32_t capacity, int32_t *n_entries);

/* ---- batched ensemble (several scenarios, meshes of uneven size) ----
 * n members; member i uses meshes[i], bathy[i], params[i] and inits[i] (inits may be NULL).
 * Members that pass the same mesh and bathymetry pointers share one copy of the static mesh
 * data.  All members must use the same p and precision; each has its own CFL time step, forcing
 * and wet/dry state.  A step advances every member by one of its own time steps, either in one
 * persistent cooperative kernel launch (forcing, element update and limiter/wet-dry phases over a
 * flat list of (member, element tile) work items, separated by grid barriers whose waits are
 * bounded in time) or in one launch per phase; the step is captured in a CUDA graph.  For an
 * ensemble, tuning->variant selects DGSWEM_ENSEMBLE_PERSISTENT or DGSWEM_ENSEMBLE_PHASED (0:
 * the autotuner times both), tuning->block the tile size (0: timed among 64, 128, 256).  The
 * element update always computes its own edge fluxes (the fused organisation).  dgswem_step,
 * dgswem_sync, dgswem_set_kernel_timing, dgswem_kernel_times, dgswem_graph_info,
 * dgswem_workspace_size, dgswem_attach and dgswem_destroy apply to an ensemble context. */
#define DGSWEM_ENSEMBLE_PERSISTENT 1
#define DGSWEM_ENSEMBLE_PHASED 2
DGSWEM_API int dgswem_ensemble_create(int32_t n, const dgswem_mesh *const *meshes,
                           const double *const *bathy, const dgswem_params *params,
                           const dgswem_init *inits, const dgswem_tuning *tuning,
                           dgswem_ctx **out);
/* Advance every member n_steps of its own time step (Sec. 2.2 Eq. RKSSP, as dgswem_step):
 * dgswem_step on an ensemble context (one replay of the captured ensemble step per step), checked
 * to be one.  DGSWEM_EINVAL for a single-model context or n_steps < 0. */
DGSWEM_API int dgswem_ensemble_step(dgswem_ctx *ctx, int32_t n_steps);
/* Member `member`'s modal state (the Dubiner coefficients of Sec. 2.2, Eq. dubiner), laid out as
 * dgswem_get_state in that member's mesh order.  Synchronises.  DGSWEM_EINVAL for a member out of
 * range or a single-model context. */
DGSWEM_API int dgswem_ensemble_get_state(dgswem_ctx *ctx, int32_t member, double *h_zeta, double *h_qx,
                              double *h_qy);
/* Member `member`'s wet/dry flags (0 wet, 1 partially wet, 2 dry; Sec. 5.2.3 WETDRY) in that
 * member's mesh order, as dgswem_get_flags.  Synchronises.  DGSWEM_EINVAL for a null pointer, a
 * member out of range or a single-model context. */
DGSWEM_API int dgswem_ensemble_get_flags(dgswem_ctx *ctx, int32_t member, uint8_t *h_flags);
/* Member `member`'s fixed time step (Sec. 6.1), time and steps done; as dgswem_info. */
DGSWEM_API int dgswem_ensemble_info(dgswem_ctx *ctx, int32_t member, double *dt, double *t,
                         int64_t *steps_done);
/* Test hook (no paper passage): when on, one block skips every grid-barrier arrival, so the other
 * blocks' bounded waits expire and the step reports DGSWEM_ETIMEOUT instead of hanging.  Needs the
 * persistent launch (DGSWEM_EINVAL otherwise). */
DGSWEM_API int dgswem_ensemble_set_fault(dgswem_ctx *ctx, int32_t skip_arrival);

/* ---- one model on several GPUs: domain decomposition (Sec. 5.3) ----
 * The paper runs DG-SWEM on several GPUs by splitting the mesh among MPI ranks and exchanging the
 * states of the ghost elements at the part boundaries, packed into contiguous buffers on the GPU
 * (Sec. 5.3, Listings code:mpi and code:pack).  Here a part is one context on one GPU whose
 * sub-mesh holds its own elements and two layers of ghost elements: the part updates its own
 * elements and, redundantly, the first ghost layer (so that every neighbour mean its own elements'
 * limiter needs is local), limits and wets/dries its own elements, and then receives the ghost
 * elements' states and wet/dry flags from their owners, once per Runge-Kutta stage.  Moving the
 * packed bytes between GPUs (NCCL send/recv, MPI, a copy) is the caller's; the library only packs
 * and unpacks.  These host functions allocate nothing and touch no device. */

/* Recursive coordinate bisection: part[e] in [0, n_parts) for every element e (caller order), the
 * parts' element counts proportional to their share of parts at every split (the paper partitions
 * with METIS; this is the geometric stand-in).  Ties in a coordinate go by element index, so the
 * result is deterministic.  Errors: DGSWEM_EINVAL (null pointer, bad mesh indices, n_parts < 1 or
 * above the element count). */
DGSWEM_API int dgswem_partition_rcb(const dgswem_mesh *mesh, int32_t n_parts, int32_t *part);

/* Sizes of part `rank`'s sub-mesh and exchange lists: nodes, elements (own + ghost layers 1 and 2),
 * boundary-edge entries, peers (the other parts it exchanges with) and the total lengths of its
 * send and receive lists. */
typedef struct {
  int32_t n_nodes, n_elems, n_bedges, n_own, n_ghost1, n_ghost2, n_peers, n_send, n_recv;
} dgswem_part_counts;
/* Errors: DGSWEM_EINVAL (null pointer, part entries or rank out of range, empty part),
 * DGSWEM_EMESH (an edge shared by more than two elements, a boundary edge out of range). */
DGSWEM_API int dgswem_part_sizes(const dgswem_mesh *mesh, const int32_t *part, int32_t n_parts, int32_t rank,
                                 dgswem_part_counts *sizes);

/* Caller-owned output arrays of dgswem_part_build, sized by dgswem_part_sizes.  The sub-mesh keeps
 * the global element and node order: element i of the part is global element elem_global[i]
 * (increasing), node j is global node node_global[j] (increasing), so a sub-mesh edge keeps its
 * orientation.  elem_class[i]: 0 own, 1 first ghost layer (shares an edge with an own element),
 * 2 second ghost layer.  bedge / bedge_type: the global boundary-edge entries of the part's
 * elements.  For peer k (peer[k], increasing): send_count[k] own elements that are ghosts of that
 * peer and recv_count[k] ghosts that it owns, concatenated over k in send_elems / recv_elems as
 * part-local element indices, each group in increasing global index, so that this part's send
 * group for q and q's receive group for this part list the same elements in the same order. */
typedef struct {
  double *xy;             /* [n_nodes][2] */
  int32_t *tri;           /* [n_elems][3] */
  int32_t *bedge;         /* [n_bedges][2] (may be NULL when n_bedges = 0) */
  int32_t *bedge_type;    /* [n_bedges] */
  double *bathy;          /* [n_nodes] */
  int32_t *elem_global;   /* [n_elems] */
  int32_t *elem_class;    /* [n_elems] */
  int32_t *node_global;   /* [n_nodes] */
  int32_t *peer, *send_count, *recv_count; /* [n_peers] */
  int32_t *send_elems;    /* [n_send] */
  int32_t *recv_elems;    /* [n_recv] */
} dgswem_part_out;
/* Fill the sub-mesh and exchange lists of part `rank` (errors as dgswem_part_sizes). */
DGSWEM_API int dgswem_part_build(const dgswem_mesh *mesh, const double *bathy, const int32_t *part,
                                 int32_t n_parts, int32_t rank, const dgswem_part_out *out);

/* One part of a partitioned domain: dgswem_create with the sub-mesh of dgswem_part_build (its
 * elements in the sub-mesh order), their classes, and the send / receive lists as sub-mesh element
 * indices in the order of the packed buffers (send: own elements; receive: ghost elements).  The
 * part needs a fixed time step (params->dt > 0: the global one, the same on every part).  The
 * context then updates its own elements and the first ghost layer and limits and wets/dries its own
 * elements; dgswem_mass sums its own elements (the caller adds the parts' sums); the state calls
 * see every sub-mesh element.  A part steps stage by stage (dgswem_stage_compute / _finish), not
 * with dgswem_step (DGSWEM_ESTATE).  Errors: as dgswem_create; DGSWEM_EINVAL also for a missing
 * class array, dt <= 0, or a list entry out of range or of the wrong class. */
typedef struct {
  const int32_t *elem_class;  /* [n_elems]: 0 own, 1 first ghost layer, 2 second */
  int32_t n_send;
  const int32_t *send_elems;  /* [n_send] own elements, in send-buffer order */
  int32_t n_recv;
  const int32_t *recv_elems;  /* [n_recv] ghost elements, in receive-buffer order */
} dgswem_part;
DGSWEM_API int dgswem_create_part(const dgswem_mesh *mesh, const double *bathy, const dgswem_params *params,
                                  const dgswem_init *init, const dgswem_tuning *tuning, const dgswem_part *part,
                                  dgswem_ctx **out);
/* Bytes of the packed send and receive buffers: one record of 3 ndof + 1 doubles per listed element
 * (its modal state, then its wet/dry flag as a double), as in the paper's packElems (Listing
 * code:pack).  DGSWEM_EINVAL for a context that is not a part. */
DGSWEM_API int dgswem_halo_sizes(dgswem_ctx *ctx, size_t *send_bytes, size_t *recv_bytes);
/* Bind caller-owned device buffers of dgswem_halo_sizes bytes (8-byte aligned; the caller keeps
 * them alive, and moves the bytes between parts itself: NCCL send/recv, MPI or copies). */
DGSWEM_API int dgswem_halo_attach(dgswem_ctx *ctx, void *d_send, void *d_recv);
/* One Runge-Kutta stage of a part, in two calls around the caller's exchange (Sec. 5.3, Listing
 * code:mpi: pack, exchange, unpack).  dgswem_stage_compute issues the stage's kernels on the own
 * elements and the first ghost layer (element update, limiter and wet/dry on the own elements) and
 * packs the send list's records into the send buffer; the caller then delivers each peer's packed
 * records into this part's receive buffer, ordered on the context stream; dgswem_stage_finish
 * unpacks them into the ghost elements' states and flags.  After the scheme's last stage the step is
 * complete.  Both calls are asynchronous.  Errors: DGSWEM_ESTATE (not attached, calls out of order,
 * no halo buffers), DGSWEM_EINVAL (not a part). */
DGSWEM_API int dgswem_stage_compute(dgswem_ctx *ctx);
DGSWEM_API int dgswem_stage_finish(dgswem_ctx *ctx);

/* ---- allocation-free mass sums ----
 * The paper has no counterpart: this is a service for callers that may not allocate device
 * memory.  Examples are a host model or coupler that owns the whole GPU memory budget and
 * forbids allocations by the libraries it calls, and a time-critical loop where the implicit
 * synchronisation and possible failure of cudaMalloc are not acceptable.  Such a caller passes
 * only its own device arrays; the library neither allocates nor frees anything.
 *
 * Computes, like dgswem_mass, d_out[0] = sum_e area[e] * zeta00[e] and
 * d_out[1] = sum_e area[e] * (zeta00[e] + hb_mean[e]) as compensated double sums in a fixed
 * block order, from caller-owned device arrays of n_elems doubles (element mean surface, element
 * area, element mean bathymetry); d_out is a caller-owned device array of two doubles.  Work is
 * queued on `stream` (cudaStream_t as void*, NULL = legacy default stream); the call returns
 * without waiting, so read d_out after synchronising that stream.
 *
 * The block partial sums live in one fixed device buffer inside the library, sized for at most
 * DGSWEM_NOALLOC_MAX_ELEMS elements (1 MiB; every GPU that loads the library holds it until the
 * process exits).  Larger n_elems is rejected with DGSWEM_ETOOBIG before any device work;
 * n_elems < 1 or a NULL pointer gives DGSWEM_EINVAL.  The first call on each device looks up the
 * buffer's device address (that device must be current), so make the first call before any
 * stream capture.  The address is kept for the life of the process, which assumes that the
 * device's primary context is not reset (cudaDeviceReset) or destroyed meanwhile.  All calls share the buffer: calls that can overlap on the GPU (different
 * streams, or different host threads) race and must be serialised by the caller.  Each call
 * overwrites every partial it reads, so no state carries over from a previous call. */
#define DGSWEM_NOALLOC_MAX_ELEMS (1 << 26)
DGSWEM_API int dgswem_mass_noalloc(const double *d_zeta00, const double *d_area,
                                   const double *d_hb_mean, int32_t n_elems, double *d_out,
                                   void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DGSWEM_H */
