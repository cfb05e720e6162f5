/*
 * dgswem_oracle.c -- plain, slow, FP64 CPU oracle of the DG-SWEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The product (the CUDA
 * library under paper_2508_21208_gb300/) shares no code, header, table or
 * constant generator with it, and never calls it.
 *
 * It follows Wichitrnithed, Valseth, Kubatko, Bunya & Dawson, "GPU-acceleration
 * of the Discontinuous Galerkin Shallow Water Equations Model (DG-SWEM) with
 * OpenACC" (arXiv 2508.21208):
 *   - Sec. 2.1, Eq. (SWE): 2D shallow water equations in (zeta, Hu_x, Hu_y);
 *   - Sec. 2.2, conservative form and Eq. (elem_weak_form): DG weak form per
 *     element; Eq. (dubiner): orthogonal Dubiner modal basis; Eq. (RKSSP):
 *     semi-discrete ODE advanced by SSP Runge-Kutta, optional slope limiter;
 *   - Sec. 5.2.1, Algorithm 1 (AREA), Sec. 5.2.2, Algorithm 2 (EDGE) and
 *     Algorithm 3 (GATHER): area integrals into RHS, per-(element, local edge)
 *     flux slots filled by an interior-edge loop, then a fixed-order gather;
 *   - Sec. 5.2.3: SLOPELIM, WETDRY and WIND kernels.
 * The array names (ZE/QX/QY, RHS_*, PHI_AREA, PHI_EDGE, XFAC/YFAC/SRFAC,
 * EDGE_*, NIEDN/NEDEL/LED) are the paper's (Table "tab:arrays", Alg. 2).
 *
 * Where the paper is silent or garbled, this file takes these readings:
 *   - the volume term enters with a plus sign, +(grad v, F): integration by
 *     parts gives it, and Alg. 1 accumulates +W_x F_x (Eq. elem_weak_form prints
 *     a minus);
 *   - the pressure flux is (g/2)(H^2 - h_b^2) (the flux matrix of Sec. 2.2 drops
 *     the 1/2; Eq. SWE and Sec. 5.2.1 keep it), written as (g/2) zeta (zeta + 2 h_b);
 *   - numerical flux: local Lax-Friedrichs, or Roe (Sec. 2.2 names both): Roe-averaged depth
 *     (H_i + H_o)/2 and sqrt(H)-weighted velocity, |A| from its eigen-decomposition in the edge
 *     frame, Harten's entropy fix on the two acoustic waves with delta = c/10;
 *   - "Gauss-Lobatto quadrature": a triangle needs a 2D rule; area integrals use
 *     Dunavant's symmetric rules (degree 4, 6 points for p=1; degree 6, 12 points
 *     for p=2) and edges Gauss-Legendre (2 points for p=1, 4 for p=2);
 *   - h_b is given at nodes and linear in each element; forcing is nodal and
 *     linear in each element;
 *   - friction tau_b = g n^2 |q| / H^(7/3) (Manning) or C_f |q| / H^2 (quadratic);
 *   - where the total depth H is not positive (no water), the velocity q/H, the wave speed and
 *     the friction are zero in the fluxes and the area integrals (the equations divide by H and
 *     give no rule there); the pressure term stays;
 *   - SSP Runge-Kutta (Sec. 2.2: Shu-Osher SSPRK; the paper's production scheme is a DG-optimised
 *     SSPRK(s,q), Kubatko et al. 2014) in the two-register Shu-Osher form
 *     u^(i) = a_i u^n + b_i u^(i-1) + c_i dt L(u^(i-1)): SSP(2,2) (default) and SSP(3,3)
 *     (Shu & Osher 1988), SSP(s,2) for s = 3, 4, 5 (Ketcheson 2008), SSP(4,3) (Spiteri & Ruuth
 *     2002), or caller coefficients; boundary data and forcing of stage i at t_n + tau_(i-1) dt with
 *     tau_0 = 0, tau_i = b_i tau_(i-1) + c_i;
 *   - limiter: Cockburn-Shu minmod limiter for triangles (nu = 1.5) on the linear
 *     modes of each variable; wet/dry: mean-preserving vertex-depth fix (Bunya et
 *     al. 2009 style), see wetdry() below;
 *   - land boundary: mirror ghost state; open boundary: zeta = A sin(2 pi t/T + phi),
 *     q taken from the interior; river boundary (Gamma_river, named in Sec. 2.1): the land mirror
 *     shifted so that the mean normal discharge of the two traces is the inflow -q_in;
 *   - rain R (Eq. SWE): a uniform rate in the continuity equation;
 *   - hurricane: Holland (1980) pressure and gradient wind, Garratt (1977) drag.
 * Readings pinned by their own cases: slope limiter (invariants, hand-worked examples of the
 * limiting and of the neighbour-pair order, and a recomputation from the mesh geometry) and
 * wet/dry (invariants, hand-worked examples, the edge rule against a sloshing wet element, and
 * convergence to Thacker's moving-shoreline solution in a parabolic bowl).
 *
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared (optionally -fopenmp).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXD 6   /* modes per variable at p <= 2 */
#define MAXQA 12 /* area quadrature points at p <= 2 */
#define MAXQE 4  /* edge quadrature points at p <= 2 */
#define NHQ 64   /* high-order rule used for projection and error norms */

/* ---------------------------------------------------------------- params */
typedef struct {
  int32_t p;
  double g, cfl, dt, h0;
  int32_t friction; /* 0 none, 1 Manning, 2 quadratic */
  double manning_n, cf;
  int32_t limiter;
  int32_t coriolis;
  double coriolis_lat_deg;
  double tide_amp, tide_period, tide_phase;
  int32_t hurricane;
  double pc_hpa, pn_hpa, rmax_m, holland_b, vt_ms, track_x0, track_y0, track_heading;
  double rho_air, rho_water;
  int32_t rk_scheme; /* 0 SSP(2,2), 1 SSP(3,3), 2 SSP(3,2), 3 SSP(4,2), 4 SSP(5,2), 5 SSP(4,3), 6 custom */
  int32_t rk_stages; /* custom: number of stages */
  double rk_coeffs[24]; /* custom: (a_i, b_i, c_i) per stage */
  int32_t flux;         /* 0 local Lax-Friedrichs, 1 Roe */
  double rain_rate;     /* R of Eq. SWE, uniform (m/s) */
  double river_q;       /* inflow discharge per unit width on river edges (m^2/s) */
} orc_params;

typedef void (*orc_field_cb)(double t, int32_t n, const double *xy, double *out);

typedef struct {
  orc_params prm;
  int p, nd, nqa, nqe;
  int nn, ne, ned, nint;
  double *x, *y, *hb;
  int *tri;
  /* edges: NEDEL[2*ed] = (e+, e-), LED[2*ed] = (l+, l-), ENODE[2*ed] = (a, b) in e+'s
   * counter-clockwise order, ETYPE: -1 interior, 0 land, 1 open; NIEDN: interior edge list */
  int *NEDEL, *LED, *ENODE, *ETYPE, *NIEDN, *EL_EDGE;
  double *EN_X, *EN_Y, *ELEN; /* unit normal outward from e+, edge length */
  /* element geometry */
  double *detJ, *rx, *ry, *sx, *sy, *area;
  /* limiter geometry: for local edge i, neighbour pair (j1, j2) and weights (a1, a2) */
  int *LIM_J;      /* [e][3][2], -1 = no admissible pair */
  double *LIM_A;   /* [e][3][2] */
  /* reference tables */
  double XQ[MAXQA], YQ[MAXQA], WQ[MAXQA];
  double PHI_AREA[MAXD][MAXQA], DPHI_XI[MAXD][MAXQA], DPHI_ETA[MAXD][MAXQA];
  double SQ[MAXQE], WE[MAXQE];
  double PHI_EDGE[3][MAXD][MAXQE]; /* basis on local edge l at its own parameter s_g */
  double NORM[MAXD];
  double HXQ[NHQ], HYQ[NHQ], HWQ[NHQ];
  /* state: U[(irk*3 + var)*nd + k][e]; irk 0 = u^n, 1 = u^(1) */
  double *U, *RHS, *EDGE; /* EDGE[((var*ne + e)*3 + l)*nd + k] */
  unsigned char *WD;      /* 0 wet, 1 partially wet, 2 dry */
  double *TSX, *TSY, *PA; /* nodal wind stress / rho_w and pressure anomaly (p - pn) / rho_w */
  double *MEAN;           /* scratch: element means used by the limiter */
  double dt, t0;
  int64_t nstep;
  /* the time step in progress, one stage at a time (orc_stage): next stage index, the stage-time
   * fraction tau and the register holding u^(i-1) */
  int st_i, st_prev;
  double st_tau;
  /* test-only manufactured-solution hooks */
  orc_field_cb mms_src, mms_bnd;
  int transmissive; /* test-only: every boundary ghost equals the interior trace */
  double *QXY;  /* physical coordinates of all area quadrature points [e][i][2] */
  double *QSRC; /* source values there [e][i][3] */
  double *BXY, *BVAL;
  int nbnd;
  int *BLIST;
} orc;

/* ------------------------------------------------------- Dubiner basis */
/* Eq. (dubiner): psi_ij(xi, eta) = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b), a = 2(1+xi)/(1-eta) - 1,
 * b = eta, on the reference triangle {xi, eta >= -1, xi + eta <= 0}.  Expanded for i+j <= 2 in
 * the mode order (0,0), (1,0), (0,1), (2,0), (1,1), (0,2). */
static void dubiner(int p, double xi, double eta, double *phi, double *dxi, double *deta) {
  phi[0] = 1.0;                      dxi[0] = 0.0;  deta[0] = 0.0;
  phi[1] = xi + 0.5 * eta + 0.5;     dxi[1] = 1.0;  deta[1] = 0.5;
  phi[2] = 0.5 * (1.0 + 3.0 * eta);  dxi[2] = 0.0;  deta[2] = 1.5;
  if (p >= 2) {
    phi[3] = 1.5 * xi * xi + 1.5 * xi * eta + 1.5 * xi + 0.25 * eta * eta + eta + 0.25;
    dxi[3] = 3.0 * xi + 1.5 * eta + 1.5;
    deta[3] = 1.5 * xi + 0.5 * eta + 1.0;
    phi[4] = 2.5 * xi * eta + 1.5 * xi + 1.25 * eta * eta + 2.0 * eta + 0.75;
    dxi[4] = 2.5 * eta + 1.5;
    deta[4] = 2.5 * xi + 2.5 * eta + 2.0;
    phi[5] = 2.5 * eta * eta + eta - 0.5;
    dxi[5] = 0.0;
    deta[5] = 5.0 * eta + 1.0;
  }
}

/* squared reference norms of the modes (orthogonality makes the mass matrix diagonal) */
static const double REF_NORM[MAXD] = {2.0, 1.0 / 3.0, 1.0, 2.0 / 15.0, 2.0 / 9.0, 2.0 / 3.0};

/* ----------------------------------------------------------- quadrature */
/* Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_n (three-term recurrence). */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[n - 1 - i] = z; /* ascending order */
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  /* symmetrise exactly so that node g and node n-1-g are mirror images */
  for (int i = 0; i < n / 2; ++i) {
    double a = 0.5 * (x[n - 1 - i] - x[i]), b = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = -a; x[n - 1 - i] = a; w[i] = b; w[n - 1 - i] = b;
  }
  if (n % 2) x[n / 2] = 0.0;
}

/* Dunavant (1985) symmetric triangle rules, barycentric orbits; weights sum to 1. */
static int dunavant(int degree, double *l1, double *l2, double *wt) {
  int n = 0;
#define ORBIT3(a, w)                                                    \
  do {                                                                 \
    double b_ = 1.0 - 2.0 * (a);                                       \
    l1[n] = (a); l2[n] = (a); wt[n++] = (w);                            \
    l1[n] = (a); l2[n] = b_; wt[n++] = (w);                             \
    l1[n] = b_; l2[n] = (a); wt[n++] = (w);                             \
  } while (0)
#define ORBIT6(a, b, w)                                                 \
  do {                                                                 \
    double c_ = 1.0 - (a) - (b);                                       \
    l1[n] = (a); l2[n] = (b); wt[n++] = (w);                            \
    l1[n] = (b); l2[n] = (a); wt[n++] = (w);                            \
    l1[n] = (a); l2[n] = c_; wt[n++] = (w);                             \
    l1[n] = c_; l2[n] = (a); wt[n++] = (w);                             \
    l1[n] = (b); l2[n] = c_; wt[n++] = (w);                             \
    l1[n] = c_; l2[n] = (b); wt[n++] = (w);                             \
  } while (0)
  if (degree == 4) {
    ORBIT3(0.445948490915965, 0.223381589678011);
    ORBIT3(0.091576213509771, 0.109951743655322);
  } else {
    ORBIT3(0.249286745170910, 0.116786275726379);
    ORBIT3(0.063089014491502, 0.050844906370207);
    ORBIT6(0.053145049844817, 0.310352451033784, 0.082851075618374);
  }
#undef ORBIT3
#undef ORBIT6
  return n;
}

/* reference vertices V0 = (-1,-1), V1 = (1,-1), V2 = (-1,1); local edge l runs from
 * vertex (l+1)%3 to vertex (l+2)%3 (counter-clockwise) and lies opposite vertex l. */
static const double RV[3][2] = {{-1.0, -1.0}, {1.0, -1.0}, {-1.0, 1.0}};

static void setup_tables(orc *o) {
  int p = o->p;
  o->nd = (p + 1) * (p + 2) / 2;
  double l1[MAXQA], l2[MAXQA], wt[MAXQA];
  o->nqa = dunavant(p == 1 ? 4 : 6, l1, l2, wt);
  for (int i = 0; i < o->nqa; ++i) {
    /* barycentric (l1, l2, 1-l1-l2) attached to vertices V1, V2, V0 */
    double l0 = 1.0 - l1[i] - l2[i];
    o->XQ[i] = l0 * RV[0][0] + l1[i] * RV[1][0] + l2[i] * RV[2][0];
    o->YQ[i] = l0 * RV[0][1] + l1[i] * RV[1][1] + l2[i] * RV[2][1];
    o->WQ[i] = 2.0 * wt[i]; /* reference triangle area is 2 */
    double ph[MAXD], dx[MAXD], dy[MAXD];
    dubiner(p, o->XQ[i], o->YQ[i], ph, dx, dy);
    for (int k = 0; k < o->nd; ++k) {
      o->PHI_AREA[k][i] = ph[k];
      o->DPHI_XI[k][i] = dx[k];
      o->DPHI_ETA[k][i] = dy[k];
    }
  }
  o->nqe = (p == 1) ? 2 : 4;
  gauss_legendre(o->nqe, o->SQ, o->WE);
  for (int l = 0; l < 3; ++l) {
    int a = (l + 1) % 3, b = (l + 2) % 3;
    for (int g = 0; g < o->nqe; ++g) {
      double s = o->SQ[g];
      double xi = 0.5 * (1.0 - s) * RV[a][0] + 0.5 * (1.0 + s) * RV[b][0];
      double eta = 0.5 * (1.0 - s) * RV[a][1] + 0.5 * (1.0 + s) * RV[b][1];
      double ph[MAXD], dx[MAXD], dy[MAXD];
      dubiner(p, xi, eta, ph, dx, dy);
      for (int k = 0; k < o->nd; ++k) o->PHI_EDGE[l][k][g] = ph[k];
    }
  }
  for (int k = 0; k < o->nd; ++k) o->NORM[k] = REF_NORM[k];
  /* collapsed-coordinate product rule (Duffy map) with 8x8 Gauss-Legendre points */
  double gx[8], gw[8];
  gauss_legendre(8, gx, gw);
  int n = 0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double a = gx[i], b = gx[j];
      o->HXQ[n] = 0.5 * (1.0 + a) * (1.0 - b) - 1.0;
      o->HYQ[n] = b;
      o->HWQ[n] = gw[i] * gw[j] * 0.5 * (1.0 - b);
      ++n;
    }
}

/* linear (P1) shape functions of the three vertices at reference point (xi, eta) */
static void shape_p1(double xi, double eta, double N[3]) {
  N[0] = -0.5 * (xi + eta);
  N[1] = 0.5 * (1.0 + xi);
  N[2] = 0.5 * (1.0 + eta);
}

/* ----------------------------------------------------------- mesh setup */
typedef struct { int lo, hi, e, l, a, b; } halfedge;

static int cmp_he(const void *pa, const void *pb) {
  const halfedge *a = pa, *b = pb;
  if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
  if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
  if (a->e != b->e) return a->e < b->e ? -1 : 1;
  return 0;
}

typedef struct { int lo, hi, type; } bkey;
static int cmp_bk(const void *pa, const void *pb) {
  const bkey *a = pa, *b = pb;
  if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
  if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
  return 0;
}

static void element_centroid(const orc *o, int e, double *cx, double *cy) {
  const int *t = o->tri + 3 * e;
  *cx = (o->x[t[0]] + o->x[t[1]] + o->x[t[2]]) / 3.0;
  *cy = (o->y[t[0]] + o->y[t[1]] + o->y[t[2]]) / 3.0;
}

static int build_edges(orc *o, int nb, const int32_t *bedge, const int32_t *btype) {
  int ne = o->ne, nh = 3 * ne;
  halfedge *h = malloc(sizeof(halfedge) * nh);
  for (int e = 0; e < ne; ++e)
    for (int l = 0; l < 3; ++l) {
      int a = o->tri[3 * e + (l + 1) % 3], b = o->tri[3 * e + (l + 2) % 3];
      halfedge *q = &h[3 * e + l];
      q->a = a; q->b = b; q->e = e; q->l = l;
      q->lo = a < b ? a : b; q->hi = a < b ? b : a;
    }
  qsort(h, nh, sizeof(halfedge), cmp_he);
  bkey *bk = malloc(sizeof(bkey) * (nb > 0 ? nb : 1));
  for (int i = 0; i < nb; ++i) {
    int a = bedge[2 * i], b = bedge[2 * i + 1];
    bk[i].lo = a < b ? a : b; bk[i].hi = a < b ? b : a; bk[i].type = btype[i];
  }
  qsort(bk, nb, sizeof(bkey), cmp_bk);
  int ned = 0, nint = 0, bad = 0;
  for (int i = 0; i < nh;) {
    int j = i + 1;
    while (j < nh && h[j].lo == h[i].lo && h[j].hi == h[i].hi) ++j;
    if (j - i > 2) bad = 1;
    if (j - i == 2 && !(h[i].a == h[i + 1].b && h[i].b == h[i + 1].a)) bad = 1;
    ned++;
    if (j - i == 2) nint++;
    i = j;
  }
  if (bad) { free(h); free(bk); return -1; }
  o->ned = ned; o->nint = nint;
  o->NEDEL = malloc(sizeof(int) * 2 * ned);
  o->LED = malloc(sizeof(int) * 2 * ned);
  o->ENODE = malloc(sizeof(int) * 2 * ned);
  o->ETYPE = malloc(sizeof(int) * ned);
  o->NIEDN = malloc(sizeof(int) * (nint > 0 ? nint : 1));
  o->EL_EDGE = malloc(sizeof(int) * 3 * ne);
  o->EN_X = malloc(sizeof(double) * ned);
  o->EN_Y = malloc(sizeof(double) * ned);
  o->ELEN = malloc(sizeof(double) * ned);
  int ed = 0, ii = 0;
  for (int i = 0; i < nh;) {
    int j = i + 1;
    while (j < nh && h[j].lo == h[i].lo && h[j].hi == h[i].hi) ++j;
    const halfedge *P = &h[i]; /* lower element index first: e+ */
    o->NEDEL[2 * ed] = P->e; o->LED[2 * ed] = P->l;
    o->ENODE[2 * ed] = P->a; o->ENODE[2 * ed + 1] = P->b;
    o->EL_EDGE[3 * P->e + P->l] = ed;
    if (j - i == 2) {
      const halfedge *M = &h[i + 1];
      o->NEDEL[2 * ed + 1] = M->e; o->LED[2 * ed + 1] = M->l;
      o->EL_EDGE[3 * M->e + M->l] = ed;
      o->ETYPE[ed] = -1;
      o->NIEDN[ii++] = ed;
    } else {
      o->NEDEL[2 * ed + 1] = -1; o->LED[2 * ed + 1] = -1;
      bkey key = {P->lo, P->hi, 0};
      bkey *f = nb > 0 ? bsearch(&key, bk, nb, sizeof(bkey), cmp_bk) : NULL;
      o->ETYPE[ed] = f ? f->type : 0;
    }
    double tx = o->x[P->b] - o->x[P->a], ty = o->y[P->b] - o->y[P->a];
    double L = sqrt(tx * tx + ty * ty);
    o->ELEN[ed] = L;
    o->EN_X[ed] = ty / L; /* outward for a counter-clockwise e+ */
    o->EN_Y[ed] = -tx / L;
    ed++;
    i = j;
  }
  free(h); free(bk);
  return 0;
}

static int build_geometry(orc *o) {
  int ne = o->ne;
  o->detJ = malloc(sizeof(double) * ne); o->area = malloc(sizeof(double) * ne);
  o->rx = malloc(sizeof(double) * ne); o->ry = malloc(sizeof(double) * ne);
  o->sx = malloc(sizeof(double) * ne); o->sy = malloc(sizeof(double) * ne);
  for (int e = 0; e < ne; ++e) {
    const int *t = o->tri + 3 * e;
    /* affine map x = -(xi+eta)/2 x0 + (1+xi)/2 x1 + (1+eta)/2 x2 */
    double xr = 0.5 * (o->x[t[1]] - o->x[t[0]]), xs = 0.5 * (o->x[t[2]] - o->x[t[0]]);
    double yr = 0.5 * (o->y[t[1]] - o->y[t[0]]), ys = 0.5 * (o->y[t[2]] - o->y[t[0]]);
    double J = xr * ys - xs * yr;
    if (!(J > 0.0)) return -1;
    o->detJ[e] = J;
    o->area[e] = 2.0 * J;
    o->rx[e] = ys / J; o->ry[e] = -xs / J;
    o->sx[e] = -yr / J; o->sy[e] = xr / J;
  }
  return 0;
}

/* Cockburn-Shu limiter geometry: write m_i - b0 = a1 (b_j1 - b0) + a2 (b_j2 - b0), a1, a2 >= 0,
 * with b_j the barycentre of the neighbour across local edge j (or, on the boundary, the mirror
 * image of b0 in that edge). Pairs are tried in the order (i,i+1), (i+2,i), (i+1,i+2). */
static void build_limiter_geometry(orc *o) {
  int ne = o->ne;
  o->LIM_J = malloc(sizeof(int) * 6 * ne);
  o->LIM_A = malloc(sizeof(double) * 6 * ne);
  for (int e = 0; e < ne; ++e) {
    double b0x, b0y, bx[3], by[3], mx[3], my[3];
    element_centroid(o, e, &b0x, &b0y);
    for (int j = 0; j < 3; ++j) {
      int ed = o->EL_EDGE[3 * e + j];
      int a = o->tri[3 * e + (j + 1) % 3], b = o->tri[3 * e + (j + 2) % 3];
      mx[j] = 0.5 * (o->x[a] + o->x[b]);
      my[j] = 0.5 * (o->y[a] + o->y[b]);
      int nb = (o->NEDEL[2 * ed] == e) ? o->NEDEL[2 * ed + 1] : o->NEDEL[2 * ed];
      if (nb >= 0) {
        element_centroid(o, nb, &bx[j], &by[j]);
      } else { /* reflect b0 across the edge line */
        double tx = o->x[b] - o->x[a], ty = o->y[b] - o->y[a];
        double s = ((b0x - o->x[a]) * tx + (b0y - o->y[a]) * ty) / (tx * tx + ty * ty);
        double fx = o->x[a] + s * tx, fy = o->y[a] + s * ty;
        bx[j] = 2.0 * fx - b0x;
        by[j] = 2.0 * fy - b0y;
      }
    }
    for (int i = 0; i < 3; ++i) {
      int pairs[3][2] = {{i, (i + 1) % 3}, {(i + 2) % 3, i}, {(i + 1) % 3, (i + 2) % 3}};
      int *J = o->LIM_J + 6 * e + 2 * i;
      double *A = o->LIM_A + 6 * e + 2 * i;
      J[0] = J[1] = -1;
      A[0] = A[1] = 0.0;
      for (int c = 0; c < 3; ++c) {
        int j1 = pairs[c][0], j2 = pairs[c][1];
        double d1x = bx[j1] - b0x, d1y = by[j1] - b0y, d2x = bx[j2] - b0x, d2y = by[j2] - b0y;
        double rx = mx[i] - b0x, ry = my[i] - b0y;
        double det = d1x * d2y - d2x * d1y;
        if (det == 0.0) continue;
        double a1 = (rx * d2y - d2x * ry) / det, a2 = (d1x * ry - rx * d1y) / det;
        if (a1 >= -1e-10 && a2 >= -1e-10) {
          J[0] = j1; J[1] = j2; A[0] = a1; A[1] = a2;
          break;
        }
      }
    }
  }
}

/* ---------------------------------------------------------- state access */
#define UIX(o, irk, v, k, e) ((size_t)(((irk) * 3 + (v)) * (o)->nd + (k)) * (o)->ne + (e))
#define RIX(o, v, k, e) ((size_t)((v) * (o)->nd + (k)) * (o)->ne + (e))
#define EIX(o, v, e, l, k) ((size_t)(((v) * (o)->ne + (e)) * 3 + (l)) * (o)->nd + (k))

static int wetdry_on(const orc *o) { return o->prm.h0 > 0.0; }

/* ----------------------------------------------------------------- WIND */
/* Holland (1980) parametric vortex: p(r) = pc + (pn - pc) exp(-(Rmax/r)^B), gradient wind
 * V = sqrt(B/rho_a (pn-pc) (Rmax/r)^B exp(-(Rmax/r)^B) + (r f/2)^2) - r f/2, surface wind 0.9 V,
 * counter-clockwise, plus half the translation velocity; Garratt (1977) drag
 * C_d = min(0.75 + 0.067 |U|, 3.5) 1e-3; stress / rho_w = rho_a/rho_w C_d |U| U.
 * The pressure enters Eq. SWE only through its gradient, so the stored value is the anomaly
 * p - pn = (pn - pc) expm1(-(Rmax/r)^B): the same gradient, without the cancellation of
 * differencing values near pn (about 1e5 Pa) across an element. */
static void wind(orc *o, double t) {
  const orc_params *P = &o->prm;
  double f = 2.0 * 7.2921e-5 * sin(P->coriolis_lat_deg * M_PI / 180.0);
  double cx = P->track_x0 + P->vt_ms * cos(P->track_heading) * t;
  double cy = P->track_y0 + P->vt_ms * sin(P->track_heading) * t;
  double pc = 100.0 * P->pc_hpa, pn = 100.0 * P->pn_hpa, B = P->holland_b;
#pragma omp parallel for
  for (int n = 0; n < o->nn; ++n) {
    double dx = o->x[n] - cx, dy = o->y[n] - cy;
    double r = sqrt(dx * dx + dy * dy);
    double pr, ux, uy;
    if (r < 1.0) {
      pr = pc - pn;
      ux = 0.5 * P->vt_ms * cos(P->track_heading);
      uy = 0.5 * P->vt_ms * sin(P->track_heading);
    } else {
      double A = pow(P->rmax_m / r, B), E = exp(-A);
      pr = (pn - pc) * expm1(-A);
      double V = sqrt(B / P->rho_air * (pn - pc) * A * E + (0.5 * r * f) * (0.5 * r * f)) - 0.5 * r * f;
      ux = 0.9 * V * (-dy / r) + 0.5 * P->vt_ms * cos(P->track_heading);
      uy = 0.9 * V * (dx / r) + 0.5 * P->vt_ms * sin(P->track_heading);
    }
    double U = sqrt(ux * ux + uy * uy);
    double cd = 0.75 + 0.067 * U;
    if (cd > 3.5) cd = 3.5;
    cd *= 1e-3;
    o->TSX[n] = P->rho_air / P->rho_water * cd * U * ux;
    o->TSY[n] = P->rho_air / P->rho_water * cd * U * uy;
    o->PA[n] = pr / P->rho_water;
  }
}

/* ------------------------------------------------- point physics (Eq. SWE) */
static double friction_tau(const orc_params *P, double qx, double qy, double H) {
  if (!(H > 0.0)) return 0.0; /* no water: zero velocity (see flux_n) */
  double qm = sqrt(qx * qx + qy * qy);
  if (P->friction == 1) return P->g * P->manning_n * P->manning_n * qm / pow(H, 7.0 / 3.0);
  if (P->friction == 2) return P->cf * qm / (H * H);
  return 0.0;
}

/* normal component F(w).n of the physical flux; w = (zeta, qx, qy).  The velocity q/H is taken
 * as zero where the total depth H is not positive (no water there; the paper's equations divide
 * by H without a rule for it), here, in the wave speeds and in the area integrals and friction. */
static void flux_n(double g, const double w[3], double hb, double nx, double ny, double F[3]) {
  double H = w[0] + hb;
  double qn = w[1] * nx + w[2] * ny;
  double P = 0.5 * g * w[0] * (w[0] + 2.0 * hb);
  F[0] = qn;
  F[1] = H > 0.0 ? w[1] * qn / H + P * nx : P * nx;
  F[2] = H > 0.0 ? w[2] * qn / H + P * ny : P * ny;
}

/* local Lax-Friedrichs flux, n pointing from the inner (wi) to the outer (wo) state */
static void llf(double g, const double wi[3], const double wo[3], double hb, double nx, double ny,
                double out[3]) {
  double Fi[3], Fo[3];
  flux_n(g, wi, hb, nx, ny, Fi);
  flux_n(g, wo, hb, nx, ny, Fo);
  double Hi = wi[0] + hb, Ho = wo[0] + hb;
  double si = Hi > 0.0 ? fabs((wi[1] * nx + wi[2] * ny) / Hi) + sqrt(g * Hi) : 0.0;
  double so = Ho > 0.0 ? fabs((wo[1] * nx + wo[2] * ny) / Ho) + sqrt(g * Ho) : 0.0;
  double lam = si > so ? si : so;
  for (int v = 0; v < 3; ++v) out[v] = 0.5 * (Fi[v] + Fo[v]) - 0.5 * lam * (wo[v] - wi[v]);
}

/* Roe (1981) flux, n from the inner (wi) to the outer (wo) state.  In the edge frame (normal n,
 * tangent t = (-ny, nx)) the state is (H, q_n, q_t); the Roe averages are H~ = (Hi + Ho)/2,
 * u~ = (sqrt(Hi) ui + sqrt(Ho) uo) / (sqrt(Hi) + sqrt(Ho)) (both components), c~ = sqrt(g H~); the
 * eigenvalues u~_n - c~, u~_n, u~_n + c~ have right eigenvectors (1, u~_n - c~, u~_t),
 * (0, 0, 1), (1, u~_n + c~, u~_t) and wave strengths
 * a1 = ((u~_n + c~) dH - dq_n) / (2 c~), a2 = dq_t - u~_t dH, a3 = (dq_n - (u~_n - c~) dH) / (2 c~);
 * Fhat = (F(wi) + F(wo)).n / 2 - sum_k |lambda_k| a_k r_k / 2, with |lambda| of the acoustic waves
 * replaced by (lambda^2 + d^2) / (2 d) below d = c~/10 (Harten).  dH = d zeta (h_b continuous). */
static double harten(double lam, double d) {
  double a = fabs(lam);
  return (a < d) ? 0.5 * (lam * lam + d * d) / d : a;
}

static void roe(double g, const double wi[3], const double wo[3], double hb, double nx, double ny, double out[3]) {
  double Fi[3], Fo[3];
  flux_n(g, wi, hb, nx, ny, Fi);
  flux_n(g, wo, hb, nx, ny, Fo);
  double Hi = wi[0] + hb, Ho = wo[0] + hb;
  double qni = wi[1] * nx + wi[2] * ny, qti = -wi[1] * ny + wi[2] * nx;
  double qno = wo[1] * nx + wo[2] * ny, qto = -wo[1] * ny + wo[2] * nx;
  double si = sqrt(Hi > 0.0 ? Hi : 0.0), so = sqrt(Ho > 0.0 ? Ho : 0.0);
  double un = 0.0, ut = 0.0;
  if (si + so > 0.0) {
    un = (si * (Hi > 0.0 ? qni / Hi : 0.0) + so * (Ho > 0.0 ? qno / Ho : 0.0)) / (si + so);
    ut = (si * (Hi > 0.0 ? qti / Hi : 0.0) + so * (Ho > 0.0 ? qto / Ho : 0.0)) / (si + so);
  }
  double Hm = 0.5 * (Hi + Ho);
  double c = sqrt(g * (Hm > 0.0 ? Hm : 0.0));
  double dH = wo[0] - wi[0], dqn = qno - qni, dqt = qto - qti;
  double dn = 0.0, dt = 0.0, dh = 0.0; /* |A| dw in the edge frame */
  if (c > 0.0) {
    double a1 = ((un + c) * dH - dqn) / (2.0 * c);
    double a3 = (dqn - (un - c) * dH) / (2.0 * c);
    double a2 = dqt - ut * dH;
    double l1 = harten(un - c, 0.1 * c), l2 = fabs(un), l3 = harten(un + c, 0.1 * c);
    dh = l1 * a1 + l3 * a3;
    dn = l1 * a1 * (un - c) + l3 * a3 * (un + c);
    dt = l1 * a1 * ut + l2 * a2 + l3 * a3 * ut;
  }
  out[0] = 0.5 * (Fi[0] + Fo[0]) - 0.5 * dh;
  out[1] = 0.5 * (Fi[1] + Fo[1]) - 0.5 * (dn * nx - dt * ny);
  out[2] = 0.5 * (Fi[2] + Fo[2]) - 0.5 * (dn * ny + dt * nx);
}

/* the numerical flux selected by the parameters */
static void num_flux(const orc_params *P, const double wi[3], const double wo[3], double hb, double nx, double ny,
                     double out[3]) {
  if (P->flux == 1)
    roe(P->g, wi, wo, hb, nx, ny, out);
  else
    llf(P->g, wi, wo, hb, nx, ny, out);
}

/* land boundary: mirror ghost zeta- = zeta+, q- = q+ - 2 (q+.n) n, then the numerical flux */
static void wall_flux(const orc_params *P, const double wi[3], double hb, double nx, double ny, double out[3]) {
  double qn = wi[1] * nx + wi[2] * ny;
  double wo[3] = {wi[0], wi[1] - 2.0 * qn * nx, wi[2] - 2.0 * qn * ny};
  num_flux(P, wi, wo, hb, nx, ny, out);
}

/* ------------------------------------------------------ AREA (Alg. 1) */
static void area_integrals(orc *o, int irk) {
  const orc_params *P = &o->prm;
  const int nd = o->nd;
  double f = P->coriolis ? 2.0 * 7.2921e-5 * sin(P->coriolis_lat_deg * M_PI / 180.0) : 0.0;
#pragma omp parallel for
  for (int L = 0; L < o->ne; ++L) {
    const int *t = o->tri + 3 * L;
    double hbv[3] = {o->hb[t[0]], o->hb[t[1]], o->hb[t[2]]};
    /* constant gradients of linear nodal fields (bathymetry, pressure) */
    double dN_dx[3], dN_dy[3];
    {
      const double dxi[3] = {-0.5, 0.5, 0.0}, deta[3] = {-0.5, 0.0, 0.5};
      for (int a = 0; a < 3; ++a) {
        dN_dx[a] = o->rx[L] * dxi[a] + o->sx[L] * deta[a];
        dN_dy[a] = o->ry[L] * dxi[a] + o->sy[L] * deta[a];
      }
    }
    double dhb_dx = 0, dhb_dy = 0, dpa_dx = 0, dpa_dy = 0;
    for (int a = 0; a < 3; ++a) {
      dhb_dx += hbv[a] * dN_dx[a];
      dhb_dy += hbv[a] * dN_dy[a];
      if (P->hurricane) {
        dpa_dx += o->PA[t[a]] * dN_dx[a];
        dpa_dy += o->PA[t[a]] * dN_dy[a];
      }
    }
    double rhs[3][MAXD];
    memset(rhs, 0, sizeof rhs);
    for (int i = 0; i < o->nqa; ++i) {
      double ze = 0, qx = 0, qy = 0;
      for (int k = 0; k < nd; ++k) {
        double Phi = o->PHI_AREA[k][i];
        ze += o->U[UIX(o, irk, 0, k, L)] * Phi;
        qx += o->U[UIX(o, irk, 1, k, L)] * Phi;
        qy += o->U[UIX(o, irk, 2, k, L)] * Phi;
      }
      double N[3];
      shape_p1(o->XQ[i], o->YQ[i], N);
      double hbq = N[0] * hbv[0] + N[1] * hbv[1] + N[2] * hbv[2];
      double H = ze + hbq;
      double Pp = 0.5 * P->g * ze * (ze + 2.0 * hbq);
      /* Continuity_Flux, X_Flux, Y_Flux */
      double Fx = qx, Fy = qy;
      double Gx = Pp, Gy = 0.0, Hx = 0.0, Hy = Pp; /* zero velocity where H <= 0 (see flux_n) */
      if (H > 0.0) {
        Gx = qx * qx / H + Pp;
        Gy = qx * qy / H;
        Hx = qx * qy / H;
        Hy = qy * qy / H + Pp;
      }
      /* Continuity_Source, X_Source, Y_Source */
      double SR = P->rain_rate;
      double tau = friction_tau(P, qx, qy, H);
      double Sx = P->g * ze * dhb_dx - tau * qx + f * qy;
      double Sy = P->g * ze * dhb_dy - tau * qy - f * qx;
      if (P->hurricane) {
        double wsx = N[0] * o->TSX[t[0]] + N[1] * o->TSX[t[1]] + N[2] * o->TSX[t[2]];
        double wsy = N[0] * o->TSY[t[0]] + N[1] * o->TSY[t[1]] + N[2] * o->TSY[t[2]];
        Sx += wsx - H * dpa_dx;
        Sy += wsy - H * dpa_dy;
      }
      if (o->mms_src) {
        const double *s = o->QSRC + ((size_t)L * o->nqa + i) * 3;
        SR += s[0]; Sx += s[1]; Sy += s[2];
      }
      for (int k = 0; k < nd; ++k) {
        /* integration weights XFAC, YFAC, SRFAC of Table tab:arrays */
        double Wx = o->WQ[i] * o->detJ[L] * (o->rx[L] * o->DPHI_XI[k][i] + o->sx[L] * o->DPHI_ETA[k][i]);
        double Wy = o->WQ[i] * o->detJ[L] * (o->ry[L] * o->DPHI_XI[k][i] + o->sy[L] * o->DPHI_ETA[k][i]);
        double Ws = o->WQ[i] * o->detJ[L] * o->PHI_AREA[k][i];
        rhs[0][k] += Wx * Fx + Wy * Fy + Ws * SR;
        rhs[1][k] += Wx * Gx + Wy * Gy + Ws * Sx;
        rhs[2][k] += Wx * Hx + Wy * Hy + Ws * Sy;
      }
    }
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < nd; ++k) o->RHS[RIX(o, v, k, L)] = rhs[v][k];
  }
}

/* --------------------------------------------- EDGE (Alg. 2) and boundaries */
static void trace(const orc *o, int irk, int e, int l, int g, double w[3]) {
  for (int v = 0; v < 3; ++v) {
    double s = 0.0;
    for (int k = 0; k < o->nd; ++k) s += o->U[UIX(o, irk, v, k, e)] * o->PHI_EDGE[l][k][g];
    w[v] = s;
  }
}

static double edge_hb(const orc *o, int ed, int g) {
  double s = o->SQ[g];
  return 0.5 * (1.0 - s) * o->hb[o->ENODE[2 * ed]] + 0.5 * (1.0 + s) * o->hb[o->ENODE[2 * ed + 1]];
}

/* add -<phi_k, Fhat.n> (n outward from element e) for one quadrature point to its edge slot */
static void add_slot(orc *o, int e, int l, int g_own, double wlen, const double F[3]) {
  for (int v = 0; v < 3; ++v)
    for (int k = 0; k < o->nd; ++k)
      o->EDGE[EIX(o, v, e, l, k)] -= wlen * o->PHI_EDGE[l][k][g_own] * F[v];
}

/* wetting/drying edge rule: an edge touching a dry element carries no flow (both sides see a
 * wall) unless the wet side's surface trace rises above the highest bed (-h_b) on the edge */
static int edge_flows(const orc *o, int irk, int ed) {
  if (!wetdry_on(o)) return 1;
  int ep = o->NEDEL[2 * ed], em = o->NEDEL[2 * ed + 1];
  int dp = o->WD[ep] == 2, dm = o->WD[em] == 2;
  if (!dp && !dm) return 1;
  if (dp && dm) return 0;
  double bed = -o->hb[o->ENODE[2 * ed]];
  double bed2 = -o->hb[o->ENODE[2 * ed + 1]];
  if (bed2 > bed) bed = bed2;
  int ew = dp ? em : ep, lw = dp ? o->LED[2 * ed + 1] : o->LED[2 * ed];
  double zmax = -INFINITY;
  for (int g = 0; g < o->nqe; ++g) {
    int gw = dp ? o->nqe - 1 - g : g;
    double w[3];
    trace(o, irk, ew, lw, gw, w);
    if (w[0] > zmax) zmax = w[0];
  }
  return zmax > bed;
}

static void edge_integrals(orc *o, int irk, double ts) {
  const orc_params *P = &o->prm;
  const int nq = o->nqe;
  memset(o->EDGE, 0, sizeof(double) * 3 * (size_t)o->ne * 3 * o->nd);
  /* interior edges (Alg. 2); each edge writes only its own two slots */
#pragma omp parallel for
  for (int D = 0; D < o->nint; ++D) {
    int L = o->NIEDN[D];
    int ep = o->NEDEL[2 * L], em = o->NEDEL[2 * L + 1];
    int lp = o->LED[2 * L], lm = o->LED[2 * L + 1];
    int flows = edge_flows(o, irk, L);
    double nx = o->EN_X[L], ny = o->EN_Y[L];
    for (int i = 0; i < nq; ++i) {
      int im = nq - 1 - i; /* the same point seen from e- */
      double wp[3], wm[3], hb = edge_hb(o, L, i);
      trace(o, irk, ep, lp, i, wp);
      trace(o, irk, em, lm, im, wm);
      double wlen = 0.5 * o->ELEN[L] * o->WE[i];
      if (flows) {
        double F[3], Fm[3];
        num_flux(P, wp, wm, hb, nx, ny, F);
        add_slot(o, ep, lp, i, wlen, F);
        for (int v = 0; v < 3; ++v) Fm[v] = -F[v]; /* n(e-) = -n(e+) */
        add_slot(o, em, lm, im, wlen, Fm);
      } else {
        double Fp[3], Fm[3];
        wall_flux(P, wp, hb, nx, ny, Fp);
        wall_flux(P, wm, hb, -nx, -ny, Fm);
        add_slot(o, ep, lp, i, wlen, Fp);
        add_slot(o, em, lm, im, wlen, Fm);
      }
    }
  }
  /* boundary edges: land (mirror) and open (tidal elevation) */
  double zt = P->tide_amp * sin(2.0 * M_PI * ts / P->tide_period + P->tide_phase);
  for (int L = 0; L < o->ned; ++L) {
    if (o->ETYPE[L] < 0) continue;
    int ep = o->NEDEL[2 * L], lp = o->LED[2 * L];
    double nx = o->EN_X[L], ny = o->EN_Y[L];
    for (int i = 0; i < nq; ++i) {
      double wp[3], F[3], hb = edge_hb(o, L, i);
      trace(o, irk, ep, lp, i, wp);
      if (o->transmissive) {
        num_flux(P, wp, wp, hb, nx, ny, F);
      } else if (o->mms_bnd) {
        int bi = -1;
        for (int b = 0; b < o->nbnd; ++b)
          if (o->BLIST[b] == L) { bi = b; break; }
        num_flux(P, wp, o->BVAL + ((size_t)bi * nq + i) * 3, hb, nx, ny, F);
      } else if (o->ETYPE[L] == 1) {
        double wo[3] = {zt, wp[1], wp[2]};
        num_flux(P, wp, wo, hb, nx, ny, F);
      } else if (o->ETYPE[L] == 2) {
        /* river: q- = q+ - 2 (q+.n + q_in) n, so that (q+ + q-).n / 2 = -q_in */
        double qn = wp[1] * nx + wp[2] * ny;
        double wo[3] = {wp[0], wp[1] - 2.0 * (qn + P->river_q) * nx, wp[2] - 2.0 * (qn + P->river_q) * ny};
        num_flux(P, wp, wo, hb, nx, ny, F);
      } else {
        wall_flux(P, wp, hb, nx, ny, F);
      }
      add_slot(o, ep, lp, i, 0.5 * o->ELEN[L] * o->WE[i], F);
    }
  }
}

/* ------------------------------------------------------ GATHER (Alg. 3) */
static void flux_gather(orc *o) {
#pragma omp parallel for
  for (int L = 0; L < o->ne; ++L)
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < o->nd; ++k)
        for (int i = 0; i < 3; ++i) o->RHS[RIX(o, v, k, L)] += o->EDGE[EIX(o, v, L, i, k)];
}

/* ------------------------------------------------- SLOPELIM (Sec. 5.2.3) */
static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

static void slope_limiter(orc *o, int irk) {
  const int nd = o->nd, ne = o->ne;
  const double nu = 1.5;
  /* reference edge midpoints and the linear modes' values there */
  double ph_m[3][MAXD];
  for (int i = 0; i < 3; ++i) {
    int a = (i + 1) % 3, b = (i + 2) % 3;
    double dx[MAXD], dy[MAXD];
    dubiner(o->p, 0.5 * (RV[a][0] + RV[b][0]), 0.5 * (RV[a][1] + RV[b][1]), ph_m[i], dx, dy);
  }
  for (int v = 0; v < 3; ++v)
    for (int e = 0; e < ne; ++e) o->MEAN[v * ne + e] = o->U[UIX(o, irk, v, 0, e)];
#pragma omp parallel for
  for (int e = 0; e < ne; ++e) {
    int nbr[3];
    for (int j = 0; j < 3; ++j) {
      int ed = o->EL_EDGE[3 * e + j];
      nbr[j] = (o->NEDEL[2 * ed] == e) ? o->NEDEL[2 * ed + 1] : o->NEDEL[2 * ed];
    }
    int any = 0;
    double newlin[3][2];
    int act[3] = {0, 0, 0};
    for (int v = 0; v < 3; ++v) {
      double u0 = o->MEAN[v * ne + e], ub[3], ut[3], d[3];
      for (int j = 0; j < 3; ++j) ub[j] = nbr[j] >= 0 ? o->MEAN[v * ne + nbr[j]] : u0;
      double u1 = o->U[UIX(o, irk, v, 1, e)], u2 = o->U[UIX(o, irk, v, 2, e)];
      for (int i = 0; i < 3; ++i) {
        ut[i] = u1 * ph_m[i][1] + u2 * ph_m[i][2];
        const int *J = o->LIM_J + 6 * e + 2 * i;
        const double *A = o->LIM_A + 6 * e + 2 * i;
        double db = (J[0] >= 0) ? A[0] * (ub[J[0]] - u0) + A[1] * (ub[J[1]] - u0) : 0.0;
        d[i] = minmod(ut[i], nu * db);
        if (d[i] != ut[i]) act[v] = 1;
      }
      if (!act[v]) continue;
      any = 1;
      double pos = 0.0, neg = 0.0;
      for (int i = 0; i < 3; ++i) {
        pos += d[i] > 0.0 ? d[i] : 0.0;
        neg += d[i] < 0.0 ? -d[i] : 0.0;
      }
      double tp = pos > 0.0 ? (neg / pos < 1.0 ? neg / pos : 1.0) : 0.0;
      double tm = neg > 0.0 ? (pos / neg < 1.0 ? pos / neg : 1.0) : 0.0;
      double dh[3];
      for (int i = 0; i < 3; ++i) dh[i] = tp * (d[i] > 0.0 ? d[i] : 0.0) - tm * (d[i] < 0.0 ? -d[i] : 0.0);
      /* the linear function with deviations dh at the midpoints of edges 0 and 1 */
      double det = ph_m[0][1] * ph_m[1][2] - ph_m[0][2] * ph_m[1][1];
      newlin[v][0] = (dh[0] * ph_m[1][2] - ph_m[0][2] * dh[1]) / det;
      newlin[v][1] = (ph_m[0][1] * dh[1] - dh[0] * ph_m[1][1]) / det;
    }
    if (!any) continue;
    for (int v = 0; v < 3; ++v) {
      if (!act[v]) continue;
      o->U[UIX(o, irk, v, 1, e)] = newlin[v][0];
      o->U[UIX(o, irk, v, 2, e)] = newlin[v][1];
    }
    if (o->p >= 2) /* a limited element drops its quadratic modes (all variables) */
      for (int v = 0; v < 3; ++v)
        for (int k = 3; k < nd; ++k) o->U[UIX(o, irk, v, k, e)] = 0.0;
  }
}

/* --------------------------------------------------- WETDRY (Sec. 5.2.3) */
/* Vertex depths H_i = zeta(V_i) + h_b,i of the linear part; dry if their mean <= h0 (flatten);
 * otherwise, if some H_i < h0, lift those to h0 and scale the others' excess over h0 so that the
 * sum (hence the mean) is kept; wet if all fixed depths exceed h0, else partially wet.  Dry
 * elements, and partially wet ones whose mean surface lies below the highest bed among their
 * vertices at h0, lose all momentum; at p = 2 non-wet elements drop their quadratic modes.
 * "At h0" and "mean <= h0" are taken with a tolerance WD_TOL (1e-10 m), so that a depth rebuilt
 * from the modes with rounding error still classifies the same way. */
#define WD_TOL 1e-10
static void wetdry(orc *o, int irk) {
  const double h0 = o->prm.h0;
  const int nd = o->nd;
  double phv[3][MAXD];
  for (int i = 0; i < 3; ++i) {
    double dx[MAXD], dy[MAXD];
    dubiner(o->p, RV[i][0], RV[i][1], phv[i], dx, dy);
  }
#pragma omp parallel for
  for (int e = 0; e < o->ne; ++e) {
    const int *t = o->tri + 3 * e;
    double hbv[3] = {o->hb[t[0]], o->hb[t[1]], o->hb[t[2]]};
    double z0 = o->U[UIX(o, irk, 0, 0, e)], z1 = o->U[UIX(o, irk, 0, 1, e)], z2 = o->U[UIX(o, irk, 0, 2, e)];
    double H[3];
    for (int i = 0; i < 3; ++i) H[i] = z0 * phv[i][0] + z1 * phv[i][1] + z2 * phv[i][2] + hbv[i];
    double Hm = (H[0] + H[1] + H[2]) / 3.0;
    int flag;
    int changed = 0;
    if (Hm <= h0 + WD_TOL) {
      H[0] = H[1] = H[2] = Hm;
      flag = 2;
      changed = 1;
    } else {
      double hmin = H[0] < H[1] ? (H[0] < H[2] ? H[0] : H[2]) : (H[1] < H[2] ? H[1] : H[2]);
      if (hmin < h0) {
        double ex = 0.0;
        for (int i = 0; i < 3; ++i)
          if (H[i] >= h0) ex += H[i] - h0;
        double S = (3.0 * Hm - 3.0 * h0) / ex;
        for (int i = 0; i < 3; ++i) H[i] = (H[i] < h0) ? h0 : h0 + (H[i] - h0) * S;
        changed = 1;
      }
      flag = (H[0] > h0 + WD_TOL && H[1] > h0 + WD_TOL && H[2] > h0 + WD_TOL) ? 0 : 1;
    }
    if (changed) {
      /* Dubiner linear modes of the interpolant through the vertex surface values (mode 0 kept) */
      double zv[3] = {H[0] - hbv[0], H[1] - hbv[1], H[2] - hbv[2]};
      o->U[UIX(o, irk, 0, 1, e)] = 0.5 * (zv[1] - zv[0]);
      o->U[UIX(o, irk, 0, 2, e)] = (2.0 * zv[2] - zv[0] - zv[1]) / 6.0;
    }
    int zero_q = (flag == 2);
    if (flag == 1) {
      double bed = -INFINITY;
      for (int i = 0; i < 3; ++i)
        if (H[i] <= h0 + WD_TOL && -hbv[i] > bed) bed = -hbv[i];
      if (z0 < bed) zero_q = 1;
    }
    if (zero_q)
      for (int k = 0; k < nd; ++k) o->U[UIX(o, irk, 1, k, e)] = o->U[UIX(o, irk, 2, k, e)] = 0.0;
    if (flag != 0 && o->p >= 2)
      for (int v = 0; v < 3; ++v)
        for (int k = 3; k < nd; ++k) o->U[UIX(o, irk, v, k, e)] = 0.0;
    o->WD[e] = (unsigned char)flag;
  }
}

/* ------------------------------------------------------- right-hand side */
static void prepare_mms(orc *o, double ts) {
  if (o->mms_src) o->mms_src(ts, o->ne * o->nqa, o->QXY, o->QSRC);
  if (o->mms_bnd) o->mms_bnd(ts, o->nbnd * o->nqe, o->BXY, o->BVAL);
}

/* L_h(w) of Eq. (RKSSP): RHS = AREA + GATHER(EDGE), then the inverse (diagonal) mass matrix */
static void eval_L(orc *o, int irk, double ts) {
  if (o->prm.hurricane) wind(o, ts);
  prepare_mms(o, ts);
  area_integrals(o, irk);
  edge_integrals(o, irk, ts);
  flux_gather(o);
#pragma omp parallel for
  for (int e = 0; e < o->ne; ++e)
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < o->nd; ++k) o->RHS[RIX(o, v, k, e)] /= o->detJ[e] * o->NORM[k];
}

static void postprocess(orc *o, int irk) {
  if (o->prm.limiter) slope_limiter(o, irk);
  if (wetdry_on(o)) wetdry(o, irk);
}

/* stage coefficients (a_i, b_i, c_i) of the two-register Shu-Osher form; returns the stage count */
static int rk_table(const orc_params *P, double a[8], double b[8], double c[8]) {
  int s = 0;
#define ST(A, B, C) do { a[s] = (A); b[s] = (B); c[s] = (C); ++s; } while (0)
  switch (P->rk_scheme) {
    case 0: /* SSP(2,2) */
      ST(0.0, 1.0, 1.0); ST(0.5, 0.5, 0.5);
      break;
    case 1: /* SSP(3,3) */
      ST(0.0, 1.0, 1.0); ST(0.75, 0.25, 0.25); ST(1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0);
      break;
    case 2: case 3: case 4: { /* SSP(s,2): s-1 forward Euler steps of dt/(s-1), then the average */
      const int n = P->rk_scheme + 1;
      for (int i = 0; i < n - 1; ++i) ST(0.0, 1.0, 1.0 / (n - 1));
      ST(1.0 / n, (n - 1.0) / n, 1.0 / n);
      break;
    }
    case 5: /* SSP(4,3) */
      ST(0.0, 1.0, 0.5); ST(0.0, 1.0, 0.5); ST(2.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0); ST(0.0, 1.0, 0.5);
      break;
    case 6:
      for (int i = 0; i < P->rk_stages && i < 8; ++i)
        ST(P->rk_coeffs[3 * i], P->rk_coeffs[3 * i + 1], P->rk_coeffs[3 * i + 2]);
      break;
    default:
      return 0;
  }
#undef ST
  return s;
}

/* one stage of the SSP-RK step in progress: u^(0) = u^n, u^(i) = a_i u^n + b_i u^(i-1) +
 * c_i dt L(u^(i-1)), then limiter and wet/dry; u^(n+1) = u^(s).  Buffers: 0 = u^n, 1 and 2
 * alternate, the last stage writes 0.  Returns the buffer written. */
static int ssprk_stage(orc *o) {
  const double dt = o->dt;
  double a[8], b[8], c[8];
  const int s = rk_table(&o->prm, a, b, c);
  size_t n = (size_t)3 * o->nd * o->ne;
  const int i = o->st_i;
  if (i == 0) {
    o->st_tau = 0.0;
    o->st_prev = 0;
  }
  const int prev = o->st_prev;
  double ts = o->t0 + ((double)o->nstep + o->st_tau) * dt;
  eval_L(o, prev, ts);
  int out = (i == s - 1) ? 0 : (i % 2 == 0 ? 1 : 2);
  double *U0 = o->U, *Up = o->U + (size_t)prev * n, *Uo = o->U + (size_t)out * n;
  for (size_t k = 0; k < n; ++k) Uo[k] = a[i] * U0[k] + b[i] * Up[k] + c[i] * dt * o->RHS[k];
  postprocess(o, out);
  o->st_prev = out;
  o->st_tau = b[i] * o->st_tau + c[i];
  if (i == s - 1) {
    o->st_i = 0;
    o->nstep++;
  } else {
    o->st_i = i + 1;
  }
  return out;
}

static void ssprk_step(orc *o) {
  double a[8], b[8], c[8];
  const int s = rk_table(&o->prm, a, b, c);
  for (int i = o->st_i; i < s; ++i) ssprk_stage(o);
}

/* ------------------------------------------------------------- time step */
/* dt = CFL * 3/(2p+1) * min_e r_e / lambda_e, r_e the inradius and lambda_e the largest
 * |u| + sqrt(g max(H, h0)) over the element's vertices (state at t0).  (With the inscribed
 * diameter 2 r_e in place of r_e, CFL 0.3 is unstable for P1 / SSP-RK2.) */
static double compute_dt(const orc *o) {
  double phv[3][MAXD];
  for (int i = 0; i < 3; ++i) {
    double dx[MAXD], dy[MAXD];
    dubiner(o->p, RV[i][0], RV[i][1], phv[i], dx, dy);
  }
  double best = INFINITY;
  for (int e = 0; e < o->ne; ++e) {
    const int *t = o->tri + 3 * e;
    double per = 0.0;
    for (int a = 0; a < 3; ++a) {
      int n0 = t[a], n1 = t[(a + 1) % 3];
      double dx = o->x[n1] - o->x[n0], dy = o->y[n1] - o->y[n0];
      per += sqrt(dx * dx + dy * dy);
    }
    double r = 2.0 * o->area[e] / per;
    double lam = 0.0;
    for (int i = 0; i < 3; ++i) {
      double w[3];
      for (int v = 0; v < 3; ++v) {
        double s = 0.0;
        for (int k = 0; k < o->nd; ++k) s += o->U[UIX(o, 0, v, k, e)] * phv[i][k];
        w[v] = s;
      }
      double H = w[0] + o->hb[t[i]];
      double Hc = H > o->prm.h0 ? H : o->prm.h0;
      double um = Hc > 0.0 ? sqrt(w[1] * w[1] + w[2] * w[2]) / Hc : 0.0;
      double s = um + sqrt(o->prm.g * Hc);
      if (s > lam) lam = s;
    }
    if (lam > 0.0 && r / lam < best) best = r / lam;
  }
  return o->prm.cfl * 3.0 / (2.0 * o->p + 1.0) * best;
}

/* ==================================================================== API */
void orc_destroy(orc *o);

orc *orc_create(int32_t nn, int32_t ne, const double *xy, const int32_t *tri, int32_t nb,
                const int32_t *bedge, const int32_t *btype, const double *hb, const orc_params *prm,
                const double *init_nodal, const double *init_modal, double t0) {
  if (nn <= 0 || ne <= 0 || !xy || !tri || !hb || !prm) return NULL;
  if (prm->p < 1 || prm->p > 2) return NULL;
  {
    double a[8], b[8], c[8];
    int st = rk_table(prm, a, b, c);
    if (st < 2) return NULL;
  }
  orc *o = calloc(1, sizeof(orc));
  o->prm = *prm;
  o->p = prm->p;
  o->nn = nn; o->ne = ne;
  setup_tables(o);
  o->x = malloc(sizeof(double) * nn); o->y = malloc(sizeof(double) * nn); o->hb = malloc(sizeof(double) * nn);
  for (int n = 0; n < nn; ++n) { o->x[n] = xy[2 * n]; o->y[n] = xy[2 * n + 1]; o->hb[n] = hb[n]; }
  o->tri = malloc(sizeof(int) * 3 * ne);
  for (int i = 0; i < 3 * ne; ++i) {
    if (tri[i] < 0 || tri[i] >= nn) { free(o->tri); o->tri = NULL; orc_destroy(o); return NULL; }
    o->tri[i] = tri[i];
  }
  if (build_geometry(o) || build_edges(o, nb, bedge, btype)) { orc_destroy(o); return NULL; }
  build_limiter_geometry(o);
  size_t n = (size_t)3 * o->nd * ne;
  o->U = calloc(3 * n, sizeof(double));
  o->RHS = calloc(n, sizeof(double));
  o->EDGE = calloc(3 * n, sizeof(double));
  o->WD = calloc(ne, 1);
  o->MEAN = calloc(3 * (size_t)ne, sizeof(double));
  o->TSX = calloc(nn, sizeof(double)); o->TSY = calloc(nn, sizeof(double)); o->PA = calloc(nn, sizeof(double));
  if (init_modal) {
    memcpy(o->U, init_modal, sizeof(double) * n);
  } else if (init_nodal) {
    /* linear interpolant of the nodal values, expressed in the Dubiner modes */
    for (int v = 0; v < 3; ++v)
      for (int e = 0; e < ne; ++e) {
        const int *t = o->tri + 3 * e;
        double f0 = init_nodal[(size_t)v * nn + t[0]], f1 = init_nodal[(size_t)v * nn + t[1]];
        double f2 = init_nodal[(size_t)v * nn + t[2]];
        o->U[UIX(o, 0, v, 0, e)] = (f0 + f1 + f2) / 3.0;
        o->U[UIX(o, 0, v, 1, e)] = 0.5 * (f1 - f0);
        o->U[UIX(o, 0, v, 2, e)] = (2.0 * f2 - f0 - f1) / 6.0;
      }
  }
  o->t0 = t0;
  o->nstep = 0;
  if (wetdry_on(o)) wetdry(o, 0);
  o->dt = prm->dt > 0.0 ? prm->dt : compute_dt(o);
  if (!(o->dt > 0.0) || !isfinite(o->dt)) { orc_destroy(o); return NULL; }
  /* physical coordinates of the area quadrature points (used by the test hooks) */
  o->QXY = malloc(sizeof(double) * 2 * (size_t)ne * o->nqa);
  o->QSRC = calloc(3 * (size_t)ne * o->nqa, sizeof(double));
  for (int e = 0; e < ne; ++e) {
    const int *t = o->tri + 3 * e;
    for (int i = 0; i < o->nqa; ++i) {
      double N[3];
      shape_p1(o->XQ[i], o->YQ[i], N);
      o->QXY[((size_t)e * o->nqa + i) * 2] = N[0] * o->x[t[0]] + N[1] * o->x[t[1]] + N[2] * o->x[t[2]];
      o->QXY[((size_t)e * o->nqa + i) * 2 + 1] = N[0] * o->y[t[0]] + N[1] * o->y[t[1]] + N[2] * o->y[t[2]];
    }
  }
  return o;
}

void orc_destroy(orc *o) {
  if (!o) return;
  void *ptrs[] = {o->x, o->y, o->hb, o->tri, o->NEDEL, o->LED, o->ENODE, o->ETYPE, o->NIEDN, o->EL_EDGE,
                  o->EN_X, o->EN_Y, o->ELEN, o->detJ, o->rx, o->ry, o->sx, o->sy, o->area, o->LIM_J,
                  o->LIM_A, o->U, o->RHS, o->EDGE, o->WD, o->TSX, o->TSY, o->PA, o->MEAN, o->QXY,
                  o->QSRC, o->BXY, o->BVAL, o->BLIST};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
  free(o);
}

int32_t orc_sizes(const orc *o, int32_t *out) {
  out[0] = o->nd; out[1] = o->nqa; out[2] = o->nqe; out[3] = o->ned; out[4] = o->nint;
  return 0;
}

void orc_step(orc *o, int32_t n) {
  for (int i = 0; i < n; ++i) ssprk_step(o);
}

/* The time step one stage at a time, for a domain split into parts (Sec. 5.3): each part advances
 * its own and ghost elements by one stage, then the ghost elements' states and wet/dry flags are
 * replaced by their owners' (orc_set_register, orc_set_flags) before the next stage.  orc_stage
 * returns the state buffer the stage wrote (0 at the last stage, which completes the step). */
int32_t orc_stage(orc *o) { return ssprk_stage(o); }

int32_t orc_stage_count(const orc *o) {
  double a[8], b[8], c[8];
  return rk_table(&o->prm, a, b, c);
}

/* state buffer r (0 = u^n, 1 and 2 the stage buffers) as [3][nd][ne] arrays */
void orc_get_register(const orc *o, int32_t r, double *ze, double *qx, double *qy) {
  size_t m = (size_t)o->nd * o->ne, n = 3 * m;
  const double *U = o->U + (size_t)r * n;
  memcpy(ze, U, sizeof(double) * m);
  memcpy(qx, U + m, sizeof(double) * m);
  memcpy(qy, U + 2 * m, sizeof(double) * m);
}

void orc_set_register(orc *o, int32_t r, const double *ze, const double *qx, const double *qy) {
  size_t m = (size_t)o->nd * o->ne, n = 3 * m;
  double *U = o->U + (size_t)r * n;
  memcpy(U, ze, sizeof(double) * m);
  memcpy(U + m, qx, sizeof(double) * m);
  memcpy(U + 2 * m, qy, sizeof(double) * m);
}

void orc_set_flags(orc *o, const unsigned char *f) { memcpy(o->WD, f, o->ne); }

/* state as [3][nd][ne] arrays (zeta, qx, qy) in the caller's element order */
void orc_get_state(const orc *o, double *ze, double *qx, double *qy) {
  size_t m = (size_t)o->nd * o->ne;
  memcpy(ze, o->U, sizeof(double) * m);
  memcpy(qx, o->U + m, sizeof(double) * m);
  memcpy(qy, o->U + 2 * m, sizeof(double) * m);
}

void orc_set_state(orc *o, const double *ze, const double *qx, const double *qy, double t) {
  size_t m = (size_t)o->nd * o->ne;
  memcpy(o->U, ze, sizeof(double) * m);
  memcpy(o->U + m, qx, sizeof(double) * m);
  memcpy(o->U + 2 * m, qy, sizeof(double) * m);
  o->t0 = t;
  o->nstep = 0;
  o->st_i = 0;
}

void orc_info(const orc *o, double *dt, double *t, int64_t *steps) {
  *dt = o->dt;
  *t = o->t0 + (double)o->nstep * o->dt;
  *steps = o->nstep;
}

/* Neumaier-compensated sums of |Omega_e| zeta_e,00 and |Omega_e| (zeta_e,00 + mean h_b) */
void orc_mass(const orc *o, double *mass, double *volume) {
  double s1 = 0, c1 = 0, s2 = 0, c2 = 0;
  for (int e = 0; e < o->ne; ++e) {
    const int *t = o->tri + 3 * e;
    double z = o->U[UIX(o, 0, 0, 0, e)];
    double a = o->area[e] * z;
    double b = o->area[e] * (z + (o->hb[t[0]] + o->hb[t[1]] + o->hb[t[2]]) / 3.0);
    double u = s1 + a;
    c1 += fabs(s1) >= fabs(a) ? (s1 - u) + a : (a - u) + s1;
    s1 = u;
    u = s2 + b;
    c2 += fabs(s2) >= fabs(b) ? (s2 - u) + b : (b - u) + s2;
    s2 = u;
  }
  *mass = s1 + c1;
  *volume = s2 + c2;
}

/* L_h(u^n) at time t with the current wet/dry flags: out is [3][nd][ne] */
void orc_rhs(orc *o, double t, double *out) {
  eval_L(o, 0, t);
  memcpy(out, o->RHS, sizeof(double) * 3 * (size_t)o->nd * o->ne);
}

void orc_apply_limiter(orc *o) { slope_limiter(o, 0); }
void orc_apply_wetdry(orc *o) { wetdry(o, 0); }

void orc_flags(const orc *o, unsigned char *out) { memcpy(out, o->WD, o->ne); }

/* nodal forcing at time t: out is [3][nn] = (tau_x/rho_w, tau_y/rho_w, (p_a - p_n)/rho_w) */
void orc_forcing(orc *o, double t, double *out) {
  wind(o, t);
  memcpy(out, o->TSX, sizeof(double) * o->nn);
  memcpy(out + o->nn, o->TSY, sizeof(double) * o->nn);
  memcpy(out + 2 * (size_t)o->nn, o->PA, sizeof(double) * o->nn);
}

/* the point numerical flux, for checking its properties directly */
void orc_numflux(const orc_params *P, const double *wi, const double *wo, double hb, double nx, double ny,
                 double *out) {
  num_flux(P, wi, wo, hb, nx, ny, out);
}

/* reference tables, for checking against closed forms */
void orc_basis(int32_t p, double xi, double eta, double *phi, double *dxi, double *deta) {
  dubiner(p, xi, eta, phi, dxi, deta);
}
int32_t orc_area_rule(int32_t p, double *xi, double *eta, double *w) {
  orc tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.p = p;
  setup_tables(&tmp);
  for (int i = 0; i < tmp.nqa; ++i) { xi[i] = tmp.XQ[i]; eta[i] = tmp.YQ[i]; w[i] = tmp.WQ[i]; }
  return tmp.nqa;
}
int32_t orc_high_rule(double *xi, double *eta, double *w) {
  orc tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.p = 1;
  setup_tables(&tmp);
  for (int i = 0; i < NHQ; ++i) { xi[i] = tmp.HXQ[i]; eta[i] = tmp.HYQ[i]; w[i] = tmp.HWQ[i]; }
  return NHQ;
}
int32_t orc_edge_rule(int32_t n, double *s, double *w) {
  gauss_legendre(n, s, w);
  return n;
}

/* test-only manufactured-solution hooks: an extra source at every area quadrature point and an
 * exact exterior state on every boundary edge, both from callbacks called once per stage */
void orc_set_mms(orc *o, orc_field_cb src, orc_field_cb bnd) {
  o->mms_src = src;
  o->mms_bnd = bnd;
  free(o->BXY); free(o->BVAL); free(o->BLIST);
  o->BXY = o->BVAL = NULL; o->BLIST = NULL; o->nbnd = 0;
  if (!bnd) return;
  int nb = 0;
  for (int L = 0; L < o->ned; ++L) nb += o->ETYPE[L] >= 0;
  o->nbnd = nb;
  o->BLIST = malloc(sizeof(int) * (nb > 0 ? nb : 1));
  o->BXY = malloc(sizeof(double) * 2 * (size_t)(nb > 0 ? nb : 1) * o->nqe);
  o->BVAL = calloc(3 * (size_t)(nb > 0 ? nb : 1) * o->nqe, sizeof(double));
  int b = 0;
  for (int L = 0; L < o->ned; ++L) {
    if (o->ETYPE[L] < 0) continue;
    o->BLIST[b] = L;
    for (int i = 0; i < o->nqe; ++i) {
      double s = o->SQ[i];
      int a = o->ENODE[2 * L], c = o->ENODE[2 * L + 1];
      o->BXY[((size_t)b * o->nqe + i) * 2] = 0.5 * (1.0 - s) * o->x[a] + 0.5 * (1.0 + s) * o->x[c];
      o->BXY[((size_t)b * o->nqe + i) * 2 + 1] = 0.5 * (1.0 - s) * o->y[a] + 0.5 * (1.0 + s) * o->y[c];
    }
    b++;
  }
}

/* test-only: boundary ghosts equal the interior trace (zero-gradient), so a uniform state has a
 * vanishing spatial operator and evolves by the time integrator alone */
void orc_set_transmissive(orc *o, int32_t on) { o->transmissive = on; }

/* L2 projection of a callback field onto the modes (high-order rule) */
void orc_project(orc *o, orc_field_cb f, double t) {
  int ne = o->ne;
  double *xy = malloc(sizeof(double) * 2 * (size_t)ne * NHQ), *val = malloc(sizeof(double) * 3 * (size_t)ne * NHQ);
  for (int e = 0; e < ne; ++e) {
    const int *tr = o->tri + 3 * e;
    for (int i = 0; i < NHQ; ++i) {
      double N[3];
      shape_p1(o->HXQ[i], o->HYQ[i], N);
      xy[((size_t)e * NHQ + i) * 2] = N[0] * o->x[tr[0]] + N[1] * o->x[tr[1]] + N[2] * o->x[tr[2]];
      xy[((size_t)e * NHQ + i) * 2 + 1] = N[0] * o->y[tr[0]] + N[1] * o->y[tr[1]] + N[2] * o->y[tr[2]];
    }
  }
  f(t, ne * NHQ, xy, val);
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < 3; ++v)
      for (int k = 0; k < o->nd; ++k) {
        double s = 0.0;
        for (int i = 0; i < NHQ; ++i) {
          double ph[MAXD], dx[MAXD], dy[MAXD];
          dubiner(o->p, o->HXQ[i], o->HYQ[i], ph, dx, dy);
          s += o->HWQ[i] * ph[k] * val[((size_t)e * NHQ + i) * 3 + v];
        }
        o->U[UIX(o, 0, v, k, e)] = s / o->NORM[k];
      }
  free(xy); free(val);
}

/* L2 norm over the domain of (w_h - f) per variable (high-order rule) */
void orc_l2err(orc *o, orc_field_cb f, double t, double *err) {
  int ne = o->ne;
  double *xy = malloc(sizeof(double) * 2 * (size_t)ne * NHQ), *val = malloc(sizeof(double) * 3 * (size_t)ne * NHQ);
  for (int e = 0; e < ne; ++e) {
    const int *tr = o->tri + 3 * e;
    for (int i = 0; i < NHQ; ++i) {
      double N[3];
      shape_p1(o->HXQ[i], o->HYQ[i], N);
      xy[((size_t)e * NHQ + i) * 2] = N[0] * o->x[tr[0]] + N[1] * o->x[tr[1]] + N[2] * o->x[tr[2]];
      xy[((size_t)e * NHQ + i) * 2 + 1] = N[0] * o->y[tr[0]] + N[1] * o->y[tr[1]] + N[2] * o->y[tr[2]];
    }
  }
  f(t, ne * NHQ, xy, val);
  double acc[3] = {0, 0, 0};
  for (int e = 0; e < ne; ++e)
    for (int i = 0; i < NHQ; ++i) {
      double ph[MAXD], dx[MAXD], dy[MAXD];
      dubiner(o->p, o->HXQ[i], o->HYQ[i], ph, dx, dy);
      for (int v = 0; v < 3; ++v) {
        double wh = 0.0;
        for (int k = 0; k < o->nd; ++k) wh += o->U[UIX(o, 0, v, k, e)] * ph[k];
        double d = wh - val[((size_t)e * NHQ + i) * 3 + v];
        acc[v] += o->HWQ[i] * o->detJ[e] * d * d;
      }
    }
  for (int v = 0; v < 3; ++v) err[v] = sqrt(acc[v]);
  free(xy); free(val);
}
