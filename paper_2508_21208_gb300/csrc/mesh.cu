// mesh.cu -- host-side mesh preprocessing and reference tables (run once per context).
//
// Builds, from a counter-clockwise triangle list, what the element/edge kernels index: the edge
// list with both adjacent elements and their local edge numbers (the paper's NEDEL / LED arrays,
// Alg. 2), element-to-edge and element-to-neighbour maps (so every edge contribution is gathered
// by its owning element in a fixed order, without atomics, cf. Alg. 3), boundary tags, the
// Cockburn-Shu limiter geometry, and a Hilbert-curve relabelling of the elements for locality.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace dg {
namespace {

struct HalfEdge {
  int lo, hi, e, l, a, b;
};

// Hilbert index of (x, y) on a 2^16 x 2^16 grid (classic rotate-and-reflect walk).
uint64_t hilbert_index(uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
    uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = (s - 1) - (x & (s - 1)) + (x & ~(s - 1));
        y = (s - 1) - (y & (s - 1)) + (y & ~(s - 1));
      }
      std::swap(x, y);
    }
  }
  return d;
}

}  // namespace

int preprocess_mesh(const dgswem_mesh &m, const double *bathy, bool hilbert, HostMesh &H,
                    std::string &msg, const int32_t *elem_class) {
  const int nn = m.n_nodes, ne = m.n_elems;
  if (nn < 3 || ne < 1 || !m.xy || !m.tri || !bathy || m.n_bedges < 0 ||
      (m.n_bedges > 0 && (!m.bedge || !m.bedge_type))) {
    msg = "mesh: null pointer or empty mesh";
    return DGSWEM_EINVAL;
  }
  for (int i = 0; i < nn; ++i)
    if (!std::isfinite(m.xy[2 * i]) || !std::isfinite(m.xy[2 * i + 1]) || !std::isfinite(bathy[i])) {
      msg = "mesh: non-finite node coordinate or bathymetry at node " + std::to_string(i);
      return DGSWEM_EINVAL;
    }
  for (long i = 0; i < 3L * ne; ++i)
    if (m.tri[i] < 0 || m.tri[i] >= nn) {
      msg = "mesh: node index out of range in triangle " + std::to_string(i / 3);
      return DGSWEM_EMESH;
    }
  // ---- element order
  H.ne = ne;
  H.nn = nn;
  H.nown = H.nact = ne;
  if (elem_class) {
    int cnt[3] = {0, 0, 0};
    for (int e = 0; e < ne; ++e) {
      if (elem_class[e] < 0 || elem_class[e] > 2) {
        msg = "mesh: element class must be 0 (own), 1 or 2 (ghost layers)";
        return DGSWEM_EINVAL;
      }
      cnt[elem_class[e]]++;
    }
    if (cnt[0] < 1) {
      msg = "mesh: a part needs at least one own element";
      return DGSWEM_EINVAL;
    }
    H.nown = cnt[0];
    H.nact = cnt[0] + cnt[1];
  }
  H.perm.resize(ne);
  std::iota(H.perm.begin(), H.perm.end(), 0);
  if (hilbert) {
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int i = 0; i < nn; ++i) {
      xmin = std::min(xmin, m.xy[2 * i]); xmax = std::max(xmax, m.xy[2 * i]);
      ymin = std::min(ymin, m.xy[2 * i + 1]); ymax = std::max(ymax, m.xy[2 * i + 1]);
    }
    double sx = 65535.0 / std::max(xmax - xmin, 1e-300), sy = 65535.0 / std::max(ymax - ymin, 1e-300);
    std::vector<uint64_t> key(ne);
    for (int e = 0; e < ne; ++e) {
      const int *t = m.tri + 3 * e;
      double cx = (m.xy[2 * t[0]] + m.xy[2 * t[1]] + m.xy[2 * t[2]]) / 3.0;
      double cy = (m.xy[2 * t[0] + 1] + m.xy[2 * t[1] + 1] + m.xy[2 * t[2] + 1]) / 3.0;
      key[e] = hilbert_index((uint32_t)((cx - xmin) * sx), (uint32_t)((cy - ymin) * sy));
    }
    std::stable_sort(H.perm.begin(), H.perm.end(), [&](int a, int b) { return key[a] < key[b]; });
  }
  if (elem_class)  // own, then ghost layer 1, then 2 (stable: Hilbert order within each class)
    std::stable_sort(H.perm.begin(), H.perm.end(), [&](int a, int b) { return elem_class[a] < elem_class[b]; });
  H.iperm.assign(ne, 0);
  for (int i = 0; i < ne; ++i) H.iperm[H.perm[i]] = i;
  // ---- vertices and geometry (internal order)
  H.vnode.assign(3 * (size_t)ne, 0);
  H.geo.assign(NGEO * (size_t)ne, 0.0);
  H.hbv.assign(3 * (size_t)ne, 0.0);
  H.area.assign(ne, 0.0);
  H.inradius.assign(ne, 0.0);
  H.nodexy.resize(2 * (size_t)nn);
  for (int i = 0; i < nn; ++i) {
    H.nodexy[i] = m.xy[2 * i];
    H.nodexy[nn + i] = m.xy[2 * i + 1];
  }
  auto X = [&](int n) { return m.xy[2 * n]; };
  auto Y = [&](int n) { return m.xy[2 * n + 1]; };
  for (int e = 0; e < ne; ++e) {
    const int *t = m.tri + 3 * H.perm[e];
    for (int a = 0; a < 3; ++a) {
      H.vnode[(size_t)a * ne + e] = t[a];
      H.hbv[(size_t)a * ne + e] = bathy[t[a]];
    }
    // x(xi, eta) = -(xi+eta)/2 x0 + (1+xi)/2 x1 + (1+eta)/2 x2
    double xr = 0.5 * (X(t[1]) - X(t[0])), xs = 0.5 * (X(t[2]) - X(t[0]));
    double yr = 0.5 * (Y(t[1]) - Y(t[0])), ys = 0.5 * (Y(t[2]) - Y(t[0]));
    double J = xr * ys - xs * yr;
    if (!(J > 0.0) || !std::isfinite(J)) {
      msg = "mesh: triangle " + std::to_string(H.perm[e]) + " is clockwise or degenerate";
      return DGSWEM_EMESH;
    }
    double *g = H.geo.data();
    g[GEO_RX * (size_t)ne + e] = ys / J;
    g[GEO_RY * (size_t)ne + e] = -xs / J;
    g[GEO_SX * (size_t)ne + e] = -yr / J;
    g[GEO_SY * (size_t)ne + e] = xr / J;
    g[GEO_DETJ * (size_t)ne + e] = J;
    double per = 0.0;
    for (int l = 0; l < 3; ++l) {
      int a = t[(l + 1) % 3], b = t[(l + 2) % 3];
      double tx = X(b) - X(a), ty = Y(b) - Y(a), L = std::sqrt(tx * tx + ty * ty);
      g[(GEO_NX0 + l) * (size_t)ne + e] = ty / L;
      g[(GEO_NY0 + l) * (size_t)ne + e] = -tx / L;
      g[(GEO_HL0 + l) * (size_t)ne + e] = 0.5 * L;
      per += L;
    }
    H.area[e] = 2.0 * J;
    H.inradius[e] = 2.0 * H.area[e] / per;
  }
  // ---- edges
  std::vector<HalfEdge> he(3 * (size_t)ne);
  for (int e = 0; e < ne; ++e)
    for (int l = 0; l < 3; ++l) {
      int a = H.vnode[(size_t)((l + 1) % 3) * ne + e], b = H.vnode[(size_t)((l + 2) % 3) * ne + e];
      he[3 * (size_t)e + l] = HalfEdge{std::min(a, b), std::max(a, b), e, l, a, b};
    }
  std::sort(he.begin(), he.end(), [](const HalfEdge &p, const HalfEdge &q) {
    if (p.lo != q.lo) return p.lo < q.lo;
    if (p.hi != q.hi) return p.hi < q.hi;
    return p.e < q.e;
  });
  struct BKey { int lo, hi, type; };
  std::vector<BKey> bk(m.n_bedges);
  for (int i = 0; i < m.n_bedges; ++i) {
    int a = m.bedge[2 * i], b = m.bedge[2 * i + 1];
    if (a < 0 || a >= nn || b < 0 || b >= nn) {
      msg = "mesh: boundary edge " + std::to_string(i) + " has a node index out of range";
      return DGSWEM_EMESH;
    }
    int ty = m.bedge_type[i];
    if (ty != DGSWEM_BC_LAND && ty != DGSWEM_BC_OPEN && ty != DGSWEM_BC_RIVER) {
      msg = "mesh: unknown boundary type at boundary edge " + std::to_string(i);
      return DGSWEM_EINVAL;
    }
    bk[i] = BKey{std::min(a, b), std::max(a, b), ty};
  }
  std::sort(bk.begin(), bk.end(), [](const BKey &p, const BKey &q) {
    return p.lo != q.lo ? p.lo < q.lo : p.hi < q.hi;
  });
  std::vector<char> bused(bk.size(), 0);
  H.nbr.assign(3 * (size_t)ne, NBR_LAND);
  H.nle.assign(ne, 0);
  H.eledge.assign(3 * (size_t)ne, -1);
  struct IEdge { int ep, lp, em, lm, a, b; };
  std::vector<IEdge> ie;
  ie.reserve(3 * (size_t)ne / 2 + 1);
  int nbnd = 0;
  for (size_t i = 0; i < he.size();) {
    size_t j = i + 1;
    while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
    if (j - i > 2) {
      msg = "mesh: edge (" + std::to_string(he[i].lo) + "," + std::to_string(he[i].hi) +
            ") is shared by more than two triangles";
      return DGSWEM_EMESH;
    }
    const HalfEdge &P = he[i];
    if (j - i == 2) {
      const HalfEdge &M = he[i + 1];
      if (!(P.a == M.b && P.b == M.a)) {
        msg = "mesh: triangles " + std::to_string(H.perm[P.e]) + " and " + std::to_string(H.perm[M.e]) +
              " have inconsistent orientation";
        return DGSWEM_EMESH;
      }
      ie.push_back(IEdge{P.e, P.l, M.e, M.l, P.a, P.b});
    } else {
      ++nbnd;
      BKey key{P.lo, P.hi, 0};
      auto it = std::lower_bound(bk.begin(), bk.end(), key, [](const BKey &p, const BKey &q) {
        return p.lo != q.lo ? p.lo < q.lo : p.hi < q.hi;
      });
      int ty = DGSWEM_BC_LAND;
      if (it != bk.end() && it->lo == P.lo && it->hi == P.hi) {
        ty = it->type;
        bused[it - bk.begin()] = 1;
      }
      H.nbr[(size_t)P.l * ne + P.e] = (ty == DGSWEM_BC_OPEN) ? NBR_OPEN : (ty == DGSWEM_BC_RIVER ? NBR_RIVER : NBR_LAND);
    }
    i = j;
  }
  for (size_t i = 0; i < bk.size(); ++i)
    if (!bused[i]) {
      // a listed pair that is not a boundary edge (interior or absent)
      bool dup = i > 0 && bk[i].lo == bk[i - 1].lo && bk[i].hi == bk[i - 1].hi;
      if (!dup) {
        msg = "mesh: listed boundary edge (" + std::to_string(bk[i].lo) + "," + std::to_string(bk[i].hi) +
              ") is not a boundary edge of the triangulation";
        return DGSWEM_EMESH;
      }
    }
  // interior edges sorted by their plus element so that an edge block touches nearby elements
  std::stable_sort(ie.begin(), ie.end(), [](const IEdge &p, const IEdge &q) {
    return std::min(p.ep, p.em) < std::min(q.ep, q.em);
  });
  const int nint = (int)ie.size();
  H.nint = nint;
  H.nbnd = nbnd;
  H.edel.assign(2 * (size_t)nint, 0);
  H.edle.assign(nint, 0);
  H.edgeo.assign(3 * (size_t)nint, 0.0);
  H.edhb.assign(2 * (size_t)nint, 0.0);
  for (int d = 0; d < nint; ++d) {
    IEdge E = ie[d];
    if (E.em < E.ep) {  // the lower internal index is the plus side
      std::swap(E.ep, E.em);
      std::swap(E.lp, E.lm);
      std::swap(E.a, E.b);
    }
    H.edel[d] = E.ep;
    H.edel[nint + d] = E.em;
    H.edle[d] = (uint8_t)(E.lp | (E.lm << 2));
    double tx = X(E.b) - X(E.a), ty = Y(E.b) - Y(E.a), L = std::sqrt(tx * tx + ty * ty);
    H.edgeo[d] = ty / L;
    H.edgeo[nint + d] = -tx / L;
    H.edgeo[2 * (size_t)nint + d] = 0.5 * L;
    H.edhb[d] = bathy[E.a];
    H.edhb[nint + d] = bathy[E.b];
    H.nbr[(size_t)E.lp * ne + E.ep] = E.em;
    H.nbr[(size_t)E.lm * ne + E.em] = E.ep;
    H.nle[E.ep] |= (uint8_t)(E.lm << (2 * E.lp));
    H.nle[E.em] |= (uint8_t)(E.lp << (2 * E.lm));
    H.eledge[(size_t)E.lp * ne + E.ep] = d;
    H.eledge[(size_t)E.lm * ne + E.em] = d | (int)0x80000000u;
  }
  // ---- limiter geometry: m_i - b0 = a1 (b_j1 - b0) + a2 (b_j2 - b0) with a1, a2 >= 0, where b_j
  // is the barycentre across local edge j (mirror image of b0 in a boundary edge); pairs are
  // tried in the order (i, i+1), (i+2, i), (i+1, i+2).
  H.lima.assign(6 * (size_t)ne, 0.0);
  H.limj.assign(ne, 0);
  auto centroid = [&](int e, double &cx, double &cy) {
    int a = H.vnode[e], b = H.vnode[(size_t)ne + e], c = H.vnode[2 * (size_t)ne + e];
    cx = (X(a) + X(b) + X(c)) / 3.0;
    cy = (Y(a) + Y(b) + Y(c)) / 3.0;
  };
  for (int e = 0; e < ne; ++e) {
    double b0x, b0y, bx[3], by[3], mx[3], my[3];
    centroid(e, b0x, b0y);
    for (int j = 0; j < 3; ++j) {
      int a = H.vnode[(size_t)((j + 1) % 3) * ne + e], b = H.vnode[(size_t)((j + 2) % 3) * ne + e];
      mx[j] = 0.5 * (X(a) + X(b));
      my[j] = 0.5 * (Y(a) + Y(b));
      int nb = H.nbr[(size_t)j * ne + e];
      if (nb >= 0) {
        centroid(nb, bx[j], by[j]);
      } else {
        double tx = X(b) - X(a), ty = Y(b) - Y(a);
        double s = ((b0x - X(a)) * tx + (b0y - Y(a)) * ty) / (tx * tx + ty * ty);
        bx[j] = 2.0 * (X(a) + s * tx) - b0x;
        by[j] = 2.0 * (Y(a) + s * ty) - b0y;
      }
    }
    uint16_t code = 0;
    for (int i = 0; i < 3; ++i) {
      const int pairs[3][2] = {{i, (i + 1) % 3}, {(i + 2) % 3, i}, {(i + 1) % 3, (i + 2) % 3}};
      int j1 = 3, j2 = 3;
      double a1 = 0.0, a2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        int p1 = pairs[c][0], p2 = pairs[c][1];
        double d1x = bx[p1] - b0x, d1y = by[p1] - b0y, d2x = bx[p2] - b0x, d2y = by[p2] - b0y;
        double rx = mx[i] - b0x, ry = my[i] - b0y;
        double det = d1x * d2y - d2x * d1y;
        if (det == 0.0) continue;
        double c1 = (rx * d2y - d2x * ry) / det, c2 = (d1x * ry - rx * d1y) / det;
        if (c1 >= -1e-10 && c2 >= -1e-10) {
          j1 = p1; j2 = p2; a1 = c1; a2 = c2;
          break;
        }
      }
      code |= (uint16_t)((j1 | (j2 << 2)) << (4 * i));
      H.lima[(size_t)(2 * i) * ne + e] = a1;
      H.lima[(size_t)(2 * i + 1) * ne + e] = a2;
    }
    H.limj[e] = code;
  }
  return 0;
}

void build_tile_edges(const HostMesh &H, int tile, TileEdges &T) {
  const int ne = H.ne, nint = H.nint, nact = H.nact;
  T.tile = tile;
  T.ntiles = (nact + tile - 1) / tile;  // tiles cover the updated elements [0, nact)
  std::vector<int> count(T.ntiles + 1, 0);
  auto tile_of = [&](int e) { return e < nact ? e / tile : -1; };  // -1: not updated here
  for (int d = 0; d < nint; ++d) {
    const int ta = tile_of(H.edel[d]), tb = tile_of(H.edel[nint + d]);
    if (ta >= 0) count[ta]++;
    if (tb >= 0 && tb != ta) count[tb]++;
  }
  for (int l = 0; l < 3; ++l)
    for (int e = 0; e < nact; ++e)
      if (H.nbr[(size_t)l * ne + e] < 0) count[tile_of(e)]++;
  T.start.assign(T.ntiles + 1, 0);
  for (int t = 0; t < T.ntiles; ++t) T.start[t + 1] = T.start[t] + count[t];
  T.n = T.start[T.ntiles];
  T.ea.assign(T.n, 0);
  T.eb.assign(T.n, 0);
  T.code.assign(T.n, 0);
  T.geo.assign(3 * (size_t)T.n, 0.0);
  T.hb.assign(2 * (size_t)T.n, 0.0);
  std::vector<int> fill(T.start.begin(), T.start.end() - 1);
  auto put = [&](int t, int a, int b, int la, int lb, bool ina, bool inb, double nx, double ny, double hl, double ha,
                 double hbb) {
    const int i = fill[t]++;
    T.ea[i] = a;
    T.eb[i] = b;
    T.code[i] = (uint8_t)(la | (lb << 2) | ((ina ? 1 : 0) << 4) | ((inb ? 1 : 0) << 5));
    T.geo[i] = nx;
    T.geo[(size_t)T.n + i] = ny;
    T.geo[2 * (size_t)T.n + i] = hl;
    T.hb[i] = ha;
    T.hb[(size_t)T.n + i] = hbb;
  };
  for (int d = 0; d < nint; ++d) {
    const int a = H.edel[d], b = H.edel[nint + d];
    const int la = H.edle[d] & 3, lb = H.edle[d] >> 2;
    const double nx = H.edgeo[d], ny = H.edgeo[nint + d], hl = H.edgeo[2 * (size_t)nint + d];
    const double ha = H.edhb[d], hbb = H.edhb[nint + d];
    const int ta = tile_of(a), tb = tile_of(b);
    if (ta >= 0 && ta == tb) {
      put(ta, a, b, la, lb, true, true, nx, ny, hl, ha, hbb);
    } else {
      if (ta >= 0) put(ta, a, b, la, lb, true, false, nx, ny, hl, ha, hbb);
      if (tb >= 0) put(tb, a, b, la, lb, false, true, nx, ny, hl, ha, hbb);
    }
  }
  const double *g = H.geo.data();
  for (int e = 0; e < nact; ++e)
    for (int l = 0; l < 3; ++l) {
      const int code = H.nbr[(size_t)l * ne + e];
      if (code >= 0) continue;
      // end nodes of local edge l: vertices (l+1)%3 and (l+2)%3
      const double ha = H.hbv[(size_t)((l + 1) % 3) * ne + e], hbb = H.hbv[(size_t)((l + 2) % 3) * ne + e];
      put(tile_of(e), e, code, l, 0, true, false, g[(GEO_NX0 + l) * (size_t)ne + e], g[(GEO_NY0 + l) * (size_t)ne + e],
          g[(GEO_HL0 + l) * (size_t)ne + e], ha, hbb);
    }
}

// ------------------------------------------------------------------ SSP Runge-Kutta tables
int rk_stage_table(const dgswem_params &p, double a[MAX_STAGES], double b[MAX_STAGES], double c[MAX_STAGES],
                   double tau[MAX_STAGES]) {
  int s = 0;
  auto st = [&](double x, double y, double z) {
    a[s] = x;
    b[s] = y;
    c[s] = z;
    ++s;
  };
  switch (p.rk_scheme) {
    case DGSWEM_RK_SSP22:  // Shu-Osher
      st(0.0, 1.0, 1.0);
      st(0.5, 0.5, 0.5);
      break;
    case DGSWEM_RK_SSP33:  // Shu-Osher
      st(0.0, 1.0, 1.0);
      st(0.75, 0.25, 0.25);
      st(1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0);
      break;
    case DGSWEM_RK_SSP32:
    case DGSWEM_RK_SSP42:
    case DGSWEM_RK_SSP52: {  // Ketcheson: s-1 Euler steps of dt/(s-1), then the average with u^n
      const int n = p.rk_scheme + 1;
      for (int i = 0; i < n - 1; ++i) st(0.0, 1.0, 1.0 / (n - 1));
      st(1.0 / n, (n - 1.0) / n, 1.0 / n);
      break;
    }
    case DGSWEM_RK_SSP43:  // Spiteri-Ruuth
      st(0.0, 1.0, 0.5);
      st(0.0, 1.0, 0.5);
      st(2.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0);
      st(0.0, 1.0, 0.5);
      break;
    case DGSWEM_RK_CUSTOM:
      if (p.rk_stages < 2 || p.rk_stages > MAX_STAGES) return 0;
      for (int i = 0; i < p.rk_stages; ++i) {
        const double *q = p.rk_coeffs + 3 * i;
        if (!std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2])) return 0;
        st(q[0], q[1], q[2]);
      }
      break;
    default:
      return 0;
  }
  double t = 0.0;  // stage i evaluates L at the time of its input u_(i-1)
  for (int i = 0; i < s; ++i) {
    tau[i] = t;
    t = b[i] * t + c[i];
  }
  return s;
}

void area_point_hb(int p, const HostMesh &H, std::vector<double> &out) {
  Tab<double> t;
  build_tables(p, t);
  const int nqa = nqa_of(p), ne = H.ne;
  out.assign((size_t)nqa * ne, 0.0);
  for (int q = 0; q < nqa; ++q)
    for (int e = 0; e < ne; ++e)
      out[(size_t)q * ne + e] = H.hbv[e] * t.nq[q][0] + H.hbv[(size_t)ne + e] * t.nq[q][1] +
                                H.hbv[2 * (size_t)ne + e] * t.nq[q][2];
}

void edge_point_hb(int p, const double *hA, const double *hB, int n, std::vector<double> &out) {
  Tab<double> t;
  build_tables(p, t);
  const int nqe = nqe_of(p);
  out.assign((size_t)nqe * n, 0.0);
  for (int q = 0; q < nqe; ++q)
    for (int x = 0; x < n; ++x) out[(size_t)q * n + x] = 0.5 * ((1.0 - t.se[q]) * hA[x] + (1.0 + t.se[q]) * hB[x]);
}

// ------------------------------------------------------------------ reference tables
// Dubiner basis (Sec. 2.2, Eq. dubiner) psi_ij = P_i(a) ((1-b)/2)^i P_j^(2i+1,0)(b), written out
// for i + j <= 2, with its reference gradient.
static void dubiner(double xi, double eta, double *v, double *dx, double *dy) {
  v[0] = 1.0; dx[0] = 0.0; dy[0] = 0.0;
  v[1] = xi + 0.5 * eta + 0.5; dx[1] = 1.0; dy[1] = 0.5;
  v[2] = 1.5 * eta + 0.5; dx[2] = 0.0; dy[2] = 1.5;
  v[3] = 1.5 * xi * xi + 1.5 * xi * eta + 1.5 * xi + 0.25 * eta * eta + eta + 0.25;
  dx[3] = 3.0 * xi + 1.5 * eta + 1.5; dy[3] = 1.5 * xi + 0.5 * eta + 1.0;
  v[4] = 2.5 * xi * eta + 1.5 * xi + 1.25 * eta * eta + 2.0 * eta + 0.75;
  dx[4] = 2.5 * eta + 1.5; dy[4] = 2.5 * xi + 2.5 * eta + 2.0;
  v[5] = 2.5 * eta * eta + eta - 0.5; dx[5] = 0.0; dy[5] = 5.0 * eta + 1.0;
}

void build_tables(int p, Tab<double> &t) {
  t = Tab<double>{};
  // Dunavant (1985) symmetric rules: degree 4 (6 points) for p = 1, degree 6 (12 points) for p = 2,
  // as barycentric orbits (a, a, 1-2a) and (a, b, 1-a-b) with weights summing to one.
  std::vector<std::array<double, 3>> pts;
  auto orbit3 = [&](double a, double w) {
    double b = 1.0 - 2.0 * a;
    pts.push_back({a, a, w}); pts.push_back({a, b, w}); pts.push_back({b, a, w});
  };
  auto orbit6 = [&](double a, double b, double w) {
    double c = 1.0 - a - b;
    pts.push_back({a, b, w}); pts.push_back({b, a, w}); pts.push_back({a, c, w});
    pts.push_back({c, a, w}); pts.push_back({b, c, w}); pts.push_back({c, b, w});
  };
  if (p == 1) {
    orbit3(0.445948490915965, 0.223381589678011);
    orbit3(0.091576213509771, 0.109951743655322);
  } else {
    orbit3(0.249286745170910, 0.116786275726379);
    orbit3(0.063089014491502, 0.050844906370207);
    orbit6(0.053145049844817, 0.310352451033784, 0.082851075618374);
  }
  const double V[3][2] = {{-1.0, -1.0}, {1.0, -1.0}, {-1.0, 1.0}};
  for (size_t q = 0; q < pts.size(); ++q) {
    double l1 = pts[q][0], l2 = pts[q][1], l0 = 1.0 - l1 - l2;
    double xi = l0 * V[0][0] + l1 * V[1][0] + l2 * V[2][0];
    double eta = l0 * V[0][1] + l1 * V[1][1] + l2 * V[2][1];
    t.wq[q] = 2.0 * pts[q][2];
    t.iwq[q] = 1.0 / t.wq[q];
    dubiner(xi, eta, t.phq[q], t.dxq[q], t.dyq[q]);
    t.nq[q][0] = -0.5 * (xi + eta);
    t.nq[q][1] = 0.5 * (1.0 + xi);
    t.nq[q][2] = 0.5 * (1.0 + eta);
  }
  // Gauss-Legendre: 2 points (exact to degree 3) for p = 1, 4 points (degree 7) for p = 2
  if (p == 1) {
    double s = 1.0 / std::sqrt(3.0);
    t.se[0] = -s; t.se[1] = s; t.we[0] = t.we[1] = 1.0;
  } else {
    double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    t.se[0] = -b; t.se[1] = -a; t.se[2] = a; t.se[3] = b;
    t.we[0] = wb; t.we[1] = wa; t.we[2] = wa; t.we[3] = wb;
  }
  const int nqe = nqe_of(p);
  for (int l = 0; l < 3; ++l) {
    int a = (l + 1) % 3, b = (l + 2) % 3;
    for (int g = 0; g < nqe; ++g) {
      double s = t.se[g];
      double xi = 0.5 * (1.0 - s) * V[a][0] + 0.5 * (1.0 + s) * V[b][0];
      double eta = 0.5 * (1.0 - s) * V[a][1] + 0.5 * (1.0 + s) * V[b][1];
      double dx[MAXD], dy[MAXD];
      dubiner(xi, eta, t.phe[l][g], dx, dy);
    }
    double v[MAXD], dx[MAXD], dy[MAXD];
    dubiner(0.5 * (V[a][0] + V[b][0]), 0.5 * (V[a][1] + V[b][1]), v, dx, dy);
    for (int k = 0; k < 3; ++k) t.phm[l][k] = v[k];
    dubiner(V[l][0], V[l][1], t.phv[l], dx, dy);
  }
  t.lim_idet = 1.0 / (t.phm[0][1] * t.phm[1][2] - t.phm[0][2] * t.phm[1][1]);
  const double nrm[MAXD] = {2.0, 1.0 / 3.0, 1.0, 2.0 / 15.0, 2.0 / 9.0, 2.0 / 3.0};
  for (int k = 0; k < MAXD; ++k) {
    t.nrm[k] = nrm[k];
    t.inrm[k] = 1.0 / nrm[k];
  }
}

}  // namespace dg
