// partition.cu -- host-side domain decomposition for running one model on several GPUs (Sec. 5.3,
// where DG-SWEM splits the mesh among MPI ranks and exchanges the ghost elements' states with
// packElems / unpackElems, Listings code:mpi and code:pack).  Here:
//  - recursive coordinate bisection of the elements into parts of balanced size (the paper uses
//    METIS, which is not available here);
//  - the sub-mesh of one part: its own elements and two layers of ghost elements.  A part updates
//    its own elements and, redundantly, the first ghost layer, so that it holds every neighbour
//    mean its own elements' limiter needs; one exchange of ghost states and wet/dry flags per
//    Runge-Kutta stage then suffices;
//  - the exchange lists: for every other part, the own elements it needs and the ghost elements it
//    supplies, each in increasing global element index, so that one part's send list and its
//    peer's receive list name the same elements in the same order.
// No device work happens here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/dgswem.h"

namespace {

bool mesh_ok(const dgswem_mesh *m) {
  if (!m || m->n_nodes < 3 || m->n_elems < 1 || !m->xy || !m->tri || m->n_bedges < 0) return false;
  if (m->n_bedges > 0 && (!m->bedge || !m->bedge_type)) return false;
  for (long i = 0; i < 3L * m->n_elems; ++i)
    if (m->tri[i] < 0 || m->tri[i] >= m->n_nodes) return false;
  return true;
}

// Face neighbours of every element (-1 across a boundary edge), from sorted node pairs.
// Returns false for an edge shared by more than two elements.
bool face_neighbours(const dgswem_mesh *m, std::vector<int> &nbr) {
  const int ne = m->n_elems;
  struct Half {
    int lo, hi, e, l;
  };
  std::vector<Half> h(3 * (size_t)ne);
  for (int e = 0; e < ne; ++e)
    for (int l = 0; l < 3; ++l) {
      const int a = m->tri[3 * e + (l + 1) % 3], b = m->tri[3 * e + (l + 2) % 3];
      h[3 * (size_t)e + l] = {std::min(a, b), std::max(a, b), e, l};
    }
  std::sort(h.begin(), h.end(), [](const Half &x, const Half &y) {
    if (x.lo != y.lo) return x.lo < y.lo;
    if (x.hi != y.hi) return x.hi < y.hi;
    return x.e < y.e;
  });
  nbr.assign(3 * (size_t)ne, -1);
  for (size_t i = 0; i < h.size();) {
    size_t j = i + 1;
    while (j < h.size() && h[j].lo == h[i].lo && h[j].hi == h[i].hi) ++j;
    if (j - i > 2) return false;
    if (j - i == 2) {
      nbr[3 * (size_t)h[i].e + h[i].l] = h[i + 1].e;
      nbr[3 * (size_t)h[i + 1].e + h[i + 1].l] = h[i].e;
    }
    i = j;
  }
  return true;
}

// Recursive coordinate bisection of ids[lo, hi) into parts [p0, p0 + np): split across the longer
// extent of the centroids, at the element count proportional to the two halves' part counts;
// equal coordinates are ordered by element index, so the result is deterministic.
void rcb(std::vector<int> &ids, int lo, int hi, int p0, int np, const std::vector<double> &cx,
         const std::vector<double> &cy, int32_t *part) {
  if (np == 1) {
    for (int i = lo; i < hi; ++i) part[ids[i]] = p0;
    return;
  }
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int i = lo; i < hi; ++i) {
    xmin = std::min(xmin, cx[ids[i]]);
    xmax = std::max(xmax, cx[ids[i]]);
    ymin = std::min(ymin, cy[ids[i]]);
    ymax = std::max(ymax, cy[ids[i]]);
  }
  const std::vector<double> &c = (xmax - xmin >= ymax - ymin) ? cx : cy;
  const int kl = np / 2;
  const int nl = (int)((long long)(hi - lo) * kl / np);
  std::nth_element(ids.begin() + lo, ids.begin() + lo + nl, ids.begin() + hi, [&](int a, int b) {
    return c[a] < c[b] || (c[a] == c[b] && a < b);
  });
  rcb(ids, lo, lo + nl, p0, kl, cx, cy, part);
  rcb(ids, lo + nl, hi, p0 + kl, np - kl, cx, cy, part);
}

// Everything one part needs, in the orders the ABI promises.
struct PartPlan {
  std::vector<int> elems;   // local -> global element, increasing
  std::vector<int> cls;     // 0 own, 1 first ghost layer, 2 second
  std::vector<int> nodes;   // local -> global node, increasing
  std::vector<int> bedges;  // global boundary-edge entries kept
  std::vector<int> peers;
  std::vector<std::vector<int>> send, recv;  // per peer: local element indices
};

int plan_part(const dgswem_mesh *m, const int32_t *part, int n_parts, int rank, PartPlan &P) {
  if (!mesh_ok(m) || !part || n_parts < 1 || rank < 0 || rank >= n_parts) return DGSWEM_EINVAL;
  const int ne = m->n_elems;
  for (int e = 0; e < ne; ++e)
    if (part[e] < 0 || part[e] >= n_parts) return DGSWEM_EINVAL;
  std::vector<int> nbr;
  if (!face_neighbours(m, nbr)) return DGSWEM_EMESH;
  // distance class with respect to this part's elements: 0 own, 1, 2, or 3 (not needed)
  std::vector<int> dist(ne, 3);
  for (int e = 0; e < ne; ++e)
    if (part[e] == rank) dist[e] = 0;
  for (int d = 1; d <= 2; ++d)
    for (int e = 0; e < ne; ++e)
      if (dist[e] == d - 1)
        for (int l = 0; l < 3; ++l) {
          const int j = nbr[3 * (size_t)e + l];
          if (j >= 0 && dist[j] > d) dist[j] = d;
        }
  P = PartPlan{};
  std::vector<int> local(ne, -1);
  for (int e = 0; e < ne; ++e)
    if (dist[e] <= 2) {
      local[e] = (int)P.elems.size();
      P.elems.push_back(e);
      P.cls.push_back(dist[e]);
    }
  if (std::find(P.cls.begin(), P.cls.end(), 0) == P.cls.end()) return DGSWEM_EINVAL;  // empty part
  std::vector<char> used(m->n_nodes, 0);
  for (int e : P.elems)
    for (int a = 0; a < 3; ++a) used[m->tri[3 * e + a]] = 1;
  for (int n = 0; n < m->n_nodes; ++n)
    if (used[n]) P.nodes.push_back(n);
  // boundary-edge entries whose edge bounds a local element
  std::vector<std::pair<int, int>> keys;
  keys.reserve(3 * P.elems.size());
  for (int e : P.elems)
    for (int l = 0; l < 3; ++l) {
      const int x = m->tri[3 * (size_t)e + (l + 1) % 3], y = m->tri[3 * (size_t)e + (l + 2) % 3];
      keys.emplace_back(std::min(x, y), std::max(x, y));
    }
  std::sort(keys.begin(), keys.end());
  for (int b = 0; b < m->n_bedges; ++b) {
    const int a0 = m->bedge[2 * b], a1 = m->bedge[2 * b + 1];
    if (a0 < 0 || a1 < 0 || a0 >= m->n_nodes || a1 >= m->n_nodes) return DGSWEM_EMESH;
    if (std::binary_search(keys.begin(), keys.end(), std::make_pair(std::min(a0, a1), std::max(a0, a1))))
      P.bedges.push_back(b);
  }
  // exchange lists.  Receive: the ghosts, by owner.  Send: an own element goes to every other
  // part that has an element within two face steps of it (it is a ghost there).
  std::vector<std::vector<int>> send(n_parts), recv(n_parts);
  for (size_t i = 0; i < P.elems.size(); ++i) {
    const int e = P.elems[i];
    if (P.cls[i] != 0) {
      recv[part[e]].push_back((int)i);
      continue;
    }
    std::vector<int> near;
    for (int l = 0; l < 3; ++l) {
      const int j = nbr[3 * (size_t)e + l];
      if (j < 0) continue;
      near.push_back(part[j]);
      for (int k = 0; k < 3; ++k) {
        const int jj = nbr[3 * (size_t)j + k];
        if (jj >= 0) near.push_back(part[jj]);
      }
    }
    std::sort(near.begin(), near.end());
    near.erase(std::unique(near.begin(), near.end()), near.end());
    for (int q : near)
      if (q != rank) send[q].push_back((int)i);
  }
  for (int q = 0; q < n_parts; ++q)
    if (!send[q].empty() || !recv[q].empty()) {
      P.peers.push_back(q);
      P.send.push_back(send[q]);  // local indices increase with the global index
      P.recv.push_back(recv[q]);
    }
  return 0;
}

}  // namespace

extern "C" {

int dgswem_partition_rcb(const dgswem_mesh *mesh, int32_t n_parts, int32_t *part) {
  if (!mesh_ok(mesh) || !part || n_parts < 1 || n_parts > mesh->n_elems) return DGSWEM_EINVAL;
  const int ne = mesh->n_elems;
  std::vector<double> cx(ne), cy(ne);
  for (int e = 0; e < ne; ++e) {
    const int32_t *t = mesh->tri + 3 * (size_t)e;
    cx[e] = (mesh->xy[2 * t[0]] + mesh->xy[2 * t[1]] + mesh->xy[2 * t[2]]) / 3.0;
    cy[e] = (mesh->xy[2 * t[0] + 1] + mesh->xy[2 * t[1] + 1] + mesh->xy[2 * t[2] + 1]) / 3.0;
  }
  std::vector<int> ids(ne);
  std::iota(ids.begin(), ids.end(), 0);
  rcb(ids, 0, ne, 0, n_parts, cx, cy, part);
  return DGSWEM_OK;
}

int dgswem_part_sizes(const dgswem_mesh *mesh, const int32_t *part, int32_t n_parts, int32_t rank,
                      dgswem_part_counts *sizes) {
  if (!sizes) return DGSWEM_EINVAL;
  PartPlan P;
  if (int r = plan_part(mesh, part, n_parts, rank, P)) return r;
  dgswem_part_counts &s = *sizes;
  std::memset(&s, 0, sizeof(s));
  s.n_nodes = (int32_t)P.nodes.size();
  s.n_elems = (int32_t)P.elems.size();
  s.n_bedges = (int32_t)P.bedges.size();
  for (int c : P.cls) (c == 0 ? s.n_own : c == 1 ? s.n_ghost1 : s.n_ghost2)++;
  s.n_peers = (int32_t)P.peers.size();
  for (size_t k = 0; k < P.peers.size(); ++k) {
    s.n_send += (int32_t)P.send[k].size();
    s.n_recv += (int32_t)P.recv[k].size();
  }
  return DGSWEM_OK;
}

int dgswem_part_build(const dgswem_mesh *mesh, const double *bathy, const int32_t *part, int32_t n_parts,
                      int32_t rank, const dgswem_part_out *out) {
  if (!bathy || !out || !out->xy || !out->tri || !out->bathy || !out->elem_global || !out->elem_class ||
      !out->node_global || !out->peer || !out->send_count || !out->recv_count)
    return DGSWEM_EINVAL;
  PartPlan P;
  if (int r = plan_part(mesh, part, n_parts, rank, P)) return r;
  if (!P.bedges.empty() && (!out->bedge || !out->bedge_type)) return DGSWEM_EINVAL;
  std::vector<int> lnode(mesh->n_nodes, -1);
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    const int n = P.nodes[i];
    lnode[n] = (int)i;
    out->xy[2 * i] = mesh->xy[2 * n];
    out->xy[2 * i + 1] = mesh->xy[2 * n + 1];
    out->bathy[i] = bathy[n];
    out->node_global[i] = n;
  }
  for (size_t i = 0; i < P.elems.size(); ++i) {
    const int e = P.elems[i];
    for (int a = 0; a < 3; ++a) out->tri[3 * i + a] = lnode[mesh->tri[3 * (size_t)e + a]];
    out->elem_global[i] = e;
    out->elem_class[i] = P.cls[i];
  }
  for (size_t i = 0; i < P.bedges.size(); ++i) {
    const int b = P.bedges[i];
    out->bedge[2 * i] = lnode[mesh->bedge[2 * b]];
    out->bedge[2 * i + 1] = lnode[mesh->bedge[2 * b + 1]];
    out->bedge_type[i] = mesh->bedge_type[b];
  }
  size_t ks = 0, kr = 0;
  for (size_t k = 0; k < P.peers.size(); ++k) {
    out->peer[k] = P.peers[k];
    out->send_count[k] = (int32_t)P.send[k].size();
    out->recv_count[k] = (int32_t)P.recv[k].size();
    if ((!P.send[k].empty() && !out->send_elems) || (!P.recv[k].empty() && !out->recv_elems)) return DGSWEM_EINVAL;
    for (int i : P.send[k]) out->send_elems[ks++] = i;
    for (int i : P.recv[k]) out->recv_elems[kr++] = i;
  }
  return DGSWEM_OK;
}

}  // extern "C"
