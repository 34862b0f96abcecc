// Element-slab partition of a box mesh for runs with one rank per GPU
// (Sec. 2.2: NekRS runs one MPI rank per GPU and sums shared surface values
// across ranks, overlapping the exchange with interior work).
//
// Rank r of P owns the element planes ez in [r nelz / P, (r+1) nelz / P).
// Direct stiffness summation then splits into a rank-local part (every copy
// the rank holds) and an exchange of partial sums on the interface: the
// unique nodes that also belong to another rank, which for slabs are the
// lattice planes K = ez_boundary * N (and K = 0 = nelz N when z is periodic).
// Host code only: it computes the exchange plan without building l2g.
#include <algorithm>
#include <vector>

#include "sem_internal.h"

namespace {

struct Lattice {
  int64_t nx, ny, nz;  // unique extent per direction
  int64_t Kmax;        // lattice extent in z before periodic wrap (nelz N)
};

Lattice lattice(const sem_box_desc *d) {
  Lattice L;
  L.nx = (int64_t)d->nelx * d->N + (d->periodic[0] ? 0 : 1);
  L.ny = (int64_t)d->nely * d->N + (d->periodic[1] ? 0 : 1);
  L.nz = (int64_t)d->nelz * d->N + (d->periodic[2] ? 0 : 1);
  L.Kmax = (int64_t)d->nelz * d->N;
  return L;
}

int check(const sem_box_desc *d, int nranks, int rank) {
  if (!d) return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition: NULL description");
  if (d->N < 1 || d->N > SEM_MAXN || d->nelx < 1 || d->nely < 1 || d->nelz < 1)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition: bad mesh sizes");
  if (nranks < 1 || nranks > d->nelz || rank < 0 || rank >= nranks)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition: need 1 <= nranks <= nelz and 0 <= rank < nranks");
  return SEM_OK;
}

int ez_begin(const sem_box_desc *d, int nranks, int r) { return (int)((int64_t)r * d->nelz / nranks); }

// lattice z-planes K (before wrap) touched by rank r: [ez0 N, ez1 N]
void planes(const sem_box_desc *d, int nranks, int r, int64_t &k0, int64_t &k1) {
  k0 = (int64_t)ez_begin(d, nranks, r) * d->N;
  k1 = (int64_t)ez_begin(d, nranks, r + 1) * d->N;
}

int64_t wrapK(const sem_box_desc *d, const Lattice &L, int64_t K) {
  return (d->periodic[2] && K == L.Kmax) ? 0 : K;
}

// ranks (other than r) whose plane range contains wrapped plane Kw
std::vector<int> sharers(const sem_box_desc *d, int nranks, const Lattice &L, int64_t Kw, int r) {
  std::vector<int> out;
  for (int q = 0; q < nranks; ++q) {
    if (q == r) continue;
    int64_t a, b;
    planes(d, nranks, q, a, b);
    for (int64_t K = a; K <= b; ++K)
      if (wrapK(d, L, K) == Kw) {
        out.push_back(q);
        break;
      }
  }
  return out;
}

// the interface planes of rank r (wrapped K values shared with another rank), ascending
std::vector<int64_t> iface_planes(const sem_box_desc *d, int nranks, int r) {
  const Lattice L = lattice(d);
  int64_t k0, k1;
  planes(d, nranks, r, k0, k1);
  std::vector<int64_t> out;
  for (int64_t K : {k0, k1}) {
    const int64_t Kw = wrapK(d, L, K);
    if (!sharers(d, nranks, L, Kw, r).empty() && std::find(out.begin(), out.end(), Kw) == out.end())
      out.push_back(Kw);
  }
  std::sort(out.begin(), out.end());
  return out;
}

}  // namespace

extern "C" int sem_partition_info(const sem_box_desc *d, int nranks, int rank, int64_t *e_begin, int64_t *e_end,
                                  int64_t *n_interface) {
  if (int rc = check(d, nranks, rank)) return rc;
  const int64_t plane = (int64_t)d->nelx * d->nely;
  if (e_begin) *e_begin = ez_begin(d, nranks, rank) * plane;
  if (e_end) *e_end = ez_begin(d, nranks, rank + 1) * plane;
  if (n_interface) {
    const Lattice L = lattice(d);
    *n_interface = (int64_t)iface_planes(d, nranks, rank).size() * L.nx * L.ny;
  }
  return SEM_OK;
}

extern "C" int sem_partition_interface(const sem_box_desc *d, int nranks, int rank, int64_t *gids, int32_t *nshare) {
  if (int rc = check(d, nranks, rank)) return rc;
  if (!gids) return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition_interface: NULL output");
  const Lattice L = lattice(d);
  int64_t t = 0;
  for (int64_t Kw : iface_planes(d, nranks, rank)) {
    const int32_t ns = (int32_t)sharers(d, nranks, L, Kw, rank).size() + 1;
    for (int64_t J = 0; J < L.ny; ++J)
      for (int64_t I = 0; I < L.nx; ++I) {
        gids[t] = I + L.nx * (J + L.ny * Kw);
        if (nshare) nshare[t] = ns;
        ++t;
      }
  }
  return SEM_OK;
}

extern "C" int sem_partition_peers(const sem_box_desc *d, int nranks, int rank, int32_t *peers, int64_t *counts,
                                   int32_t *npeers) {
  if (int rc = check(d, nranks, rank)) return rc;
  if (!npeers) return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition_peers: NULL npeers");
  const Lattice L = lattice(d);
  std::vector<int64_t> per(nranks, 0);
  for (int64_t Kw : iface_planes(d, nranks, rank))
    for (int q : sharers(d, nranks, L, Kw, rank)) per[q] += L.nx * L.ny;
  int32_t n = 0;
  for (int q = 0; q < nranks; ++q) {
    if (per[q] == 0) continue;
    if (peers) peers[n] = q;
    if (counts) counts[n] = per[q];
    ++n;
  }
  *npeers = n;
  return SEM_OK;
}

extern "C" int sem_partition_peer_nodes(const sem_box_desc *d, int nranks, int rank, int peer, int64_t *gids) {
  if (int rc = check(d, nranks, rank)) return rc;
  if (peer < 0 || peer >= nranks || peer == rank)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition_peer_nodes: need 0 <= peer < nranks, peer != rank");
  if (!gids) return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition_peer_nodes: NULL output");
  const Lattice L = lattice(d);
  int64_t t = 0;
  for (int64_t Kw : iface_planes(d, nranks, rank)) {
    const std::vector<int> s = sharers(d, nranks, L, Kw, rank);
    if (std::find(s.begin(), s.end(), peer) == s.end()) continue;
    for (int64_t J = 0; J < L.ny; ++J)
      for (int64_t I = 0; I < L.nx; ++I) gids[t++] = I + L.nx * (J + L.ny * Kw);
  }
  return SEM_OK;
}

extern "C" int sem_partition_surface(const sem_box_desc *d, int nranks, int rank, int64_t *elems,
                                     int64_t *n_surface) {
  if (int rc = check(d, nranks, rank)) return rc;
  if (!n_surface) return sem_fail(SEM_ERR_INVALID_ARG, "sem_partition_surface: NULL n_surface");
  const Lattice L = lattice(d);
  const int ez0 = ez_begin(d, nranks, rank), ez1 = ez_begin(d, nranks, rank + 1);
  // element planes next to a shared lattice plane: the first one (plane ez0 N) and the last (ez1 N)
  std::vector<int> eplanes;
  if (!sharers(d, nranks, L, wrapK(d, L, (int64_t)ez0 * d->N), rank).empty()) eplanes.push_back(ez0);
  if (!sharers(d, nranks, L, wrapK(d, L, (int64_t)ez1 * d->N), rank).empty() &&
      (eplanes.empty() || eplanes.back() != ez1 - 1))
    eplanes.push_back(ez1 - 1);
  const int64_t plane = (int64_t)d->nelx * d->nely;
  int64_t t = 0;
  for (int ez : eplanes)
    for (int64_t i = 0; i < plane; ++i, ++t)
      if (elems) elems[t] = (int64_t)ez * plane + i;
  *n_surface = t;
  return SEM_OK;
}
