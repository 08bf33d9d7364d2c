// Domain decomposition of the uniform mesh over ranks (the paper's primary
// level of parallelism, Sec. 3.7: the FE mesh is partitioned into subdomains
// on separate tasks, and because every FE basis function is supported on the
// cells sharing its node, only the unknowns on subdomain boundaries are
// communicated).  Host logic only; every rank evaluates it independently and
// all ranks agree on every list.
//
// Partition: the ranks form a px x py x pz grid (the factorisation of nranks
// with the smallest total interface area, each factor at most the number of
// cells on its axis); rank (ix, iy, iz) = ix + px (iy + py iz) owns the cell
// block [ix n_x / px, (ix + 1) n_x / px) x ... .  For one rank:
//   cells  : its cells, ascending global cell index (cells x fastest);
//   l2g    : the global unknowns its cells touch, ascending (the local order);
//   owner  : per local unknown, the lowest rank whose cells touch it (the
//            rank that counts it in reductions over unknowns);
//   halo   : per neighbour rank q (ascending), the local indices of the
//            unknowns touched by q's cells as well, ascending in global
//            index -- the same order on both sides of the exchange.
#include <algorithm>
#include <array>
#include <cstdint>
#include <vector>

#include "../../include/chfsi.h"

namespace {

struct Grid {
  int n[3], p, per[3], P[3];
  int64_t nd[3];
};

// Cells along one axis that contain global node g (one, or two at a cell
// boundary; periodic axes wrap, Dirichlet axes have no cell outside).
int cells_of_node(const Grid& G, int a, int64_t g, int out[2]) {
  const int n = G.n[a], p = G.p;
  int k = 0;
  if (g % p == 0) {
    int64_t c1 = g / p, c0 = c1 - 1;
    if (G.per[a]) {
      c0 = (c0 + n) % n;
      c1 = c1 % n;
      out[k++] = (int)c0;
      if (c1 != c0) out[k++] = (int)c1;
    } else {
      if (c0 >= 0) out[k++] = (int)c0;
      if (c1 < n) out[k++] = (int)c1;
    }
  } else {
    out[k++] = (int)(g / p);
  }
  return k;
}

// Global node coordinate along axis a of unknown index u_a (Dirichlet axes
// skip node 0).
int64_t node_of_unknown(const Grid& G, int a, int64_t u) { return G.per[a] ? u : u + 1; }

int part_of_cell(const Grid& G, int a, int c) {
  // part k holds [k n / P, (k + 1) n / P)
  const int n = G.n[a], P = G.P[a];
  int k = (int)((int64_t)c * P / n);
  while ((int64_t)(k + 1) * n / P <= c) ++k;
  while ((int64_t)k * n / P > c) --k;
  return k;
}

bool make_grid(const chfsi_mesh_desc* d, int nranks, Grid& G) {
  if (!d || nranks < 1 || d->p < 1 || d->p > 8) return false;
  G.p = d->p;
  for (int a = 0; a < 3; ++a) {
    G.n[a] = d->ncell[a];
    G.per[a] = d->periodic[a] != 0;
    if (G.n[a] < 1 || (G.per[a] && G.n[a] < 2) || (!G.per[a] && G.n[a] * d->p < 2)) return false;
    G.nd[a] = G.per[a] ? (int64_t)G.n[a] * G.p : (int64_t)G.n[a] * G.p - 1;
  }
  // factorisation px py pz = nranks with the smallest interface area
  double best = 1e300;
  bool found = false;
  for (int px = 1; px <= nranks; ++px) {
    if (nranks % px || px > G.n[0]) continue;
    for (int py = 1; py <= nranks / px; ++py) {
      if ((nranks / px) % py || py > G.n[1]) continue;
      const int pz = nranks / px / py;
      if (pz > G.n[2]) continue;
      const double area = (double)(px - 1) * G.n[1] * G.n[2] + (double)(py - 1) * G.n[0] * G.n[2] +
                          (double)(pz - 1) * G.n[0] * G.n[1];
      if (area < best) {
        best = area;
        G.P[0] = px;
        G.P[1] = py;
        G.P[2] = pz;
        found = true;
      }
    }
  }
  return found;
}

struct Part {
  std::vector<int32_t> cells, l2g, owner, neighbors;
  std::vector<int64_t> halo_ptr;
  std::vector<int32_t> halo;
};

void build_part(const Grid& G, int rank, Part& out) {
  const int ix = rank % G.P[0], iy = (rank / G.P[0]) % G.P[1], iz = rank / (G.P[0] * G.P[1]);
  const int me[3] = {ix, iy, iz};
  int c0[3], c1[3];
  for (int a = 0; a < 3; ++a) {
    c0[a] = (int)((int64_t)me[a] * G.n[a] / G.P[a]);
    c1[a] = (int)((int64_t)(me[a] + 1) * G.n[a] / G.P[a]);
  }
  out.cells.clear();
  for (int z = c0[2]; z < c1[2]; ++z)
    for (int y = c0[1]; y < c1[1]; ++y)
      for (int x = c0[0]; x < c1[0]; ++x)
        out.cells.push_back((int32_t)(x + G.n[0] * ((int64_t)y + (int64_t)G.n[1] * z)));
  // unknowns touched along each axis: nodes c0 p .. c1 p, wrapped / Dirichlet-dropped
  std::array<std::vector<int64_t>, 3> u1;
  for (int a = 0; a < 3; ++a) {
    for (int64_t g = (int64_t)c0[a] * G.p; g <= (int64_t)c1[a] * G.p; ++g) {
      int64_t u;
      if (G.per[a]) {
        u = g % ((int64_t)G.n[a] * G.p);
      } else {
        if (g == 0 || g == (int64_t)G.n[a] * G.p) continue;
        u = g - 1;
      }
      u1[a].push_back(u);
    }
    std::sort(u1[a].begin(), u1[a].end());
    u1[a].erase(std::unique(u1[a].begin(), u1[a].end()), u1[a].end());
  }
  out.l2g.clear();
  for (int64_t z : u1[2])
    for (int64_t y : u1[1])
      for (int64_t x : u1[0]) out.l2g.push_back((int32_t)(x + G.nd[0] * (y + G.nd[1] * z)));
  std::sort(out.l2g.begin(), out.l2g.end());
  // sharing ranks of every local unknown
  const size_t nl = out.l2g.size();
  out.owner.assign(nl, rank);
  std::vector<std::vector<int32_t>> share(nl);
  std::vector<int32_t> nbr;
  for (size_t i = 0; i < nl; ++i) {
    const int64_t gi = out.l2g[i];
    const int64_t u[3] = {gi % G.nd[0], (gi / G.nd[0]) % G.nd[1], gi / (G.nd[0] * G.nd[1])};
    int parts[3][2], np[3];
    for (int a = 0; a < 3; ++a) {
      int cs[2];
      const int k = cells_of_node(G, a, node_of_unknown(G, a, u[a]), cs);
      np[a] = 0;
      for (int t = 0; t < k; ++t) {
        const int pa = part_of_cell(G, a, cs[t]);
        if (np[a] == 0 || parts[a][0] != pa) parts[a][np[a]++] = pa;
      }
    }
    std::vector<int32_t>& s = share[i];
    for (int z = 0; z < np[2]; ++z)
      for (int y = 0; y < np[1]; ++y)
        for (int x = 0; x < np[0]; ++x)
          s.push_back(parts[0][x] + G.P[0] * (parts[1][y] + G.P[1] * parts[2][z]));
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    out.owner[i] = s.front();
    for (int32_t q : s)
      if (q != rank) nbr.push_back(q);
  }
  std::sort(nbr.begin(), nbr.end());
  nbr.erase(std::unique(nbr.begin(), nbr.end()), nbr.end());
  out.neighbors = nbr;
  out.halo_ptr.assign(1, 0);
  out.halo.clear();
  for (int32_t q : nbr) {
    for (size_t i = 0; i < nl; ++i)
      if (std::binary_search(share[i].begin(), share[i].end(), q)) out.halo.push_back((int32_t)i);
    out.halo_ptr.push_back((int64_t)out.halo.size());
  }
}

}  // namespace

extern "C" {

chfsi_status chfsi_partition_sizes(const chfsi_mesh_desc* desc, int nranks, int rank,
                                   chfsi_partition_info* out) {
  Grid G;
  if (!out || rank < 0 || rank >= nranks || !make_grid(desc, nranks, G)) return CHFSI_ERR_ARG;
  int64_t nd = G.nd[0] * G.nd[1] * G.nd[2];
  if (nd >= ((int64_t)1 << 31)) return CHFSI_ERR_ARG;
  Part P;
  build_part(G, rank, P);
  out->ncells = (int64_t)P.cells.size();
  out->nlocal = (int64_t)P.l2g.size();
  out->nneighbors = (int)P.neighbors.size();
  out->nhalo = (int64_t)P.halo.size();
  for (int a = 0; a < 3; ++a) out->grid[a] = G.P[a];
  return CHFSI_OK;
}

chfsi_status chfsi_partition_fill(const chfsi_mesh_desc* desc, int nranks, int rank, int32_t* cells,
                                  int32_t* l2g, int32_t* owner, int32_t* neighbors,
                                  int64_t* halo_ptr, int32_t* halo) {
  Grid G;
  if (rank < 0 || rank >= nranks || !make_grid(desc, nranks, G)) return CHFSI_ERR_ARG;
  if (!cells || !l2g || !owner || !halo_ptr) return CHFSI_ERR_ARG;
  if (G.nd[0] * G.nd[1] * G.nd[2] >= ((int64_t)1 << 31)) return CHFSI_ERR_ARG;
  Part P;
  build_part(G, rank, P);
  if ((!P.neighbors.empty() && !neighbors) || (!P.halo.empty() && !halo)) return CHFSI_ERR_ARG;
  std::copy(P.cells.begin(), P.cells.end(), cells);
  std::copy(P.l2g.begin(), P.l2g.end(), l2g);
  std::copy(P.owner.begin(), P.owner.end(), owner);
  std::copy(P.neighbors.begin(), P.neighbors.end(), neighbors);
  std::copy(P.halo_ptr.begin(), P.halo_ptr.end(), halo_ptr);
  std::copy(P.halo.begin(), P.halo.end(), halo);
  return CHFSI_OK;
}

}  // extern "C"
