// mg_build.cpp -- the octree hierarchy and the grid-transfer operators of the geometric
// multigrid preconditioner (host side).
//
// Coarse meshes: the octree with every leaf finer than a cap level replaced by its
// ancestor at the cap.  Capping keeps a 2:1-balanced octree balanced (two neighbours
// within one level of each other stay within one level when both are capped), and every
// coarse element is a union of fine elements, so the coarse Q1 space is contained in the
// fine one and every coarse node is a point of the fine mesh.
//
// Prolongation P: the value of a coarse Q1 field at every fine node, i.e. trilinear
// interpolation inside the coarse element holding the node, with coarse hanging corners
// expanded to their parents (so P's columns are independent coarse nodes).  Restriction
// is the transpose.  Both are stored as CSR matrices of scalar weights shared by the
// three fields.  Injection: the fine node at each coarse node's point (used to carry the
// nonlinear state down the hierarchy).
#include <algorithm>
#include <unordered_map>

#include "pnp_internal.h"

int pnp_cap_mesh_levels(const pnp_mesh& fine, int cap, pnp_mesh& coarse) {
  const int dim = fine.dim, L = fine.L;
  const int64_t E = fine.n_elem;
  std::vector<int32_t> a;
  std::vector<uint8_t> l;
  a.reserve(E * dim);
  l.reserve(E);
  std::unordered_map<uint64_t, bool> seen;
  seen.reserve((size_t)E);
  for (int64_t e = 0; e < E; ++e) {
    const int lev = std::min<int>(fine.el_level[e], cap);
    const int64_t s = int64_t(1) << (L - lev);
    int64_t p[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) p[k] = fine.el_anchor[e * dim + k] / s * s;
    const uint64_t key = (uint64_t(lev) << 56) | pnp_morton(dim, p);
    if (!seen.emplace(key, true).second) continue;
    for (int k = 0; k < dim; ++k) a.push_back((int32_t)p[k]);
    l.push_back((uint8_t)lev);
  }
  return pnp_build_mesh(coarse, dim, L, (int64_t)l.size(), a.data(), l.data(), fine.periodic);
}

namespace {
// node index of integer point p (nodes are in Morton order of their coordinates), or -1
struct NodeFinder {
  std::vector<uint64_t> key;
  int dim;
  explicit NodeFinder(const pnp_mesh& m) : dim(m.dim) {
    key.resize(m.n_nodes);
    for (int64_t i = 0; i < m.n_nodes; ++i) {
      int64_t p[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) p[k] = m.node_ijk[i * dim + k];
      key[i] = pnp_morton(dim, p);
    }
  }
  int64_t find(const int64_t* p) const {
    const uint64_t k = pnp_morton(dim, p);
    auto it = std::lower_bound(key.begin(), key.end(), k);
    if (it == key.end() || *it != k) return -1;
    return (int64_t)(it - key.begin());
  }
};
}  // namespace

int pnp_mg_transfer(const pnp_mesh& fine, const pnp_mesh& coarse, MgTransfer& T) {
  const int dim = fine.dim, L = fine.L, nc = 1 << dim;
  if (coarse.dim != dim || coarse.L != L) PNP_FAIL(PNP_ERR_ARG, "multigrid: meshes of different shape");
  if (fine.periodic || coarse.periodic) PNP_FAIL(PNP_ERR_ARG, "multigrid: periodic meshes are not supported");
  const int64_t size = int64_t(1) << L;
  // coarse leaves by (level, anchor)
  std::unordered_map<uint64_t, int64_t> leaf;
  leaf.reserve((size_t)coarse.n_elem * 2);
  int lmin = 64, lmax = 0;
  for (int64_t e = 0; e < coarse.n_elem; ++e) {
    int64_t p[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) p[k] = coarse.el_anchor[e * dim + k];
    const int lev = coarse.el_level[e];
    lmin = std::min(lmin, lev);
    lmax = std::max(lmax, lev);
    leaf[(uint64_t(lev) << 56) | pnp_morton(dim, p)] = e;
  }
  const int64_t Nf = fine.n_nodes, Nc = coarse.n_nodes;
  T.p_ptr.assign(Nf + 1, 0);
  T.p_col.clear();
  T.p_w.clear();
  T.p_col.reserve(Nf * 4);
  T.p_w.reserve(Nf * 4);
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < Nf; ++i) {
    int64_t x[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) x[k] = fine.node_ijk[i * dim + k];
    // the coarse leaf holding x (a point on the upper domain face belongs to the leaf below)
    int64_t e = -1, s = 0;
    int64_t a[3] = {0, 0, 0};
    for (int lev = lmax; lev >= lmin && e < 0; --lev) {
      s = int64_t(1) << (L - lev);
      for (int k = 0; k < dim; ++k) a[k] = std::min(x[k], size - 1) / s * s;
      auto it = leaf.find((uint64_t(lev) << 56) | pnp_morton(dim, a));
      if (it != leaf.end()) e = it->second;
    }
    if (e < 0) PNP_FAIL(PNP_ERR_MESH, "multigrid: fine node %lld lies in no coarse element", (long long)i);
    row.clear();
    for (int c = 0; c < nc; ++c) {
      double w = 1.0;
      for (int k = 0; k < dim; ++k) {
        const double xi = (double)(x[k] - a[k]) / (double)s;
        w *= ((c >> k) & 1) ? xi : 1.0 - xi;
      }
      if (w == 0.0) continue;
      const int32_t id = coarse.el_conn[e * nc + c];
      if (id >= 0) {
        row.push_back({id, w});
      } else {
        const int32_t h = -id - 1;
        const int np = coarse.hang_np[h];
        for (int p = 0; p < np; ++p) row.push_back({coarse.hang_par[4 * h + p], w / np});
      }
    }
    std::sort(row.begin(), row.end());
    for (size_t r = 0; r < row.size(); ++r) {
      if (r > 0 && row[r].first == row[r - 1].first) {
        T.p_w.back() += (float)row[r].second;  // weights are dyadic: exact in float
        continue;
      }
      T.p_col.push_back(row[r].first);
      T.p_w.push_back((float)row[r].second);
    }
    T.p_ptr[i + 1] = (int64_t)T.p_col.size();
  }
  // restriction = transpose (rows: coarse nodes, fixed order of fine rows)
  T.r_ptr.assign(Nc + 1, 0);
  for (int32_t col : T.p_col) T.r_ptr[col + 1]++;
  for (int64_t j = 0; j < Nc; ++j) T.r_ptr[j + 1] += T.r_ptr[j];
  T.r_col.assign(T.p_col.size(), 0);
  T.r_w.assign(T.p_col.size(), 0.f);
  std::vector<int64_t> fill(T.r_ptr.begin(), T.r_ptr.end() - 1);
  for (int64_t i = 0; i < Nf; ++i)
    for (int64_t q = T.p_ptr[i]; q < T.p_ptr[i + 1]; ++q) {
      const int64_t o = fill[T.p_col[q]]++;
      T.r_col[o] = (int32_t)i;
      T.r_w[o] = T.p_w[q];
    }
  // injection: the fine node at every coarse node
  NodeFinder nf(fine);
  T.inject.assign(Nc, -1);
  for (int64_t j = 0; j < Nc; ++j) {
    int64_t p[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) p[k] = coarse.node_ijk[j * dim + k];
    const int64_t f = nf.find(p);
    if (f < 0) PNP_FAIL(PNP_ERR_MESH, "multigrid: coarse node %lld is not a fine node", (long long)j);
    T.inject[j] = (int32_t)f;
  }
  return PNP_OK;
}
