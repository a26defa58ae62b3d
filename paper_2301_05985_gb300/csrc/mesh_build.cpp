// mesh_build.cpp -- octants -> Q1 mesh with hanging-node constraints (host side).
//
// Input: the leaves of a complete linear octree (Sec. 4.2 of arXiv 2301.05985 builds
// the mesh from octree leaves with a space-filling-curve order).  Output: Morton-ordered
// elements, their unique corner nodes in Morton order of the coordinates, and the
// conforming Q1 constraints of hanging nodes (face centre = mean of 4 face corners,
// edge midpoint = mean of 2 edge ends; the paper does not describe them).
//
// Periodic axes (bit k of `periodic`): the faces x_k = 0 and x_k = 1 are identified, so
// a corner at x_k = 1 is the node at x_k = 0.  Corners, midpoints and parents are keyed
// by wrapped coordinates; the neighbourhood count below then covers the wrap too, which
// makes the conformity and 2:1 checks hold across the identified faces.
//
// Validation is done on the node structure: with every octant aligned and the cover
// complete and non-overlapping (checked on Morton intervals), a mesh is conforming and
// 2:1 balanced iff at every node the elements touching it fill the node's neighbourhood
// (each as a corner owner, or -- for a hanging node -- with the node at the midpoint of
// one of its edges/faces) and their levels differ by at most one.

#include <algorithm>
#include <cstring>
#include <numeric>

#include "pnp_internal.h"

namespace {

inline uint64_t spread2(uint64_t x) {  // 32-bit -> even bits
  x &= 0xFFFFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
inline uint64_t spread3(uint64_t x) {  // 21-bit -> every third bit
  x &= 0x1FFFFFull;
  x = (x | (x << 32)) & 0x1F00000000FFFFull;
  x = (x | (x << 16)) & 0x1F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
inline uint64_t morton(int dim, const int64_t* p) {
  if (dim == 2) return spread2((uint64_t)p[0]) | (spread2((uint64_t)p[1]) << 1);
  return spread3((uint64_t)p[0]) | (spread3((uint64_t)p[1]) << 1) | (spread3((uint64_t)p[2]) << 2);
}

// LSD radix sort of (key, payload) pairs by key, 11-bit digits.
void radix_sort_pairs(std::vector<uint64_t>& key, std::vector<uint32_t>& val) {
  const size_t n = key.size();
  if (n < 2) return;
  uint64_t kmax = 0;
  for (uint64_t k : key) kmax |= k;
  int bits = 0;
  while (bits < 64 && (kmax >> bits)) ++bits;
  std::vector<uint64_t> k2(n);
  std::vector<uint32_t> v2(n);
  const int D = 11;
  const size_t R = size_t(1) << D;
  std::vector<size_t> cnt(R);
  for (int shift = 0; shift < bits; shift += D) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (size_t i = 0; i < n; ++i) ++cnt[(key[i] >> shift) & (R - 1)];
    size_t s = 0;
    for (size_t r = 0; r < R; ++r) {
      const size_t c = cnt[r];
      cnt[r] = s;
      s += c;
    }
    for (size_t i = 0; i < n; ++i) {
      const size_t d = (key[i] >> shift) & (R - 1);
      const size_t o = cnt[d]++;
      k2[o] = key[i];
      v2[o] = val[i];
    }
    key.swap(k2);
    val.swap(v2);
  }
}

}  // namespace

uint64_t pnp_morton(int dim, const int64_t* p) { return morton(dim, p); }

int pnp_build_mesh(pnp_mesh& m, int dim, int L, int64_t n, const int32_t* anchors, const uint8_t* levels,
                   int periodic) {
  if (dim != 2 && dim != 3) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: dim must be 2 or 3 (got %d)", dim);
  if (periodic < 0 || periodic >= (1 << dim))
    PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: periodic mask %d has bits beyond dim %d", periodic, dim);
  if (L < 0 || L > 16) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: max_level must be in 0..16 (got %d)", L);
  if (n <= 0 || !anchors || !levels) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: empty octant list or null pointer");
  const int nc = 1 << dim;
  const int64_t size = int64_t(1) << L;
  if (n > (int64_t(1) << 31) / nc) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: too many octants (%lld)", (long long)n);
  m = pnp_mesh();
  m.dim = dim;
  m.L = L;
  m.periodic = periodic;
  m.n_elem = n;
  // a coordinate on an identified face maps to 0
  auto wrap = [&](int64_t* p) {
    for (int k = 0; k < dim; ++k)
      if (((periodic >> k) & 1) && p[k] == size) p[k] = 0;
  };

  // ---- validate alignment, Morton-sort the octants, check the cover on Morton intervals
  std::vector<uint64_t> ekey(n);
  std::vector<uint32_t> eidx(n);
  for (int64_t e = 0; e < n; ++e) {
    const int l = levels[e];
    if (l > L) PNP_FAIL(PNP_ERR_MESH, "octant %lld: level %d > max_level %d", (long long)e, l, L);
    if (periodic && l == 0)
      PNP_FAIL(PNP_ERR_MESH, "octant %lld: a periodic axis needs at least two elements across", (long long)e);
    const int64_t s = int64_t(1) << (L - l);
    int64_t a[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      a[k] = anchors[e * dim + k];
      if (a[k] < 0 || a[k] % s || a[k] + s > size)
        PNP_FAIL(PNP_ERR_MESH, "octant %lld: anchor not aligned to its level or outside the domain", (long long)e);
    }
    ekey[e] = morton(dim, a);
    eidx[e] = (uint32_t)e;
  }
  radix_sort_pairs(ekey, eidx);
  {
    uint64_t end = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int l = levels[eidx[i]];
      const uint64_t len = uint64_t(1) << (dim * (L - l));
      if (ekey[i] < end) PNP_FAIL(PNP_ERR_MESH, "octants overlap (Morton interval %llu)", (unsigned long long)ekey[i]);
      if (ekey[i] != end) PNP_FAIL(PNP_ERR_MESH, "octants leave a gap before Morton index %llu", (unsigned long long)ekey[i]);
      end = ekey[i] + len;
    }
    if (end != (uint64_t(1) << (dim * L))) PNP_FAIL(PNP_ERR_MESH, "octants do not cover the domain");
  }
  m.el_anchor.resize(n * dim);
  m.el_level.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t e = eidx[i];
    for (int k = 0; k < dim; ++k) m.el_anchor[i * dim + k] = anchors[e * dim + k];
    m.el_level[i] = levels[e];
  }

  // ---- unique corners
  const int64_t ncor = n * nc;
  std::vector<uint64_t> ckey(ncor);
  std::vector<uint32_t> cslot(ncor);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t s = int64_t(1) << (L - m.el_level[i]);
    for (int c = 0; c < nc; ++c) {
      int64_t p[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) p[k] = m.el_anchor[i * dim + k] + (((c >> k) & 1) ? s : 0);
      wrap(p);
      ckey[i * nc + c] = morton(dim, p);
      cslot[i * nc + c] = (uint32_t)(i * nc + c);
    }
  }
  radix_sort_pairs(ckey, cslot);
  m.el_conn.assign(ncor, -1);
  std::vector<uint64_t> nkey;
  nkey.reserve(ncor / (nc > 4 ? 6 : 3) + 16);
  for (int64_t j = 0; j < ncor; ++j) {
    if (j == 0 || ckey[j] != ckey[j - 1]) nkey.push_back(ckey[j]);
    m.el_conn[cslot[j]] = (int32_t)(nkey.size() - 1);
  }
  const int64_t N = (int64_t)nkey.size();
  m.n_nodes = N;
  m.node_ijk.assign(N * dim, 0);
  m.node_faces.assign(N, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t s = int64_t(1) << (L - m.el_level[i]);
    for (int c = 0; c < nc; ++c) {
      const int32_t id = m.el_conn[i * nc + c];
      int64_t p[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) p[k] = m.el_anchor[i * dim + k] + (((c >> k) & 1) ? s : 0);
      wrap(p);
      for (int k = 0; k < dim; ++k) m.node_ijk[(int64_t)id * dim + k] = (int32_t)p[k];
    }
  }
  for (int64_t v = 0; v < N; ++v) {
    uint8_t f = 0;
    for (int k = 0; k < dim; ++k) {
      if ((periodic >> k) & 1) continue;  // identified faces are not boundary
      const int32_t x = m.node_ijk[v * dim + k];
      if (x == 0) f |= (uint8_t)(1u << (2 * k));
      if (x == size) f |= (uint8_t)(1u << (2 * k + 1));
    }
    m.node_faces[v] = f;
  }
  auto find_node = [&](const int64_t* p0) -> int64_t {
    int64_t p[3] = {p0[0], p0[1], p0[2]};
    wrap(p);
    const uint64_t k = morton(dim, p);
    auto it = std::lower_bound(nkey.begin(), nkey.end(), k);
    if (it == nkey.end() || *it != k) return -1;
    return (int64_t)(it - nkey.begin());
  };

  // ---- node neighbourhood accounting + hanging detection
  // units: each element contributes 2^(#mid coordinates) units of 2^-dim solid angle
  std::vector<int32_t> units(N, 0);
  std::vector<uint8_t> lmin(N, 255), lmax(N, 0);
  for (int64_t i = 0; i < n; ++i) {
    const uint8_t l = m.el_level[i];
    for (int c = 0; c < nc; ++c) {
      const int32_t id = m.el_conn[i * nc + c];
      units[id] += 1;
      lmin[id] = std::min(lmin[id], l);
      lmax[id] = std::max(lmax[id], l);
    }
  }
  m.node_hang.assign(N, -1);
  const int np = dim == 3 ? 27 : 9;
  for (int64_t i = 0; i < n; ++i) {
    const uint8_t l = m.el_level[i];
    if (l == L) continue;  // finest elements have no midpoint nodes
    const int64_t s = int64_t(1) << (L - l);
    const int64_t* a0 = nullptr;
    int64_t a[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) a[k] = m.el_anchor[i * dim + k];
    a0 = a;
    for (int q = 0; q < np; ++q) {
      int t3[3] = {q % 3, (q / 3) % 3, (q / 9) % 3};
      if (dim == 2) t3[2] = 0;
      int nmid = 0;
      for (int k = 0; k < dim; ++k) nmid += (t3[k] == 1);
      if (nmid == 0 || nmid == dim) continue;
      int64_t p[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) p[k] = a0[k] + t3[k] * (s / 2);
      const int64_t id = find_node(p);
      if (id < 0) continue;
      // hanging: parents are the corners of this element spanning the mid coordinates
      int32_t par[4] = {-1, -1, -1, -1};
      const int npar = 1 << nmid;
      for (int pc = 0; pc < npar; ++pc) {
        int corner = 0, bit = 0;
        for (int k = 0; k < dim; ++k) {
          int b;
          if (t3[k] == 1) b = (pc >> bit++) & 1;
          else b = t3[k] / 2;
          corner |= b << k;
        }
        par[pc] = m.el_conn[i * nc + corner];
      }
      for (int x = 1; x < npar; ++x)  // insertion sort of at most four parents
        for (int y = x; y > 0 && par[y - 1] > par[y]; --y) std::swap(par[y - 1], par[y]);
      units[id] += npar;
      lmin[id] = std::min(lmin[id], l);
      lmax[id] = std::max(lmax[id], l);
      const int32_t h = m.node_hang[id];
      if (h >= 0) {
        if (m.hang_np[h] != npar || !std::equal(par, par + npar, &m.hang_par[4 * h]))
          PNP_FAIL(PNP_ERR_MESH_UNBALANCED, "node %lld is hanging on two different coarse entities", (long long)id);
        continue;
      }
      m.node_hang[id] = (int32_t)m.hang_node.size();
      m.hang_node.push_back((int32_t)id);
      for (int k = 0; k < 4; ++k) m.hang_par.push_back(par[k]);
      m.hang_np.push_back((uint8_t)npar);
    }
  }
  for (int64_t v = 0; v < N; ++v) {
    int nb = 0;
    for (int f = 0; f < 2 * dim; ++f) nb += (m.node_faces[v] >> f) & 1;
    const int want = 1 << (dim - nb);
    if (units[v] != want)
      PNP_FAIL(PNP_ERR_MESH_UNBALANCED,
               "node %lld is not conforming (neighbourhood %d/%d): a neighbour is two or more levels finer",
               (long long)v, units[v], want);
    if (lmax[v] - lmin[v] > 1)
      PNP_FAIL(PNP_ERR_MESH_UNBALANCED, "node %lld touches elements of levels %d and %d", (long long)v, lmin[v], lmax[v]);
  }
  m.n_hanging = (int64_t)m.hang_node.size();
  for (int64_t h = 0; h < m.n_hanging; ++h)
    for (int k = 0; k < m.hang_np[h]; ++k)
      if (m.node_hang[m.hang_par[4 * h + k]] >= 0)
        PNP_FAIL(PNP_ERR_MESH_UNBALANCED, "hanging node %d has a hanging parent", m.hang_node[h]);
  for (int64_t j = 0; j < ncor; ++j) {
    const int32_t h = m.node_hang[m.el_conn[j]];
    if (h >= 0) m.el_conn[j] = -(h + 1);
  }
  return PNP_OK;
}
