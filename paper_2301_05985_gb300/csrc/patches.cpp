// patches.cpp -- Morton patches for the shared-memory element kernels (host side).
//
// A patch is a run of consecutive (Morton-ordered) elements whose target nodes -- the
// non-hanging corners and the parents of hanging corners -- fit in shared memory.  For
// each patch we record its sorted node list, each element's local corner slots, a
// greedy colouring of its elements (two elements of one colour never share a target
// node, so colour-by-colour accumulation into shared memory needs no atomics and has a
// fixed order), and which nodes are shared with other patches.  Shared nodes receive
// one partial per patch in a global buffer that a finalize pass sums in patch order.
#include <algorithm>
#include <cstring>
#include <unordered_map>

#include "patches.h"

int pnp_build_patches(const pnp_mesh& m, int max_elems, int max_nodes, PatchData& P) {
  P = PatchData();
  const int nc = 1 << m.dim;
  const int64_t E = m.n_elem, N = m.n_nodes;
  if (max_elems > 1024 || max_nodes > 0x7FFF) PNP_FAIL(PNP_ERR_ARG, "patch limits too large");
  // target list of one element corner
  auto targets = [&](int64_t e, int c, int32_t* t) -> int {
    const int32_t id = m.el_conn[e * nc + c];
    if (id >= 0) {
      t[0] = id;
      return 1;
    }
    const int32_t h = -id - 1;
    const int np = m.hang_np[h];
    for (int p = 0; p < np; ++p) t[p] = m.hang_par[4 * h + p];
    return np;
  };
  // 1. greedy partition into patches
  std::vector<int64_t> starts;
  {
    std::unordered_map<int32_t, int> seen;
    seen.reserve(2 * (size_t)max_nodes);
    int64_t e0 = 0;
    starts.push_back(0);
    int cnt = 0;
    for (int64_t e = 0; e < E; ++e) {
      int add = 0;
      int32_t t[4];
      std::vector<int32_t> fresh;
      for (int c = 0; c < nc; ++c) {
        const int k = targets(e, c, t);
        for (int q = 0; q < k; ++q)
          if (!seen.count(t[q]) && std::find(fresh.begin(), fresh.end(), t[q]) == fresh.end()) fresh.push_back(t[q]);
      }
      add = (int)fresh.size();
      if (cnt > 0 && (e - e0 >= max_elems || (int)seen.size() + add > max_nodes)) {
        starts.push_back(e);
        e0 = e;
        seen.clear();
        cnt = 0;
        fresh.clear();
        for (int c = 0; c < nc; ++c) {
          const int k = targets(e, c, t);
          for (int q = 0; q < k; ++q)
            if (std::find(fresh.begin(), fresh.end(), t[q]) == fresh.end()) fresh.push_back(t[q]);
        }
      }
      for (int32_t v : fresh) seen[v] = 1;
      ++cnt;
    }
    starts.push_back(E);
  }
  const int64_t NP = (int64_t)starts.size() - 1;
  P.n_patches = NP;
  P.patch_e0.resize(NP + 1);
  P.patch_n0.resize(NP + 1);
  P.patch_h0.resize(NP + 1);
  P.patch_ncol.resize(NP);
  P.el_slot.assign(E * nc, 0);
  P.el_color.assign(E, 0);
  std::vector<int32_t> owner_count(N, 0);
  // 2. per patch: sorted node list, slots, hanging entries, colouring
  for (int64_t p = 0; p < NP; ++p) {
    const int64_t e0 = starts[p], e1 = starts[p + 1];
    P.patch_e0[p] = (int32_t)e0;
    std::vector<int32_t> nodes;
    int32_t t[4];
    for (int64_t e = e0; e < e1; ++e)
      for (int c = 0; c < nc; ++c) {
        const int k = targets(e, c, t);
        for (int q = 0; q < k; ++q) nodes.push_back(t[q]);
      }
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    if ((int)nodes.size() > max_nodes) PNP_FAIL(PNP_ERR_STATE, "patch node list overflow");
    P.patch_n0[p] = (int32_t)P.pnode.size();
    P.patch_h0[p] = (int32_t)P.hc_np.size();
    for (int32_t v : nodes) {
      P.pnode.push_back(v);
      owner_count[v] += 1;
    }
    auto slot_of = [&](int32_t v) {
      return (uint16_t)(std::lower_bound(nodes.begin(), nodes.end(), v) - nodes.begin());
    };
    std::vector<uint64_t> used(nodes.size(), 0);
    int ncol = 0;
    for (int64_t e = e0; e < e1; ++e) {
      uint64_t forbid = 0;
      std::vector<uint16_t> my;
      for (int c = 0; c < nc; ++c) {
        const int32_t id = m.el_conn[e * nc + c];
        if (id >= 0) {
          const uint16_t s = slot_of(id);
          P.el_slot[e * nc + c] = s;
          my.push_back(s);
        } else {
          const int k = targets(e, c, t);
          const int32_t hl = (int32_t)P.hc_np.size() - P.patch_h0[p];
          if (hl >= 0x8000) PNP_FAIL(PNP_ERR_STATE, "too many hanging corners in a patch");
          P.el_slot[e * nc + c] = (uint16_t)(0x8000 | hl);
          P.hc_np.push_back((uint8_t)k);
          for (int q = 0; q < 4; ++q) {
            const uint16_t s = q < k ? slot_of(t[q]) : 0;
            P.hc_par.push_back(s);
            if (q < k) my.push_back(s);
          }
        }
      }
      for (uint16_t s : my) forbid |= used[s];
      int col = 0;
      while (col < 64 && ((forbid >> col) & 1)) ++col;
      if (col >= 64) PNP_FAIL(PNP_ERR_STATE, "patch colouring needs more than 64 colours");
      P.el_color[e] = (uint8_t)col;
      for (uint16_t s : my) used[s] |= (uint64_t(1) << col);
      ncol = std::max(ncol, col + 1);
    }
    P.patch_ncol[p] = (uint8_t)ncol;
    P.max_colors = std::max(P.max_colors, ncol);
  }
  P.patch_e0[NP] = (int32_t)E;
  P.patch_n0[NP] = (int32_t)P.pnode.size();
  P.patch_h0[NP] = (int32_t)P.hc_np.size();
  // 3. shared nodes: one partial per (patch, node); finalize lists in patch order
  P.pbslot.assign(P.pnode.size(), -1);
  std::vector<int32_t> bindex(N, -1);
  std::vector<int32_t> bcount;
  for (int64_t v = 0; v < N; ++v)
    if (owner_count[v] > 1) {
      bindex[v] = (int32_t)P.bnode.size();
      P.bnode.push_back((int32_t)v);
      bcount.push_back(0);
    }
  P.bptr.assign(P.bnode.size() + 1, 0);
  for (size_t s = 0; s < P.pnode.size(); ++s) {
    const int32_t b = bindex[P.pnode[s]];
    if (b >= 0) P.bptr[b + 1]++;
  }
  for (size_t b = 0; b < P.bnode.size(); ++b) P.bptr[b + 1] += P.bptr[b];
  P.n_partials = P.bptr.back();
  std::vector<int32_t> fill(P.bnode.size(), 0);
  P.blist.assign(P.n_partials, 0);
  for (size_t s = 0; s < P.pnode.size(); ++s) {  // slots are in patch order
    const int32_t b = bindex[P.pnode[s]];
    if (b < 0) continue;
    const int32_t q = P.bptr[b] + fill[b]++;
    P.pbslot[s] = q;
    P.blist[q] = q;  // partial q belongs to node b; kept for clarity of the layout
  }
  P.max_nodes = 0;
  for (int64_t p = 0; p < NP; ++p) P.max_nodes = std::max(P.max_nodes, P.patch_n0[p + 1] - P.patch_n0[p]);
  return PNP_OK;
}

// Verify the invariants the patch kernels rely on; returns the number of violations.
int64_t pnp_check_patches(const pnp_mesh& m, const PatchData& P) {
  const int nc = 1 << m.dim;
  int64_t bad = 0;
  std::vector<int32_t> covered(m.n_nodes, 0);
  for (int64_t p = 0; p < P.n_patches; ++p) {
    const int32_t n0 = P.patch_n0[p], nn = P.patch_n0[p + 1] - n0, h0 = P.patch_h0[p];
    std::vector<std::vector<int>> by_color(64);
    for (int32_t e = P.patch_e0[p]; e < P.patch_e0[p + 1]; ++e) {
      std::vector<int> sl;
      for (int c = 0; c < nc; ++c) {
        const uint16_t s = P.el_slot[(int64_t)e * nc + c];
        const int32_t id = m.el_conn[(int64_t)e * nc + c];
        if (!(s & 0x8000)) {
          if (id < 0 || s >= nn || P.pnode[n0 + s] != id) ++bad;
          sl.push_back(s);
        } else {
          const int hc = h0 + (s & 0x7FFF);
          if (id >= 0 || hc >= P.patch_h0[p + 1]) { ++bad; continue; }
          const int32_t h = -id - 1;
          if (P.hc_np[hc] != m.hang_np[h]) ++bad;
          for (int q = 0; q < P.hc_np[hc]; ++q) {
            const uint16_t ps = P.hc_par[4 * hc + q];
            if (ps >= nn || P.pnode[n0 + ps] != m.hang_par[4 * h + q]) ++bad;
            sl.push_back(ps);
          }
        }
      }
      const int col = P.el_color[e];
      if (col >= P.patch_ncol[p]) ++bad;
      for (int other : by_color[col])
        for (int s : sl)
          for (int c2 = 0; c2 < nc; ++c2) {
            const uint16_t s2 = P.el_slot[(int64_t)other * nc + c2];
            if (!(s2 & 0x8000)) {
              if (s2 == s) ++bad;
            } else {
              const int hc = h0 + (s2 & 0x7FFF);
              for (int q = 0; q < P.hc_np[hc]; ++q)
                if (P.hc_par[4 * hc + q] == s) ++bad;
            }
          }
      by_color[col].push_back(e);
    }
    for (int32_t s = 0; s < nn; ++s) covered[P.pnode[n0 + s]]++;
  }
  int64_t partials = 0;
  for (int64_t v = 0; v < m.n_nodes; ++v) {
    const bool hanging = m.node_hang[v] >= 0;
    if (hanging != (covered[v] == 0)) ++bad;
    if (covered[v] > 1) partials += covered[v];
  }
  if (partials != P.n_partials) ++bad;
  return bad;
}
