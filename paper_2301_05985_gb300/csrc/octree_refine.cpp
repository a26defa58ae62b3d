// octree_refine.cpp -- refinement of a complete linear octree to per-leaf target levels,
// followed by 2:1 balancing (host side).
//
// The paper builds its meshes top-down with a refinement predicate evaluated on the
// octants' coordinates and on field values (Sec. 4.2), and refines near the membrane and
// where the solution varies fastest (Sec. 5.2).  This file provides the octree operation
// behind that: every leaf is split until it reaches its target level, then leaves are
// split until the octree is 2:1 balanced across faces, edges and corners (the condition
// pnp_mesh_create checks).  The result is the coarsest balanced octree that refines every
// input leaf to at least its target: a leaf is only ever split because a target or a
// neighbour two levels finer requires it.
//
// Data structure: one open-addressing hash table holding every octant of the tree,
// leaves and interior octants, keyed by (level, Morton code of the anchor).  Balance is
// done level by level from the finest: for a leaf at level l and each of its 3^d - 1
// same-size neighbour positions b, the octree is balanced there iff the level-(l-1)
// octant containing b belongs to the tree (as a leaf or as an interior octant); otherwise
// a leaf coarser than l-1 contains b, and it is split along the path to b down to level
// l-1.  Leaves created by a split are coarser than l, so they are checked when their own
// level is processed.
#include <algorithm>
#include <cstring>
#include <new>

#include "pnp_internal.h"

namespace {

constexpr uint8_t kEmpty = 0, kLeaf = 1, kInterior = 2;

struct OctTable {
  std::vector<uint64_t> key;
  std::vector<uint8_t> state;
  size_t mask = 0, used = 0;

  explicit OctTable(size_t expect) {
    size_t cap = 1024;
    while (cap < 2 * expect + 16) cap <<= 1;
    key.assign(cap, 0);
    state.assign(cap, kEmpty);
    mask = cap - 1;
  }
  static uint64_t hash(uint64_t k) {  // SplitMix64 finaliser as a mixing function
    k += 0x9E3779B97F4A7C15ull;
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    return k ^ (k >> 31);
  }
  size_t slot(uint64_t k) const {
    size_t i = hash(k) & mask;
    while (state[i] != kEmpty && key[i] != k) i = (i + 1) & mask;
    return i;
  }
  uint8_t get(uint64_t k) const { return state[slot(k)]; }
  void grow() {
    std::vector<uint64_t> ok;
    std::vector<uint8_t> os;
    ok.swap(key);
    os.swap(state);
    key.assign(ok.size() * 2, 0);
    state.assign(ok.size() * 2, kEmpty);
    mask = key.size() - 1;
    for (size_t i = 0; i < ok.size(); ++i)
      if (os[i] != kEmpty) {
        const size_t j = slot(ok[i]);
        key[j] = ok[i];
        state[j] = os[i];
      }
  }
  void set(uint64_t k, uint8_t s) {
    if (2 * (used + 1) > key.size()) grow();
    const size_t i = slot(k);
    if (state[i] == kEmpty) {
      ++used;
      key[i] = k;
    }
    state[i] = s;
  }
};

struct Refiner {
  int dim, L, periodic;
  int64_t size;
  OctTable tab;
  std::vector<std::vector<uint64_t>> by_level;  // Morton codes of leaves created per level

  Refiner(int d, int l, int p, size_t expect) : dim(d), L(l), periodic(p), size(int64_t(1) << l), tab(expect) {
    by_level.resize(L + 1);
  }
  uint64_t code(const int64_t* a) const { return pnp_morton(dim, a); }
  static uint64_t key(int l, uint64_t m) { return (uint64_t(l) << 56) | m; }
  void decode(uint64_t m, int64_t* a) const {
    for (int k = 0; k < 3; ++k) a[k] = 0;
    for (int b = 0; b < 21; ++b)
      for (int k = 0; k < dim; ++k) a[k] |= int64_t((m >> (dim * b + k)) & 1) << b;
  }
  // mark the ancestors of a leaf (level l, anchor a) as interior octants; false when one of
  // them is a leaf (overlapping input)
  bool add_ancestors(int l, const int64_t* a) {
    for (int la = l - 1; la >= 0; --la) {
      const int64_t s = int64_t(1) << (L - la);
      int64_t p[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) p[k] = a[k] / s * s;
      const uint64_t kk = key(la, code(p));
      const uint8_t st = tab.get(kk);
      if (st == kLeaf) return false;
      if (st == kInterior) break;  // the rest of the chain is already present
      tab.set(kk, kInterior);
    }
    return true;
  }
  // split leaf (l, a) into its 2^d children (leaves at l + 1)
  void split(int l, const int64_t* a) {
    int64_t p[3] = {a[0], a[1], a[2]};
    tab.set(key(l, code(p)), kInterior);
    const int64_t h = int64_t(1) << (L - l - 1);
    for (int c = 0; c < (1 << dim); ++c) {
      int64_t q[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) q[k] = a[k] + (((c >> k) & 1) ? h : 0);
      const uint64_t m = code(q);
      tab.set(key(l + 1, m), kLeaf);
      by_level[l + 1].push_back(m);
    }
  }
  // split leaf (l, a) down to level t along every branch
  void refine_to(int l, const int64_t* a, int t) {
    if (l >= t) return;
    split(l, a);
    const int64_t h = int64_t(1) << (L - l - 1);
    for (int c = 0; c < (1 << dim); ++c) {
      int64_t q[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) q[k] = a[k] + (((c >> k) & 1) ? h : 0);
      refine_to(l + 1, q, t);
    }
  }
  // make the level-(l-1) octant containing point b part of the tree, splitting the
  // coarser leaf that contains b along the path to it
  void ensure(int l, const int64_t* b) {
    const int target = l - 1;
    int64_t p[3] = {0, 0, 0};
    const int64_t st = int64_t(1) << (L - target);
    for (int k = 0; k < dim; ++k) p[k] = b[k] / st * st;
    if (tab.get(key(target, code(p))) != kEmpty) return;
    // the leaf containing b: the coarsest level whose octant holding b is a leaf
    int lc = target - 1;
    int64_t a[3] = {0, 0, 0};
    for (; lc >= 0; --lc) {
      const int64_t s = int64_t(1) << (L - lc);
      for (int k = 0; k < dim; ++k) a[k] = b[k] / s * s;
      if (tab.get(key(lc, code(a))) == kLeaf) break;
    }
    if (lc < 0) return;  // cannot happen for a complete cover
    for (int lv = lc; lv < target; ++lv) {
      split(lv, a);
      const int64_t h = int64_t(1) << (L - lv - 1);
      for (int k = 0; k < dim; ++k) a[k] = b[k] / h * h;  // the child holding b
    }
  }
  void balance() {
    int dir[27][3];
    int nd = 0;
    for (int i = 0; i < (dim == 3 ? 27 : 9); ++i) {
      const int d0 = i % 3 - 1, d1 = (i / 3) % 3 - 1, d2 = dim == 3 ? i / 9 - 1 : 0;
      if (!d0 && !d1 && !d2) continue;
      dir[nd][0] = d0;
      dir[nd][1] = d1;
      dir[nd][2] = d2;
      ++nd;
    }
    for (int l = L; l >= 2; --l) {
      const int64_t s = int64_t(1) << (L - l);
      // leaves of this level: those created here plus those of the input (already listed)
      auto& lst = by_level[l];
      for (size_t i = 0; i < lst.size(); ++i) {
        const uint64_t m = lst[i];
        if (tab.get(key(l, m)) != kLeaf) continue;
        int64_t a[3];
        decode(m, a);
        for (int d = 0; d < nd; ++d) {
          int64_t b[3] = {0, 0, 0};
          bool inside = true;
          for (int k = 0; k < dim; ++k) {
            b[k] = a[k] + dir[d][k] * s;
            if (b[k] < 0 || b[k] >= size) {
              if ((periodic >> k) & 1) b[k] = (b[k] + size) % size;
              else inside = false;
            }
          }
          if (inside) ensure(l, b);
        }
      }
    }
  }
};

}  // namespace

int pnp_refine_balance(int dim, int L, int periodic, int64_t n, const int32_t* anchors, const uint8_t* levels,
                       const uint8_t* target, std::vector<int32_t>& out_anchor, std::vector<uint8_t>& out_level) {
  if (dim != 2 && dim != 3) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create_refined: dim must be 2 or 3 (got %d)", dim);
  if (L < 0 || L > 16) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create_refined: max_level must be in 0..16 (got %d)", L);
  if (periodic < 0 || periodic >= (1 << dim)) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create_refined: bad periodic mask");
  if (n <= 0 || !anchors || !levels) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create_refined: empty octant list or null pointer");
  Refiner R(dim, L, periodic, (size_t)n * 2);
  const int64_t size = int64_t(1) << L;
  for (int64_t e = 0; e < n; ++e) {
    const int l = levels[e];
    if (l > L) PNP_FAIL(PNP_ERR_MESH, "octant %lld: level %d > max_level %d", (long long)e, l, L);
    if (target && target[e] > L)
      PNP_FAIL(PNP_ERR_ARG, "octant %lld: target level %d > max_level %d", (long long)e, target[e], L);
    const int64_t s = int64_t(1) << (L - l);
    int64_t a[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      a[k] = anchors[e * dim + k];
      if (a[k] < 0 || a[k] % s || a[k] + s > size)
        PNP_FAIL(PNP_ERR_MESH, "octant %lld: anchor not aligned to its level or outside the domain", (long long)e);
    }
    const uint64_t kk = Refiner::key(l, R.code(a));
    if (R.tab.get(kk) != kEmpty) PNP_FAIL(PNP_ERR_MESH, "octants overlap (octant %lld)", (long long)e);
    R.tab.set(kk, kLeaf);
    if (!R.add_ancestors(l, a)) PNP_FAIL(PNP_ERR_MESH, "octants overlap (octant %lld)", (long long)e);
    R.by_level[l].push_back(R.code(a));
  }
  // a leaf listed as interior by a later octant's ancestors overlaps it
  for (int64_t e = 0; e < n; ++e) {
    int64_t a[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) a[k] = anchors[e * dim + k];
    if (R.tab.get(Refiner::key(levels[e], R.code(a))) != kLeaf)
      PNP_FAIL(PNP_ERR_MESH, "octants overlap (octant %lld)", (long long)e);
  }
  if (target)
    for (int64_t e = 0; e < n; ++e) {
      int64_t a[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) a[k] = anchors[e * dim + k];
      R.refine_to(levels[e], a, target[e]);
    }
  R.balance();
  out_anchor.clear();
  out_level.clear();
  out_anchor.reserve(R.tab.used * dim);
  out_level.reserve(R.tab.used);
  for (size_t i = 0; i < R.tab.key.size(); ++i) {
    if (R.tab.state[i] != kLeaf) continue;
    const uint64_t k = R.tab.key[i];
    int64_t a[3];
    R.decode(k & ((uint64_t(1) << 56) - 1), a);
    for (int d = 0; d < dim; ++d) out_anchor.push_back((int32_t)a[d]);
    out_level.push_back((uint8_t)(k >> 56));
  }
  return PNP_OK;
}
