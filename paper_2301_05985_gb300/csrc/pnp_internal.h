// pnp_internal.h -- internal data structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pnp.h"

// ------------------------------------------------------------------ errors
void pnp_set_error(const char* fmt, ...);
#define PNP_FAIL(code, ...)       \
  do {                            \
    pnp_set_error(__VA_ARGS__);   \
    return (code);                \
  } while (0)

// ------------------------------------------------------------------ host mesh
// Elements are Morton-ordered octree leaves; nodes are their unique corners in Morton
// order of the (integer) coordinates.  Corner c of an element sits at anchor + h * bits(c)
// (bit k of c = +1 along axis k).
struct pnp_mesh {
  int dim = 0;
  int L = 0;
  int periodic = 0;                 // bit k: axis k is periodic (faces 2k, 2k+1 identified)
  int64_t n_elem = 0, n_nodes = 0, n_hanging = 0;
  std::vector<int32_t> el_anchor;   // [E][dim]
  std::vector<uint8_t> el_level;    // [E]
  std::vector<int32_t> el_conn;     // [E][2^dim]: node id, or -(h+1) for hanging node h
  std::vector<int32_t> node_ijk;    // [N][dim]
  std::vector<uint8_t> node_faces;  // [N] bit f set: node lies on boundary face f
  std::vector<int32_t> node_hang;   // [N] hanging index or -1
  std::vector<int32_t> hang_node;   // [H] node id of each hanging node
  std::vector<int32_t> hang_par;    // [H][4] parent node ids (-1 padded)
  std::vector<uint8_t> hang_np;     // [H] number of parents (2 or 4)
};

int pnp_build_mesh(pnp_mesh& m, int dim, int L, int64_t n, const int32_t* anchors, const uint8_t* levels,
                   int periodic);
// Refine each octant to at least target[e] (NULL: no targets), then split leaves until the
// octree is 2:1 balanced across faces, edges and corners (periodic axes wrap); the
// coarsest such octree, as unordered leaves.
int pnp_refine_balance(int dim, int L, int periodic, int64_t n, const int32_t* anchors, const uint8_t* levels,
                       const uint8_t* target, std::vector<int32_t>& out_anchor, std::vector<uint8_t>& out_level);
// Geometric multigrid on the octree hierarchy (mg_build.cpp): the octree with every leaf
// finer than `cap` replaced by its ancestor at `cap`; the transfer operators between a fine
// mesh and its capped coarse mesh.
int pnp_cap_mesh_levels(const pnp_mesh& fine, int cap, pnp_mesh& coarse);
struct MgTransfer {
  std::vector<int64_t> p_ptr;   // [Nf+1] prolongation rows (fine nodes)
  std::vector<int32_t> p_col;   // coarse independent nodes
  std::vector<float> p_w;       // trilinear weights (dyadic)
  std::vector<int64_t> r_ptr;   // [Nc+1] restriction rows = P^T (coarse nodes)
  std::vector<int32_t> r_col;   // fine nodes
  std::vector<float> r_w;
  std::vector<int32_t> inject;  // [Nc] fine node at each coarse node's point
};
int pnp_mg_transfer(const pnp_mesh& fine, const pnp_mesh& coarse, MgTransfer& T);
// Morton (Z-order) key of an integer point (x in bit 0 of each group, then y, then z).
uint64_t pnp_morton(int dim, const int64_t* p);

// ------------------------------------------------------------------ device views
struct DevMesh {
  int dim;
  int64_t n_elem, n_nodes, n_hanging;
  const int32_t* conn;       // [E][2^dim]
  const uint8_t* level;      // [E]
  const uint8_t* node_faces; // [N]
  const int32_t* hang_node;  // [H]
  const int32_t* hang_par;   // [H][4]
  const uint8_t* hang_np;    // [H]
};

// Physics constants of one residual / Jv evaluation (passed by value to kernels).
struct PhysParams {
  double eps2x2;   // 2 Lambda^2
  double kappa;    // beta0 / dt (0 when steady)
  double tau_t;    // 4 / dt^2 (0 when steady)
  double C_I;
  int steady;
};

// Boundary-condition description for the row fix-up kernels.
struct BcTable {
  uint8_t dir_faces[3];  // per field: bit f set = Dirichlet on face f
  double val[6][3];      // Dirichlet values
};
