// patches.h -- Morton patches of elements for the shared-memory element kernels.
#pragma once

#include "pnp_internal.h"

struct PatchData {
  int64_t n_patches = 0;
  int max_nodes = 0, max_colors = 0;
  std::vector<int32_t> patch_e0;   // [P+1] element ranges
  std::vector<int32_t> patch_n0;   // [P+1] ranges into pnode
  std::vector<int32_t> patch_h0;   // [P+1] ranges into the hanging-corner table
  std::vector<uint8_t> patch_ncol; // [P] colours used by the patch
  std::vector<int32_t> pnode;      // global node id of every patch slot (sorted per patch)
  std::vector<int32_t> pbslot;     // partial-buffer index of a shared slot, or -1 (owned)
  std::vector<uint16_t> el_slot;   // [E][2^dim] local slot, or 0x8000|hanging entry
  std::vector<uint8_t> el_color;   // [E]
  std::vector<uint8_t> hc_np;      // [Hc] parent count of a hanging corner entry
  std::vector<uint16_t> hc_par;    // [Hc][4] local slots of its parents
  std::vector<int32_t> bnode;      // shared nodes
  std::vector<int32_t> bptr;       // [B+1] their partials are [bptr[b], bptr[b+1])
  std::vector<int32_t> blist;
  int64_t n_partials = 0;
};

int pnp_build_patches(const pnp_mesh& m, int max_elems, int max_nodes, PatchData& P);
int64_t pnp_check_patches(const pnp_mesh& m, const PatchData& P);

// Device view of the patch data.
struct DevPatches {
  int64_t n_patches = 0, n_bnodes = 0, n_partials = 0;
  int max_nodes = 0;
  const int32_t* patch_e0 = nullptr;
  const int32_t* patch_n0 = nullptr;
  const int32_t* patch_h0 = nullptr;
  const uint8_t* patch_ncol = nullptr;
  const int32_t* pnode = nullptr;
  const int32_t* pbslot = nullptr;
  const uint16_t* el_slot = nullptr;
  const uint8_t* el_color = nullptr;
  const uint8_t* hc_np = nullptr;
  const uint16_t* hc_par = nullptr;
  const int32_t* bnode = nullptr;
  const int32_t* bptr = nullptr;
};
