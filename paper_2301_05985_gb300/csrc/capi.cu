// capi.cu -- the extern "C" entry points declared in include/pnp.h: argument checks,
// handle management, uploads and field copies.  Work runs on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>

#include "ctx.h"

static thread_local char g_err[512] = "";

void pnp_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int ctx_check(pnp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PNP_OK;
  if (c && c->latched == cudaSuccess) c->latched = e;
  pnp_set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
  return PNP_ERR_CUDA;
}

#define CTX_GUARD(c)                                                                            \
  do {                                                                                          \
    if (!(c)) PNP_FAIL(PNP_ERR_ARG, "null context");                                            \
    if ((c)->latched != cudaSuccess)                                                            \
      PNP_FAIL(PNP_ERR_CUDA, "context latched after CUDA error %d (%s)", (int)(c)->latched,     \
               cudaGetErrorString((c)->latched));                                               \
  } while (0)

#define CK(call)                                      \
  do {                                                \
    int _rc = ctx_check(c, (call), #call);            \
    if (_rc) return _rc;                              \
  } while (0)

extern "C" {

const char* pnp_last_error(void) { return g_err; }
const char* pnp_version(void) { return "pnp-gb300 0.1 (sm_103a)"; }

void pnp_params_default(pnp_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps = 1e-2;
  p->dt = 1e-3;
  p->C_I = 6.0;
  p->beta0 = 1.0;
  p->beta1 = -1.0;
  p->beta2 = 0.0;
  p->steady = 0;
  p->bdf_order = 2;
  p->newton_rtol = 1e-8;
  p->newton_atol = 0.0;
  p->newton_max_it = 30;
  p->line_search = 1;
  p->gmres_restart = 30;
  p->gmres_max_it = 2000;
  p->gmres_rtol = 1e-8;
  p->precision = PNP_F64;
  p->start_mode = PNP_START_EXTRAPOLATE;
  p->ew_eta_max = 0.9;
  p->ew_eta_min = 1e-4;
  p->monitor = 0;
  p->f64_fallback = 1;
  p->gmres_inner = 0;
  p->newton_ew_f64 = 0;
  p->ns_blocks = 1;
  p->ns_Sc = 1.0;
  p->ns_kappa = 0.5;
  p->ns_rtol = 1e-8;
  p->ns_atol = 1e-10;
  p->ns_inner_rtol = 1e-3;
  p->ns_max_it = 4000;
  p->ns_pin = 1;
  p->ns_mg_levels = 0;
  p->ns_inner_max_it = 200;
  p->ns_fgmres = 30;
  p->pad4_ = 0;
  p->mg_levels = 0;
  p->mg_smooth = 2;
  p->mg_omega = 0.5;
  p->mg_coarse_its = 16;
}

// ------------------------------------------------------------------ mesh
int pnp_mesh_create(int dim, int max_level, int64_t n_oct, const int32_t* anchors, const uint8_t* levels,
                    pnp_mesh** out) {
  return pnp_mesh_create_periodic(dim, max_level, n_oct, anchors, levels, 0, out);
}

int pnp_mesh_create_periodic(int dim, int max_level, int64_t n_oct, const int32_t* anchors, const uint8_t* levels,
                             int periodic, pnp_mesh** out) {
  if (!out) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create: out is null");
  *out = nullptr;
  pnp_mesh* m = new (std::nothrow) pnp_mesh();
  if (!m) PNP_FAIL(PNP_ERR_NOMEM, "pnp_mesh_create: out of host memory");
  int rc;
  try {
    rc = pnp_build_mesh(*m, dim, max_level, n_oct, anchors, levels, periodic);
  } catch (const std::bad_alloc&) {
    pnp_set_error("pnp_mesh_create: out of host memory");
    rc = PNP_ERR_NOMEM;
  }
  if (rc != PNP_OK) {
    delete m;
    return rc;
  }
  *out = m;
  return PNP_OK;
}

int pnp_mesh_create_refined(int dim, int max_level, int64_t n_oct, const int32_t* anchors, const uint8_t* levels,
                            const uint8_t* target_levels, int periodic, pnp_mesh** out) {
  if (!out) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_create_refined: out is null");
  *out = nullptr;
  std::vector<int32_t> a;
  std::vector<uint8_t> l;
  int rc;
  try {
    rc = pnp_refine_balance(dim, max_level, periodic, n_oct, anchors, levels, target_levels, a, l);
  } catch (const std::bad_alloc&) {
    pnp_set_error("pnp_mesh_create_refined: out of host memory");
    rc = PNP_ERR_NOMEM;
  }
  if (rc != PNP_OK) return rc;
  return pnp_mesh_create_periodic(dim, max_level, (int64_t)l.size(), a.data(), l.data(), periodic, out);
}

int pnp_mesh_coarsen(const pnp_mesh* m, int cap_level, pnp_mesh** out) {
  if (!m || !out) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_coarsen: null argument");
  *out = nullptr;
  if (cap_level < 0 || cap_level > m->L) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_coarsen: cap level out of range");
  pnp_mesh* c = new (std::nothrow) pnp_mesh();
  if (!c) PNP_FAIL(PNP_ERR_NOMEM, "pnp_mesh_coarsen: out of host memory");
  int rc;
  try {
    rc = pnp_cap_mesh_levels(*m, cap_level, *c);
  } catch (const std::bad_alloc&) {
    pnp_set_error("pnp_mesh_coarsen: out of host memory");
    rc = PNP_ERR_NOMEM;
  }
  if (rc != PNP_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return PNP_OK;
}

int pnp_mesh_transfer(const pnp_mesh* fine, const pnp_mesh* coarse, int64_t* nnz, int64_t* ptr, int32_t* col,
                      float* w, int32_t* inject) {
  if (!fine || !coarse || !nnz) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_transfer: null argument");
  MgTransfer T;
  int rc;
  try {
    rc = pnp_mg_transfer(*fine, *coarse, T);
  } catch (const std::bad_alloc&) {
    PNP_FAIL(PNP_ERR_NOMEM, "pnp_mesh_transfer: out of host memory");
  }
  if (rc != PNP_OK) return rc;
  *nnz = (int64_t)T.p_col.size();
  if (ptr) std::copy(T.p_ptr.begin(), T.p_ptr.end(), ptr);
  if (col) std::copy(T.p_col.begin(), T.p_col.end(), col);
  if (w) std::copy(T.p_w.begin(), T.p_w.end(), w);
  if (inject) std::copy(T.inject.begin(), T.inject.end(), inject);
  return PNP_OK;
}

void pnp_mesh_destroy(pnp_mesh* m) { delete m; }

int pnp_mesh_info(const pnp_mesh* m, int* dim, int* max_level, int64_t* n_elem, int64_t* n_nodes,
                  int64_t* n_hanging) {
  if (!m) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_info: null mesh");
  if (dim) *dim = m->dim;
  if (max_level) *max_level = m->L;
  if (n_elem) *n_elem = m->n_elem;
  if (n_nodes) *n_nodes = m->n_nodes;
  if (n_hanging) *n_hanging = m->n_hanging;
  return PNP_OK;
}

int pnp_mesh_node_coords(const pnp_mesh* m, int32_t* ijk) {
  if (!m || !ijk) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_node_coords: null argument");
  std::memcpy(ijk, m->node_ijk.data(), m->node_ijk.size() * sizeof(int32_t));
  return PNP_OK;
}

int pnp_mesh_hanging(const pnp_mesh* m, uint8_t* flags) {
  if (!m || !flags) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_hanging: null argument");
  for (int64_t i = 0; i < m->n_nodes; ++i) flags[i] = m->node_hang[i] >= 0;
  return PNP_OK;
}

int pnp_mesh_patch_stats(const pnp_mesh* m, int64_t* stats) {
  if (!m || !stats) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_patch_stats: null argument");
  PatchData P;
  if (int rc = pnp_build_patches(*m, 256, 640, P)) return rc;
  stats[0] = P.n_patches;
  stats[1] = P.max_nodes;
  stats[2] = P.max_colors;
  stats[3] = (int64_t)P.bnode.size();
  stats[4] = P.n_partials;
  stats[5] = (int64_t)P.pnode.size();
  stats[6] = pnp_check_patches(*m, P);
  return PNP_OK;
}

int pnp_mesh_elements(const pnp_mesh* m, int32_t* anchors, uint8_t* levels) {
  if (!m) PNP_FAIL(PNP_ERR_ARG, "pnp_mesh_elements: null mesh");
  if (anchors) std::memcpy(anchors, m->el_anchor.data(), m->el_anchor.size() * sizeof(int32_t));
  if (levels) std::memcpy(levels, m->el_level.data(), m->el_level.size());
  return PNP_OK;
}

// ------------------------------------------------------------------ context
static int check_params(const pnp_params* p) {
  if (!p) PNP_FAIL(PNP_ERR_ARG, "null params");
  if (!(p->eps > 0) || !std::isfinite(p->eps)) PNP_FAIL(PNP_ERR_ARG, "params: eps must be > 0");
  if (!p->steady && (!(p->dt > 0) || !std::isfinite(p->dt))) PNP_FAIL(PNP_ERR_ARG, "params: dt must be > 0");
  if (!(p->C_I > 0)) PNP_FAIL(PNP_ERR_ARG, "params: C_I must be > 0");
  if (p->gmres_restart < 1 || p->gmres_restart > 200) PNP_FAIL(PNP_ERR_ARG, "params: gmres_restart in 1..200");
  if (p->gmres_max_it < 1) PNP_FAIL(PNP_ERR_ARG, "params: gmres_max_it >= 1");
  if (p->newton_max_it < 0) PNP_FAIL(PNP_ERR_ARG, "params: newton_max_it >= 0");
  if (p->precision != PNP_F64 && p->precision != PNP_F32) PNP_FAIL(PNP_ERR_ARG, "params: bad precision");
  if (p->start_mode < 0 || p->start_mode > 2) PNP_FAIL(PNP_ERR_ARG, "params: bad start_mode");
  if (p->bdf_order != 1 && p->bdf_order != 2) PNP_FAIL(PNP_ERR_ARG, "params: bdf_order must be 1 or 2");
  if (p->gmres_inner < 0 || p->gmres_inner > inner_max_depth())
    PNP_FAIL(PNP_ERR_ARG, "params: gmres_inner in 0..%d", inner_max_depth());
  if (p->mg_levels < 0 || p->mg_levels > 16 || p->mg_smooth < 1 || p->mg_smooth > 16 || !(p->mg_omega > 0) ||
      !(p->mg_omega <= 2) || p->mg_coarse_its < 1 || p->mg_coarse_its > 1000)
    PNP_FAIL(PNP_ERR_ARG, "params: multigrid settings out of range");
  if (p->dt_retries < 0 || p->dt_retries > 16) PNP_FAIL(PNP_ERR_ARG, "params: dt_retries in 0..16");
  if (p->ns_blocks < 1 || p->ns_blocks > 16 || !(p->ns_Sc > 0) || !std::isfinite(p->ns_Sc) ||
      !std::isfinite(p->ns_kappa) || !(p->ns_rtol >= 0) || !(p->ns_atol >= 0) || !(p->ns_inner_rtol > 0) ||
      !(p->ns_inner_rtol < 1) || p->ns_max_it < 1 || (p->ns_pin != 0 && p->ns_pin != 1) || p->ns_mg_levels < 0 ||
      p->ns_mg_levels > 16 || p->ns_inner_max_it < 1 || p->ns_fgmres < 0 || p->ns_fgmres > 200)
    PNP_FAIL(PNP_ERR_ARG, "params: Navier-Stokes settings out of range");
  return PNP_OK;
}

static void free_ctx_memory(pnp_ctx* c) {
  void* ptrs[] = {c->d_conn, c->d_anchor, c->d_level, c->d_faces, c->d_hnode, c->d_hpar, c->d_hnp, c->U, c->Uk, c->Ukm1,
                  c->adv, c->vel, c->vel_prev, c->hs, c->U32, c->adv32, c->hs32, c->V32, c->JV32, c->F,
                  c->dU, c->Ut, c->Ft, c->rhs, c->Dinv, c->D32, c->basis, c->w, c->z, c->r, c->part, c->dsc,
                  c->dflag, c->Zb, c->Qin, c->Dinv32, c->isc, c->iinv, c->rec32, c->V4, c->JV4, c->qp32,
                  c->Z64, c->Qin64, c->zin64, c->isc64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->pt_alloc) cudaFree(p);
  c->pt_alloc.clear();
  if (c->part64) cudaFree(c->part64);
  if (c->part32) cudaFree(c->part32);
  if (c->hpin) cudaFreeHost(c->hpin);
}

int pnp_ctx_create(const pnp_mesh* m, const pnp_params* p, void* stream, pnp_ctx** out) {
  if (!out) PNP_FAIL(PNP_ERR_ARG, "pnp_ctx_create: out is null");
  *out = nullptr;
  if (!m) PNP_FAIL(PNP_ERR_ARG, "pnp_ctx_create: null mesh");
  if (int rc = check_params(p)) return rc;
  pnp_ctx* c = new (std::nothrow) pnp_ctx();
  if (!c) PNP_FAIL(PNP_ERR_NOMEM, "pnp_ctx_create: out of host memory");
  c->dim = m->dim;
  c->L = m->L;
  c->n_elem = m->n_elem;
  c->n_nodes = m->n_nodes;
  c->n_hanging = m->n_hanging;
  c->prm = *p;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  const int nc = 1 << m->dim;
  const int64_t N = m->n_nodes;
  auto fail = [&](int rc) {
    free_ctx_memory(c);
    delete c;
    return rc;
  };
#define ALLOC(ptr, bytes)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 16);               \
    if (e_ != cudaSuccess) {                                                               \
      pnp_set_error("pnp_ctx_create: cudaMalloc(%zu) failed: %s", (size_t)(bytes),         \
                    cudaGetErrorString(e_));                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA);         \
    }                                                                                      \
  } while (0)
  ALLOC(c->d_conn, sizeof(int32_t) * m->n_elem * nc);
  ALLOC(c->d_level, m->n_elem);
  ALLOC(c->d_faces, N);
  ALLOC(c->d_hnode, sizeof(int32_t) * m->n_hanging);
  ALLOC(c->d_hpar, sizeof(int32_t) * 4 * m->n_hanging);
  ALLOC(c->d_hnp, m->n_hanging);
  const size_t v3 = sizeof(double) * 3 * N;
  ALLOC(c->U, v3);
  ALLOC(c->Uk, v3);
  ALLOC(c->Ukm1, v3);
  ALLOC(c->adv, v3);
  ALLOC(c->vel, v3);
  ALLOC(c->vel_prev, v3);
  ALLOC(c->hs, sizeof(double) * 2 * N);
  ALLOC(c->U32, sizeof(float) * 3 * N);
  ALLOC(c->adv32, sizeof(float) * 3 * N);
  ALLOC(c->hs32, sizeof(float) * 2 * N);
  ALLOC(c->rec32, sizeof(float4) * 2 * N);
  ALLOC(c->V32, sizeof(float) * 3 * N);
  ALLOC(c->JV32, sizeof(float) * 3 * N);
  ALLOC(c->F, v3);
  ALLOC(c->dU, v3);
  ALLOC(c->Ut, v3);
  ALLOC(c->Ft, v3);
  ALLOC(c->rhs, v3);
  ALLOC(c->Dinv, sizeof(double) * 9 * N);
  ALLOC(c->D32, sizeof(float) * 9 * N);
  ALLOC(c->w, v3);
  ALLOC(c->z, v3);
  ALLOC(c->r, v3);
  ALLOC(c->dflag, sizeof(int) * 4);
#undef ALLOC
  std::vector<uint8_t> faces(m->node_faces);
  for (int64_t i = 0; i < N; ++i)
    if (m->node_hang[i] >= 0) faces[i] |= 0x80;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (bytes && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dflag, 0, sizeof(int) * 4, s);
  up(c->d_conn, m->el_conn.data(), sizeof(int32_t) * m->el_conn.size());
  up(c->d_level, m->el_level.data(), m->el_level.size());
  up(c->d_faces, faces.data(), faces.size());
  up(c->d_hnode, m->hang_node.data(), sizeof(int32_t) * m->hang_node.size());
  up(c->d_hpar, m->hang_par.data(), sizeof(int32_t) * m->hang_par.size());
  up(c->d_hnp, m->hang_np.data(), m->hang_np.size());
  for (double* f : {c->U, c->Uk, c->Ukm1, c->adv, c->vel, c->vel_prev})
    if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, v3, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    pnp_set_error("pnp_ctx_create: upload failed: %s", cudaGetErrorString(e));
    return fail(PNP_ERR_CUDA);
  }
  if (int rc = ctx_alloc_krylov(c, p->gmres_restart)) return fail(rc);
  try {
    c->host_mesh = *m;
  } catch (const std::bad_alloc&) {
    pnp_set_error("pnp_ctx_create: out of host memory");
    return fail(PNP_ERR_NOMEM);
  }
  {
    // "patch": deterministic shared-memory patch kernels; default: per-element kernels
    // scattering with global atomics (faster on this hardware at present)
    const char* ep = getenv("PNP_ELEMENT_PATH");
    c->use_patches = ep && std::strcmp(ep, "patch") == 0;
  }
  if (c->use_patches) {
    PatchData P;
    if (int rc = pnp_build_patches(*m, 256, 640, P)) return fail(rc);
    DevPatches& d = c->pt;
    d.n_patches = P.n_patches;
    d.n_bnodes = (int64_t)P.bnode.size();
    d.n_partials = P.n_partials;
    d.max_nodes = P.max_nodes;
    auto upload = [&](const void* src, size_t bytes) -> void* {
      void* ptr = nullptr;
      if (e != cudaSuccess) return nullptr;
      e = cudaMalloc(&ptr, bytes > 0 ? bytes : 16);
      if (e != cudaSuccess) return nullptr;
      c->pt_alloc.push_back(ptr);
      if (bytes) e = cudaMemcpyAsync(ptr, src, bytes, cudaMemcpyHostToDevice, s);
      return ptr;
    };
    d.patch_e0 = (const int32_t*)upload(P.patch_e0.data(), 4 * P.patch_e0.size());
    d.patch_n0 = (const int32_t*)upload(P.patch_n0.data(), 4 * P.patch_n0.size());
    d.patch_h0 = (const int32_t*)upload(P.patch_h0.data(), 4 * P.patch_h0.size());
    d.patch_ncol = (const uint8_t*)upload(P.patch_ncol.data(), P.patch_ncol.size());
    d.pnode = (const int32_t*)upload(P.pnode.data(), 4 * P.pnode.size());
    d.pbslot = (const int32_t*)upload(P.pbslot.data(), 4 * P.pbslot.size());
    d.el_slot = (const uint16_t*)upload(P.el_slot.data(), 2 * P.el_slot.size());
    d.el_color = (const uint8_t*)upload(P.el_color.data(), P.el_color.size());
    d.hc_np = (const uint8_t*)upload(P.hc_np.data(), P.hc_np.size());
    d.hc_par = (const uint16_t*)upload(P.hc_par.data(), 2 * P.hc_par.size());
    d.bnode = (const int32_t*)upload(P.bnode.data(), 4 * P.bnode.size());
    d.bptr = (const int32_t*)upload(P.bptr.data(), 4 * P.bptr.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->part64, sizeof(double) * 3 * std::max<int64_t>(1, P.n_partials));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->part32, sizeof(float) * 3 * std::max<int64_t>(1, P.n_partials));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      pnp_set_error("pnp_ctx_create: patch upload failed: %s", cudaGetErrorString(e));
      return fail(e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA);
    }
  }
  *out = c;
  return PNP_OK;
}

}  // extern "C"

int ctx_alloc_krylov(pnp_ctx* c, int m) {
  if (m <= c->m_alloc) return PNP_OK;
  if (c->basis) cudaFree(c->basis);
  if (c->part) cudaFree(c->part);
  if (c->dsc) cudaFree(c->dsc);
  if (c->hpin) cudaFreeHost(c->hpin);
  c->basis = nullptr;
  c->part = nullptr;
  c->dsc = nullptr;
  c->hpin = nullptr;
  c->m_alloc = 0;
  const size_t bb = sizeof(double) * (size_t)(m + 1) * (size_t)c->n3();
  cudaError_t e = cudaMalloc((void**)&c->basis, bb);
  const size_t part_rows =
      std::max<size_t>(std::max<size_t>((size_t)kRedBlocks, (size_t)kInnerBlocks), (size_t)multi_dot_blocks(c->n3()));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->part, sizeof(double) * part_rows * (m + 2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->dsc, sizeof(double) * (4 * (m + 2) + 16));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hpin, sizeof(double) * (4 * (m + 2) + 16));
  if (e != cudaSuccess) {
    pnp_set_error("Krylov scratch allocation (%zu bytes) failed: %s", bb, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA;
  }
  c->basis_bytes = (int64_t)bb;
  c->m_alloc = m;
  return PNP_OK;
}

// Buffers of the flexible outer GMRES(m) with an inner FP32 GMRES(d).
int ctx_alloc_inner(pnp_ctx* c, int m, int d) {
  if (m <= c->inner_m && d <= c->inner_d) return PNP_OK;
  m = std::max(m, c->inner_m);
  d = std::max(d, c->inner_d);
  if (int rc = ctx_alloc_krylov(c, std::max(c->m_alloc, d))) return rc;  // partials for d projections
  void* old[] = {c->Zb, c->Qin, c->Dinv32, c->isc, c->iinv, c->V4, c->JV4, c->qp32};
  for (void* q : old)
    if (q) cudaFree(q);
  c->Zb = c->Qin = c->Dinv32 = c->iinv = nullptr;
  c->isc = nullptr;
  c->V4 = c->JV4 = c->qp32 = nullptr;
  c->inner_m = c->inner_d = 0;
  const size_t n = (size_t)c->n3();
  cudaError_t e = cudaMalloc((void**)&c->Zb, sizeof(float) * (size_t)m * n);
  c->ldq = (int64_t)((n + 3) & ~(size_t)3);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->Qin, sizeof(float) * (size_t)(d + 1) * (size_t)c->ldq);
  if (e == cudaSuccess) e = cudaMemset(c->Qin, 0, sizeof(float) * (size_t)(d + 1) * (size_t)c->ldq);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->Dinv32, sizeof(float) * 9 * (size_t)c->n_nodes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->isc, sizeof(double) * (inner_scalar_doubles(d) + 5 * (size_t)(d + 2)));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->iinv, sizeof(float) * (size_t)(d + 2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->V4, sizeof(float4) * (size_t)c->n_nodes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->JV4, sizeof(float4) * (size_t)c->n_nodes);
  if (e == cudaSuccess) e = cudaMemset(c->JV4, 0, sizeof(float4) * (size_t)c->n_nodes);
  // the stored linearisation (qp32) is allocated by its first use (ctx_linearize32)
  if (e != cudaSuccess) {
    pnp_set_error("inner Krylov scratch allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA;
  }
  c->inner_m = m;
  c->inner_d = d;
  return PNP_OK;
}

int ctx_alloc_inner64(pnp_ctx* c, int m, int d) {
  if (m <= c->inner64_m && d <= c->inner64_d) return PNP_OK;
  m = std::max(m, c->inner64_m);
  d = std::max(d, c->inner64_d);
  if (int rc = ctx_alloc_krylov(c, std::max(c->m_alloc, d))) return rc;  // partials for d projections
  void* old[] = {c->Z64, c->Qin64, c->zin64, c->isc64};
  for (void* q : old)
    if (q) cudaFree(q);
  c->Z64 = c->Qin64 = c->zin64 = c->isc64 = nullptr;
  c->inner64_m = c->inner64_d = 0;
  const size_t n = (size_t)c->n3();
  cudaError_t e = cudaMalloc((void**)&c->Z64, sizeof(double) * (size_t)m * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->Qin64, sizeof(double) * (size_t)(d + 1) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->zin64, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->isc64, sizeof(double) * (3 * (size_t)(d + 2) + 2));
  if (e != cudaSuccess) {
    pnp_set_error("inner FP64 Krylov scratch allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA;
  }
  c->inner64_m = m;
  c->inner64_d = d;
  return PNP_OK;
}

extern "C" {

void pnp_ctx_destroy(pnp_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  pnp_mlp_release(c);
  ctx_mg_release(c);
  ctx_ns_release(c);
  for (auto& pe : c->ev_pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->inner_exec) cudaGraphExecDestroy(c->inner_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  free_ctx_memory(c);
  delete c;
}

int pnp_set_params(pnp_ctx* c, const pnp_params* p) {
  CTX_GUARD(c);
  if (int rc = check_params(p)) return rc;
  if (int rc = ctx_alloc_krylov(c, p->gmres_restart)) return rc;
  c->prm = *p;
  return PNP_OK;
}

int pnp_get_params(const pnp_ctx* c, pnp_params* p) {
  if (!c || !p) PNP_FAIL(PNP_ERR_ARG, "pnp_get_params: null argument");
  *p = c->prm;
  return PNP_OK;
}

int pnp_set_bc(pnp_ctx* c, int face, int field, int type, double value) {
  CTX_GUARD(c);
  if (face < 0 || face >= 2 * c->dim) PNP_FAIL(PNP_ERR_ARG, "pnp_set_bc: face %d out of range", face);
  if (field < 0 || field > 2) PNP_FAIL(PNP_ERR_ARG, "pnp_set_bc: field %d out of range", field);
  if (type != PNP_NATURAL && type != PNP_DIRICHLET) PNP_FAIL(PNP_ERR_ARG, "pnp_set_bc: bad type %d", type);
  if (!std::isfinite(value)) PNP_FAIL(PNP_ERR_ARG, "pnp_set_bc: value not finite");
  c->bc_type[face][field] = type;
  c->bc_val[face][field] = value;
  return PNP_OK;
}

int pnp_ns_set_bc(pnp_ctx* c, int face, int slot, int type, double value) {
  CTX_GUARD(c);
  if (face < 0 || face >= 2 * c->dim) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_set_bc: face %d out of range", face);
  if (slot < 0 || slot > 3) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_set_bc: slot %d out of range", slot);
  if (type != PNP_NATURAL && type != PNP_DIRICHLET) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_set_bc: bad type %d", type);
  if (!std::isfinite(value)) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_set_bc: value not finite");
  c->ns_bc_type[face][slot] = type;
  c->ns_bc_val[face][slot] = value;
  return PNP_OK;
}

static double* field_ptr(pnp_ctx* c, int which) {
  switch (which) {
    case PNP_FIELD_U: return c->U;
    case PNP_FIELD_U_PREV: return c->Uk;
    case PNP_FIELD_U_PREV2: return c->Ukm1;
    case PNP_FIELD_ADVECTION: return c->adv;
    case PNP_FIELD_VELOCITY: return c->vel;
    case PNP_FIELD_VELOCITY_PREV: return c->vel_prev;
  }
  return nullptr;
}

int pnp_set_field(pnp_ctx* c, int which, const double* src, int where) {
  CTX_GUARD(c);
  if (which == PNP_FIELD_NS) {
    if (!src || (where != PNP_DEVICE && where != PNP_HOST)) PNP_FAIL(PNP_ERR_ARG, "pnp_set_field: bad arguments");
    if (int rc = ctx_ns_alloc(c)) return rc;
    CK(cudaMemcpyAsync(ctx_ns_field(c), src, sizeof(double) * 4 * c->n_nodes,
                       where == PNP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PNP_OK;
  }
  double* dst = field_ptr(c, which);
  if (!dst || !src) PNP_FAIL(PNP_ERR_ARG, "pnp_set_field: bad field %d or null source", which);
  if (where != PNP_DEVICE && where != PNP_HOST) PNP_FAIL(PNP_ERR_ARG, "pnp_set_field: bad where");
  const bool is_vel = which >= PNP_FIELD_ADVECTION;
  const int64_t N = c->n_nodes;
  const cudaMemcpyKind kind = where == PNP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!is_vel || c->dim == 3) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * 3 * N, kind, c->stream));
  } else {
    // [N][dim] -> [N][3] through scratch (w)
    CK(cudaMemcpyAsync(c->w, src, sizeof(double) * c->dim * N, kind, c->stream));
    CK(launch_vel_pack(N, c->dim, c->w, dst, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_get_field(pnp_ctx* c, int which, double* dstp, int where) {
  CTX_GUARD(c);
  if (which == PNP_FIELD_NS) {
    if (!dstp || (where != PNP_DEVICE && where != PNP_HOST)) PNP_FAIL(PNP_ERR_ARG, "pnp_get_field: bad arguments");
    if (int rc = ctx_ns_alloc(c)) return rc;
    CK(cudaMemcpyAsync(dstp, ctx_ns_field(c), sizeof(double) * 4 * c->n_nodes,
                       where == PNP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PNP_OK;
  }
  double* src = field_ptr(c, which);
  if (!src || !dstp) PNP_FAIL(PNP_ERR_ARG, "pnp_get_field: bad field %d or null destination", which);
  if (where != PNP_DEVICE && where != PNP_HOST) PNP_FAIL(PNP_ERR_ARG, "pnp_get_field: bad where");
  const bool is_vel = which >= PNP_FIELD_ADVECTION;
  const int64_t N = c->n_nodes;
  const cudaMemcpyKind kind = where == PNP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (!is_vel || c->dim == 3) {
    CK(cudaMemcpyAsync(dstp, src, sizeof(double) * 3 * N, kind, c->stream));
  } else {
    CK(launch_vel_unpack(N, c->dim, src, c->w, c->stream));
    CK(cudaMemcpyAsync(dstp, c->w, sizeof(double) * c->dim * N, kind, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_make_consistent(pnp_ctx* c) {
  CTX_GUARD(c);
  CK(launch_make_consistent(c->rows(), c->U, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

// ------------------------------------------------------------------ operators
int pnp_residual(pnp_ctx* c, const double* U, double* F) {
  CTX_GUARD(c);
  if (!U || !F) PNP_FAIL(PNP_ERR_ARG, "pnp_residual: null pointer");
  if (int rc = ctx_prepare_history(c)) return rc;
  if (int rc = ctx_residual(c, U, F)) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_jv(pnp_ctx* c, const double* U, const void* V, void* JV, int precision) {
  CTX_GUARD(c);
  if (!U || !V || !JV) PNP_FAIL(PNP_ERR_ARG, "pnp_jv: null pointer");
  if (int rc = ctx_prepare_history(c)) return rc;
  if (precision == PNP_F64) {
    if (int rc = ctx_jv64(c, U, (const double*)V, (double*)JV)) return rc;
  } else if (precision == PNP_F32) {
    if (int rc = ctx_prepare_f32(c, U)) return rc;
    if (int rc = ctx_jv32(c, (const float*)V, (float*)JV)) return rc;
  } else {
    PNP_FAIL(PNP_ERR_ARG, "pnp_jv: bad precision %d", precision);
  }
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_linearize(pnp_ctx* c, const double* U) {
  CTX_GUARD(c);
  if (!U) PNP_FAIL(PNP_ERR_ARG, "pnp_linearize: null pointer");
  if (int rc = ctx_alloc_inner(c, c->prm.gmres_restart, std::max(1, c->prm.gmres_inner))) return rc;
  if (int rc = ctx_prepare_history(c)) return rc;
  if (int rc = ctx_prepare_f32(c, U)) return rc;
  if (int rc = ctx_linearize32(c)) return rc;
  c->lin_user = true;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_jv_linearized(pnp_ctx* c, const float* V, float* JV) {
  CTX_GUARD(c);
  if (!V || !JV) PNP_FAIL(PNP_ERR_ARG, "pnp_jv_linearized: null pointer");
  if (!c->lin_user) PNP_FAIL(PNP_ERR_STATE, "pnp_jv_linearized: no stored linearisation (call pnp_linearize)");
  if (int rc = ctx_jv32_linearized(c, V, JV)) return rc;
  return ctx_check_staged_waits(c);
}

int pnp_block_diag(pnp_ctx* c, const double* U, double* D) {
  CTX_GUARD(c);
  if (!U || !D) PNP_FAIL(PNP_ERR_ARG, "pnp_block_diag: null pointer");
  if (int rc = ctx_prepare_history(c)) return rc;
  if (int rc = ctx_block_diag(c, U, D)) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_block_diag_f32(pnp_ctx* c, const double* U, float* D) {
  CTX_GUARD(c);
  if (!U || !D) PNP_FAIL(PNP_ERR_ARG, "pnp_block_diag_f32: null pointer");
  if (int rc = ctx_prepare_history(c)) return rc;
  if (int rc = ctx_prepare_f32(c, U)) return rc;
  if (int rc = ctx_block_diag32(c, D)) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_boundary_flux(pnp_ctx* c, const double* U, int face, double* flux) {
  CTX_GUARD(c);
  if (!U || !flux) PNP_FAIL(PNP_ERR_ARG, "pnp_boundary_flux: null pointer");
  if (face < 0 || face >= 2 * c->dim) PNP_FAIL(PNP_ERR_ARG, "pnp_boundary_flux: face %d out of range", face);
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 12;
  CK(launch_boundary_flux(c->dim, c->n_elem, c->d_conn, c->d_level, c->d_faces, c->d_hnode, c->d_hpar, c->d_hnp, U,
                          face, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin + 2, slot, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  flux[0] = c->hpin[2];
  flux[1] = c->hpin[3];
  return PNP_OK;
}

int pnp_element_gradient(pnp_ctx* c, const double* U, double* G) {
  CTX_GUARD(c);
  if (!U || (!G && c->n_elem)) PNP_FAIL(PNP_ERR_ARG, "pnp_element_gradient: null pointer");
  CK(launch_element_gradient(c->dim, c->n_elem, c->d_conn, c->d_level, c->d_hpar, c->d_hnp, U, G, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_plane_average(pnp_ctx* c, const double* U, int axis, int64_t coord, double* avg) {
  CTX_GUARD(c);
  if (!U || !avg) PNP_FAIL(PNP_ERR_ARG, "pnp_plane_average: null pointer");
  if (axis < 0 || axis >= c->dim) PNP_FAIL(PNP_ERR_ARG, "pnp_plane_average: axis %d out of range", axis);
  const int L = c->host_mesh.L;
  const int64_t size = int64_t(1) << L;
  const bool per = (c->host_mesh.periodic >> axis) & 1;
  if (coord < 0 || coord > size || (per && coord == size))
    PNP_FAIL(PNP_ERR_ARG, "pnp_plane_average: coordinate %lld outside the domain", (long long)coord);
  if (!c->d_anchor) {
    const size_t bytes = sizeof(int32_t) * c->host_mesh.el_anchor.size();
    CK(cudaMalloc((void**)&c->d_anchor, bytes));
    CK(cudaMemcpyAsync(c->d_anchor, c->host_mesh.el_anchor.data(), bytes, cudaMemcpyHostToDevice, c->stream));
  }
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 12;
  CK(launch_plane_integral(c->dim, L, c->n_elem, c->d_conn, c->d_level, c->d_anchor, c->d_hnode, c->d_hpar, c->d_hnp,
                           U, axis, coord, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin + 2, slot, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // the plane's area is 1 on the unit domain
  for (int f = 0; f < 3; ++f) avg[f] = c->hpin[2 + f];
  return PNP_OK;
}

int pnp_norm2(pnp_ctx* c, const double* x, int64_t n, double* result) {
  CTX_GUARD(c);
  if (!result || n < 0 || (!x && n > 0)) PNP_FAIL(PNP_ERR_ARG, "pnp_norm2: bad arguments");
  if (n == 0) {
    *result = 0.0;
    return PNP_OK;
  }
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 9;
  CK(launch_norm2(n, x, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin + 1, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *result = c->hpin[1];
  return PNP_OK;
}

int pnp_gmres(pnp_ctx* c, const double* U, const double* b, double* x, double rtol, int precision,
              pnp_solve_stats* st) {
  CTX_GUARD(c);
  if (!U || !b || !x) PNP_FAIL(PNP_ERR_ARG, "pnp_gmres: null pointer");
  if (precision != PNP_F64 && precision != PNP_F32) PNP_FAIL(PNP_ERR_ARG, "pnp_gmres: bad precision");
  if (!(rtol > 0)) PNP_FAIL(PNP_ERR_ARG, "pnp_gmres: rtol must be > 0");
  if (int rc = ctx_prepare_history(c)) return rc;
  int its = 0;
  double rel = 0;
  c->jv_count = 0;
  c->mg_fallbacks = 0;
  const int rc = ctx_gmres(c, U, b, x, rtol, precision, c->prm.gmres_max_it, &its, &rel, false);
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->status = rc;
    st->krylov_its = its;
    st->jv_evals = c->jv_count;
    st->res_final = rel;
    st->mg_fallbacks = c->mg_fallbacks;
  }
  return rc;
}

int pnp_newton_solve(pnp_ctx* c, pnp_solve_stats* st) {
  CTX_GUARD(c);
  pnp_solve_stats local;
  return ctx_newton(c, st ? st : &local);
}

int pnp_time_step(pnp_ctx* c, pnp_solve_stats* st) {
  CTX_GUARD(c);
  pnp_solve_stats local;
  return ctx_time_step(c, st ? st : &local);
}

// ------------------------------------------------------------------ Navier-Stokes
int pnp_ns_residual(pnp_ctx* c, const double* X, double* F) {
  CTX_GUARD(c);
  if (!X || !F) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_residual: null pointer");
  if (int rc = ctx_ns_prepare(c)) return rc;
  if (int rc = ctx_ns_apply64(c, X, c->U, F, true)) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_ns_matvec(pnp_ctx* c, const void* X, void* Y, int precision) {
  CTX_GUARD(c);
  if (!X || !Y) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_matvec: null pointer");
  if (precision != PNP_F64 && precision != PNP_F32) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_matvec: bad precision");
  if (precision == PNP_F32 && (((uintptr_t)X | (uintptr_t)Y) & 15))
    PNP_FAIL(PNP_ERR_ARG, "pnp_ns_matvec: FP32 vectors must be 16-byte aligned");
  if (int rc = ctx_ns_prepare(c)) return rc;
  if (precision == PNP_F64) {
    if (int rc = ctx_ns_apply64(c, (const double*)X, nullptr, (double*)Y, false)) return rc;
  } else {
    if (int rc = ctx_ns_apply32(c, (const float4*)X, (float4*)Y)) return rc;
  }
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_ns_block_diag(pnp_ctx* c, double* D) {
  CTX_GUARD(c);
  if (!D) PNP_FAIL(PNP_ERR_ARG, "pnp_ns_block_diag: null pointer");
  if (int rc = ctx_ns_prepare(c)) return rc;
  if (int rc = ctx_ns_block_diag(c, D)) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_ns_solve(pnp_ctx* c, pnp_ns_stats* st) {
  CTX_GUARD(c);
  pnp_ns_stats local;
  return ctx_ns_solve(c, c->U, st ? st : &local);
}

int pnp_coupled_step(pnp_ctx* c, pnp_solve_stats* pst, pnp_ns_stats* nst) {
  CTX_GUARD(c);
  pnp_solve_stats lp;
  pnp_ns_stats ln;
  return ctx_coupled_step(c, pst ? pst : &lp, nst ? nst : &ln);
}

int pnp_step_count(const pnp_ctx* c, int64_t* k) {
  if (!c || !k) PNP_FAIL(PNP_ERR_ARG, "pnp_step_count: null argument");
  *k = c->step;
  return PNP_OK;
}

int pnp_set_wait_limit(pnp_ctx* c, int64_t polls) {
  if (!c) PNP_FAIL(PNP_ERR_ARG, "pnp_set_wait_limit: null context");
  if (polls > (int64_t(1) << 30)) PNP_FAIL(PNP_ERR_ARG, "pnp_set_wait_limit: at most 2^30 polls");
  c->wait_polls = polls < 0 ? -1 : (int)polls;
  return PNP_OK;
}

int pnp_set_step_count(pnp_ctx* c, int64_t k) {
  if (!c || k < 0) PNP_FAIL(PNP_ERR_ARG, "pnp_set_step_count: bad argument");
  c->step = k;
  c->history_split = false;
  return PNP_OK;
}

static void resolve_events(pnp_ctx* c) {
  for (auto& pe : c->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      c->prof_ms[pe.first] += ms;
      c->prof_cnt[pe.first] += 1;
    }
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->ev_pending.clear();
}

int pnp_profile_enable(pnp_ctx* c, int on) {
  CTX_GUARD(c);
  CK(cudaStreamSynchronize(c->stream));
  resolve_events(c);
  if (on) {
    for (int k = 0; k < PNP_PROF_KINDS; ++k) {
      c->prof_ms[k] = 0;
      c->prof_cnt[k] = 0;
      c->prof_bytes[k] = 0;
      c->prof_flops[k] = 0;
    }
  }
  c->prof_on = on != 0;
  return PNP_OK;
}

int pnp_profile_read(pnp_ctx* c, int kind, double* total_ms, int64_t* count, double* alg_bytes,
                     double* alg_flops) {
  CTX_GUARD(c);
  if (kind < 0 || kind >= PNP_PROF_KINDS) PNP_FAIL(PNP_ERR_ARG, "pnp_profile_read: bad kind %d", kind);
  CK(cudaStreamSynchronize(c->stream));
  resolve_events(c);
  if (total_ms) *total_ms = c->prof_ms[kind];
  if (count) *count = c->prof_cnt[kind];
  if (alg_bytes) *alg_bytes = c->prof_bytes[kind];
  if (alg_flops) *alg_flops = c->prof_flops[kind];
  return PNP_OK;
}

int pnp_reset_history(pnp_ctx* c) {
  CTX_GUARD(c);
  CK(cudaMemcpyAsync(c->Uk, c->U, sizeof(double) * c->n3(), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->Ukm1, c->U, sizeof(double) * c->n3(), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->step = 0;
  c->history_split = false;
  return PNP_OK;
}

}  // extern "C"
