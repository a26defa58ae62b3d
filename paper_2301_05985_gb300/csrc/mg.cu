// mg.cu -- geometric multigrid on the octree hierarchy as the preconditioner of the
// flexible Krylov solve (FP32), in place of the paper's algebraic multigrid (GAMG, App. A).
//
// Levels: level 0 is the context's mesh; level l > 0 is the octree with every leaf finer
// than (max level - l) replaced by its ancestor at that level (mg_build.cpp), with a
// context of its own.  Each level's operator is the same linearised PNP operator
// rediscretised on that level's mesh (the FP32 J V kernels), at the state injected from
// the finest level (U^{k+1} iterate, U^k, U^{k-1} and the advection at the coarse nodes'
// points).  Transfers: prolongation by trilinear interpolation of the coarse Q1 field at
// the fine nodes, restriction by its transpose; Dirichlet rows of restricted residuals and
// prolongated corrections are zero.  Smoother: damped 3x3 block Jacobi (the diagonal
// blocks of each level's operator).  One V-cycle per preconditioner application, from a
// zero initial guess, with a fixed number of sweeps: a fixed linear operator.
#include <algorithm>
#include <cstring>

#include "ctx.h"

#define CK(call)                                 \
  do {                                           \
    int _rc = ctx_check(c, (call), #call);       \
    if (_rc) return _rc;                         \
  } while (0)
#define RC(call)              \
  do {                        \
    int _rc = (call);         \
    if (_rc) return _rc;      \
  } while (0)

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// x = omega D^-1 b (first) or x += omega D^-1 (b - Ax), per node (3x3 blocks)
__global__ void k_mg_smooth(int64_t N, const float* __restrict__ Dinv, const float* __restrict__ b,
                            const float* __restrict__ Ax, float* __restrict__ x, float omega, int first) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float r[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) r[f] = first ? b[3 * i + f] : b[3 * i + f] - Ax[3 * i + f];
  const float* D = Dinv + 9 * i;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float d = omega * (D[3 * f] * r[0] + D[3 * f + 1] * r[1] + D[3 * f + 2] * r[2]);
    x[3 * i + f] = first ? d : x[3 * i + f] + d;
  }
}

// Dirichlet bit of field f at a node (faces: boundary-face bits, bit 7 hanging)
__device__ __forceinline__ bool dir_row(const BcTable& bc, uint8_t faces, int f) {
  return (faces & bc.dir_faces[f] & 0x3F) != 0;
}

// bc[j] = sum_q w_q (b - Ax)[col_q] over the fine rows that are weak-form equations:
// Dirichlet rows (U - g) and hanging rows (constraints) carry no element contributions
// and are left out; coarse Dirichlet rows are zero
__global__ void k_mg_restrict(int64_t Nc, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ w, const float* __restrict__ b, const float* __restrict__ Ax,
                              const uint8_t* __restrict__ faces_f, BcTable bcf, const uint8_t* __restrict__ faces_c,
                              BcTable bc, float* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= Nc) return;
  float s[3] = {0.f, 0.f, 0.f};
  for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) {
    const int64_t i = col[q];
    const uint8_t ff = faces_f[i];
    if (ff & 0x80) continue;  // hanging
    const float wq = w[q];
#pragma unroll
    for (int f = 0; f < 3; ++f)
      if (!dir_row(bcf, ff, f)) s[f] = fmaf(wq, b[3 * i + f] - Ax[3 * i + f], s[f]);
  }
  const uint8_t fc = faces_c[j];
#pragma unroll
  for (int f = 0; f < 3; ++f) out[3 * j + f] = dir_row(bc, fc, f) ? 0.f : s[f];
}

// x[i] += sum_q w_q xc[col_q]  (fine rows; Dirichlet rows untouched)
__global__ void k_mg_prolong_add(int64_t Nf, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const float* __restrict__ w, const float* __restrict__ xc,
                                 const uint8_t* __restrict__ faces_f, BcTable bc, float* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Nf) return;
  float s[3] = {0.f, 0.f, 0.f};
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int64_t j = col[q];
    const float wq = w[q];
#pragma unroll
    for (int f = 0; f < 3; ++f) s[f] = fmaf(wq, xc[3 * j + f], s[f]);
  }
  const uint8_t ff = faces_f[i];
#pragma unroll
  for (int f = 0; f < 3; ++f)
    if (!dir_row(bc, ff, f)) x[3 * i + f] += s[f];
}

// coarse[j] = fine[map[j]] for vectors of nf components per node
__global__ void k_mg_inject(int64_t Nc, int nf, const int32_t* __restrict__ map, const double* __restrict__ fine,
                            double* __restrict__ coarse) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Nc * nf) return;
  const int64_t j = t / nf;
  const int f = (int)(t - j * nf);
  coarse[t] = fine[(int64_t)map[j] * nf + f];
}

}  // namespace

static void mg_free_level(MgLevel& L) {
  void* p[] = {L.p_ptr, L.p_col, L.p_w, L.r_ptr, L.r_col, L.r_w, L.inject, L.b, L.x, L.Ax, L.Dinv32};
  for (void* q : p)
    if (q) cudaFree(q);
  if (L.sub) pnp_ctx_destroy(L.sub);
  L = MgLevel();
}

void ctx_mg_release(pnp_ctx* c) {
  if (!c->mg) return;
  for (auto& L : *c->mg) mg_free_level(L);
  delete c->mg;
  c->mg = nullptr;
  c->mg_built = 0;
}

// Build the hierarchy (host meshes, level contexts, transfers) for `levels` coarse levels.
int ctx_mg_setup(pnp_ctx* c, int levels) {
  if (c->mg && c->mg_built == levels) return PNP_OK;
  ctx_mg_release(c);
  if (c->host_mesh.periodic) PNP_FAIL(PNP_ERR_ARG, "multigrid: periodic meshes are not supported");
  c->mg = new std::vector<MgLevel>();
  auto& lv = *c->mg;
  lv.emplace_back();
  const int64_t N0 = c->n_nodes;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  };
  A((void**)&lv[0].b, sizeof(float) * 3 * N0);
  A((void**)&lv[0].x, sizeof(float) * 3 * N0);
  A((void**)&lv[0].Ax, sizeof(float) * 3 * N0);
  A((void**)&lv[0].Dinv32, sizeof(float) * 9 * N0);
  int lmax = 0;
  for (uint8_t l : c->host_mesh.el_level) lmax = std::max<int>(lmax, l);
  const pnp_mesh* fine = &c->host_mesh;
  pnp_mesh coarse_mesh;
  for (int l = 1; l <= levels && e == cudaSuccess; ++l) {
    const int cap = lmax - l;
    if (cap < 1) break;
    pnp_mesh cm;
    if (int rc = pnp_cap_mesh_levels(*fine, cap, cm)) {
      ctx_mg_release(c);
      return rc;
    }
    if (cm.n_elem == fine->n_elem) break;  // nothing left to coarsen
    MgTransfer T;
    if (int rc = pnp_mg_transfer(*fine, cm, T)) {
      ctx_mg_release(c);
      return rc;
    }
    pnp_params p = c->prm;
    p.gmres_restart = 2;
    p.gmres_inner = 0;
    p.mg_levels = 0;
    MgLevel L;
    if (int rc = pnp_ctx_create(&cm, &p, c->stream, &L.sub)) {
      ctx_mg_release(c);
      return rc;
    }
    std::memcpy(L.sub->bc_type, c->bc_type, sizeof(c->bc_type));
    std::memcpy(L.sub->bc_val, c->bc_val, sizeof(c->bc_val));
    const int64_t Nc = cm.n_nodes;
    A((void**)&L.p_ptr, sizeof(int64_t) * T.p_ptr.size());
    A((void**)&L.p_col, sizeof(int32_t) * T.p_col.size());
    A((void**)&L.p_w, sizeof(float) * T.p_w.size());
    A((void**)&L.r_ptr, sizeof(int64_t) * T.r_ptr.size());
    A((void**)&L.r_col, sizeof(int32_t) * T.r_col.size());
    A((void**)&L.r_w, sizeof(float) * T.r_w.size());
    A((void**)&L.inject, sizeof(int32_t) * T.inject.size());
    A((void**)&L.b, sizeof(float) * 3 * Nc);
    A((void**)&L.x, sizeof(float) * 3 * Nc);
    A((void**)&L.Ax, sizeof(float) * 3 * Nc);
    A((void**)&L.Dinv32, sizeof(float) * 9 * Nc);
    auto up = [&](void* d, const void* h, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream);
    };
    up(L.p_ptr, T.p_ptr.data(), sizeof(int64_t) * T.p_ptr.size());
    up(L.p_col, T.p_col.data(), sizeof(int32_t) * T.p_col.size());
    up(L.p_w, T.p_w.data(), sizeof(float) * T.p_w.size());
    up(L.r_ptr, T.r_ptr.data(), sizeof(int64_t) * T.r_ptr.size());
    up(L.r_col, T.r_col.data(), sizeof(int32_t) * T.r_col.size());
    up(L.r_w, T.r_w.data(), sizeof(float) * T.r_w.size());
    up(L.inject, T.inject.data(), sizeof(int32_t) * T.inject.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors go out of scope
    lv.push_back(L);
    fine = &lv.back().sub->host_mesh;
  }
  if (e != cudaSuccess) {
    ctx_mg_release(c);
    PNP_FAIL(e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA, "multigrid set-up: %s",
             cudaGetErrorString(e));
  }
  c->mg_built = levels;
  return PNP_OK;
}

static int mg_blocks(pnp_ctx* c, const double* U, float* Dinv32) {
  RC(ctx_prepare_f32(c, U));
  RC(ctx_block_diag32(c, c->D32));
  CK(launch_block_invert<float>(c->n_nodes, c->D32, c->Dinv, c->dflag, c->stream));
  CK(launch_to_f32(9 * c->n_nodes, c->Dinv, Dinv32, c->stream));
  return PNP_OK;
}

// Per Krylov solve: the state on every level and each level's inverted block diagonal
// (level 0's from the block-Jacobi set-up of the solve, which runs first).
int ctx_mg_prepare(pnp_ctx* c, const double* U) {
  auto& lv = *c->mg;
  cudaStream_t s = c->stream;
  // level 0: the inverted blocks of the solve's block-Jacobi set-up (build_preconditioner)
  CK(launch_to_f32(9 * c->n_nodes, c->Dinv, lv[0].Dinv32, s));
  const pnp_ctx* fine = c;
  const double* Uf = U;
  for (size_t l = 1; l < lv.size(); ++l) {
    pnp_ctx* sc = lv[l].sub;
    sc->prm.eps = c->prm.eps;
    sc->prm.dt = c->prm.dt;
    sc->prm.C_I = c->prm.C_I;
    sc->prm.beta0 = c->prm.beta0;
    sc->prm.beta1 = c->prm.beta1;
    sc->prm.beta2 = c->prm.beta2;
    sc->prm.steady = c->prm.steady;
    std::memcpy(sc->bc_type, c->bc_type, sizeof(c->bc_type));
    std::memcpy(sc->bc_val, c->bc_val, sizeof(c->bc_val));
    const int64_t Nc = sc->n_nodes;
    const unsigned g = nblk(3 * Nc, 256);
    k_mg_inject<<<g, 256, 0, s>>>(Nc, 3, lv[l].inject, Uf, sc->U);
    k_mg_inject<<<g, 256, 0, s>>>(Nc, 3, lv[l].inject, fine->Uk, sc->Uk);
    k_mg_inject<<<g, 256, 0, s>>>(Nc, 3, lv[l].inject, fine->Ukm1, sc->Ukm1);
    k_mg_inject<<<g, 256, 0, s>>>(Nc, 3, lv[l].inject, fine->adv, sc->adv);
    note_launches(4);
    CK(cudaGetLastError());
    RC(ctx_prepare_history(sc));
    CK(cudaMemsetAsync(sc->dflag, 0, sizeof(int), s));
    RC(mg_blocks(sc, sc->U, lv[l].Dinv32));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, sc->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag) PNP_FAIL(PNP_ERR_NAN, "multigrid level %zu: singular or non-finite 3x3 block", l);
    fine = sc;
    Uf = sc->U;
  }
  return PNP_OK;
}

static int mg_cycle(pnp_ctx* c, size_t l) {
  auto& lv = *c->mg;
  MgLevel& L = lv[l];
  pnp_ctx* lc = l == 0 ? c : L.sub;
  const int64_t N = lc->n_nodes;
  cudaStream_t s = c->stream;
  const float om = (float)c->prm.mg_omega;
  const unsigned g = nblk(N, 256);
  auto smooth = [&](bool first) -> int {
    if (!first) RC(ctx_jv32(lc, L.x, L.Ax));
    ProfScope ps(c, l == 0 ? PNP_PROF_PRECOND : -1, 48.0 * N, 24.0 * N);
    k_mg_smooth<<<g, 256, 0, s>>>(N, L.Dinv32, L.b, L.Ax, L.x, om, first ? 1 : 0);
    note_launch();
    CK(cudaGetLastError());
    return PNP_OK;
  };
  if (l + 1 == lv.size()) {
    const int sweeps = std::max(1, c->prm.mg_coarse_its);
    for (int k = 0; k < sweeps; ++k) RC(smooth(k == 0));
    return PNP_OK;
  }
  const int nu = std::max(1, c->prm.mg_smooth);
  for (int k = 0; k < nu; ++k) RC(smooth(k == 0));
  RC(ctx_jv32(lc, L.x, L.Ax));
  MgLevel& C = lv[l + 1];
  pnp_ctx* cc = C.sub;
  {
    // the coarse levels of the cycle (the transfers included) in one profile class
    ProfScope ps(c, l == 0 ? PNP_PROF_MG : -1, 0.0);
    k_mg_restrict<<<nblk(cc->n_nodes, 256), 256, 0, s>>>(cc->n_nodes, C.r_ptr, C.r_col, C.r_w, L.b, L.Ax,
                                                         lc->d_faces, lc->bc_table(), cc->d_faces, cc->bc_table(),
                                                         C.b);
    note_launch();
    CK(cudaGetLastError());
    RC(mg_cycle(c, l + 1));
    k_mg_prolong_add<<<g, 256, 0, s>>>(N, C.p_ptr, C.p_col, C.p_w, C.x, lc->d_faces, lc->bc_table(), L.x);
    note_launch();
    CK(cudaGetLastError());
  }
  for (int k = 0; k < nu; ++k) RC(smooth(false));
  return PNP_OK;
}

// z32 = one V-cycle applied to u (FP64 [N][3], any scale: the cycle is linear)
int ctx_mg_apply(pnp_ctx* c, const double* u, float* z32) {
  auto& lv = *c->mg;
  CK(launch_to_f32(c->n3(), u, lv[0].b, c->stream));
  RC(mg_cycle(c, 0));
  CK(cudaMemcpyAsync(z32, lv[0].x, sizeof(float) * c->n3(), cudaMemcpyDeviceToDevice, c->stream));
  return PNP_OK;
}

int ctx_mg_level_count(const pnp_ctx* c) { return c->mg ? (int)c->mg->size() : 0; }
