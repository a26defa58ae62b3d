// solver.cu -- residual / Jv drivers, GMRES(m) with classical Gram-Schmidt (flexible
// GMRES with an inner FP32 GMRES in mixed precision), Newton's method (Sec. 4.1 of
// arXiv 2301.05985) with Eisenstat-Walker forcing for the FP32-Jv inexact mode, and the
// BDF time step (Def. 1) with optional step splitting.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

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

template <typename T>
ElemArgs<T> elem_args(const pnp_ctx* c, const T* U, const T* V, const T* hs, const T* adv, T* out) {
  ElemArgs<T> A;
  A.n_elem = c->n_elem;
  A.conn = c->d_conn;
  A.level = c->d_level;
  A.hang_par = c->d_hpar;
  A.hang_np = c->d_hnp;
  A.U = U;
  A.V = V;
  A.hs = hs;
  A.adv = adv;
  A.out = out;
  A.P = c->phys();
  return A;
}

}  // namespace

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int ctx_prepare_history(pnp_ctx* c) {
  if (c->prm.steady) {
    CK(cudaMemsetAsync(c->hs, 0, sizeof(double) * 2 * c->n_nodes, c->stream));
  } else {
    CK(launch_history(c->n_nodes, c->Uk, c->Ukm1, c->prm.beta1, c->prm.beta2, c->prm.dt, c->hs, c->stream));
  }
  return PNP_OK;
}

template <typename T>
static PatchArgs<T> patch_args(const pnp_ctx* c, const T* U, const T* V, const T* hs, const T* adv, T* out,
                               T* partial) {
  PatchArgs<T> A;
  A.pt = c->pt;
  A.level = c->d_level;
  A.faces = c->d_faces;
  A.bc = c->bc_table();
  A.U = U;
  A.V = V;
  A.hs = hs;
  A.adv = adv;
  A.out = out;
  A.partial = partial;
  A.P = c->phys();
  return A;
}

// hanging rows only (the patch kernels write every other row, Dirichlet rows included)
template <typename T>
static int hanging_rows(pnp_ctx* c, const T* in, T* out) {
  RowArgs R = c->rows();
  R.n_nodes = 0;
  return ctx_check(c, launch_row_fixups<T>(R, in, out, 0, c->stream), "hanging rows");
}

int ctx_residual(pnp_ctx* c, const double* U, double* F) {
  if (c->use_patches) {
    {
      ProfScope ps(c, PNP_PROF_RESIDUAL, 88.0 * c->n_nodes + c->conn_bytes(),
                   element_kernel_flops(c->dim, false) * c->n_elem);
      CK(launch_patch<double>(c->dim, false, patch_args<double>(c, U, nullptr, c->hs, c->adv, F, c->part64),
                              c->stream));
    }
    RC(hanging_rows<double>(c, U, F));
  } else {
    CK(cudaMemsetAsync(F, 0, sizeof(double) * c->n3(), c->stream));
    if (residual_double_float()) {
      // FP32-pipe operations of the double-float formulation
      ProfScope ps(c, PNP_PROF_RESIDUAL, 88.0 * c->n_nodes + c->conn_bytes(),
                   kDfFlopsPerFlop * element_kernel_flops(c->dim, false) * c->n_elem);
      CK(launch_residual_df(c->dim, elem_args<double>(c, U, nullptr, c->hs, c->adv, F), c->stream));
    } else {
      ProfScope ps(c, PNP_PROF_RESIDUAL, 88.0 * c->n_nodes + c->conn_bytes(),
                   element_kernel_flops(c->dim, false) * c->n_elem);
      CK(launch_element<double>(c->dim, false, elem_args<double>(c, U, nullptr, c->hs, c->adv, F), c->stream));
    }
    CK(launch_row_fixups<double>(c->rows(), U, F, 0, c->stream));
  }
  c->res_count++;
  return PNP_OK;
}

int ctx_jv64(pnp_ctx* c, const double* U, const double* V, double* JV) {
  if (c->use_patches) {
    {
      ProfScope ps(c, PNP_PROF_JV64, 112.0 * c->n_nodes + c->conn_bytes(), element_kernel_flops(c->dim, true) * c->n_elem);
      CK(launch_patch<double>(c->dim, true, patch_args<double>(c, U, V, c->hs, c->adv, JV, c->part64), c->stream));
    }
    RC(hanging_rows<double>(c, V, JV));
  } else {
    CK(cudaMemsetAsync(JV, 0, sizeof(double) * c->n3(), c->stream));
    {
      ProfScope ps(c, PNP_PROF_JV64, 112.0 * c->n_nodes + c->conn_bytes(), element_kernel_flops(c->dim, true) * c->n_elem);
      CK(launch_element<double>(c->dim, true, elem_args<double>(c, U, V, c->hs, c->adv, JV), c->stream));
    }
    CK(launch_row_fixups<double>(c->rows(), V, JV, 1, c->stream));
  }
  c->jv_count++;
  return PNP_OK;
}

// the FP32 J V of hexahedral meshes runs the two-lanes-per-element kernel (jv_pair.cu)
static bool use_jv_pair(const pnp_ctx* c) { return c->dim == 3 && !c->use_patches && element_kernel_is_lanes(); }

int ctx_prepare_f32(pnp_ctx* c, const double* U) {
  if (use_jv_pair(c)) {
    double vn = 0.0;
    RC(ctx_norm(c, c->adv, &vn));
    c->adv_zero = vn == 0.0;
  }
  CK(launch_to_f32(c->n3(), U, c->U32, c->stream));
  CK(launch_to_f32(2 * c->n_nodes, c->hs, c->hs32, c->stream));
  CK(launch_to_f32(c->n3(), c->adv, c->adv32, c->stream));
  CK(launch_node_records(c->n_nodes, U, c->hs, c->adv, c->rec32, c->stream));
  return PNP_OK;
}

int ctx_jv32(pnp_ctx* c, const float* V32, float* JV32) {
  if (c->use_patches) {
    {
      ProfScope ps(c, PNP_PROF_JV32, 56.0 * c->n_nodes + c->conn_bytes(), element_kernel_flops(c->dim, true) * c->n_elem);
      CK(launch_patch<float>(c->dim, true, patch_args<float>(c, c->U32, V32, c->hs32, c->adv32, JV32, c->part32),
                             c->stream));
    }
    RC(hanging_rows<float>(c, V32, JV32));
  } else {
    CK(cudaMemsetAsync(JV32, 0, sizeof(float) * c->n3(), c->stream));
    ElemArgs<float> A = elem_args<float>(c, c->U32, V32, c->hs32, c->adv32, JV32);
    A.rec = c->rec32;
    if (use_jv_pair(c)) {
      ProfScope ps(c, PNP_PROF_JV32, 56.0 * c->n_nodes + c->conn_bytes(), jv_pair_flops(!c->adv_zero) * c->n_elem);
      CK(launch_jv_pair(A, !c->adv_zero, c->stream));
    } else {
      ProfScope ps(c, PNP_PROF_JV32, 56.0 * c->n_nodes + c->conn_bytes(), element_kernel_flops(c->dim, true) * c->n_elem);
      CK(launch_element<float>(c->dim, true, A, c->stream));
    }
    CK(launch_row_fixups<float>(c->rows(), V32, JV32, 1, c->stream));
  }
  c->jv_count++;
  return PNP_OK;
}

int ctx_block_diag(pnp_ctx* c, const double* U, double* D) {
  CK(cudaMemsetAsync(D, 0, sizeof(double) * 9 * c->n_nodes, c->stream));
  {
    ProfScope ps(c, PNP_PROF_BLOCKDIAG, 136.0 * c->n_nodes + c->conn_bytes(), block_diag_flops(c->dim) * c->n_elem);
    CK(launch_block_diag_lanes<double>(c->dim, elem_args<double>(c, U, nullptr, c->hs, c->adv, nullptr), D,
                                       c->stream));
  }
  CK(launch_diag_rows<double>(c->rows(), D, c->stream));
  return PNP_OK;
}

// FP32 block diagonal at the FP32 copy of the state (ctx_prepare_f32 first)
int ctx_block_diag32(pnp_ctx* c, float* D) {
  CK(cudaMemsetAsync(D, 0, sizeof(float) * 9 * c->n_nodes, c->stream));
  {
    ProfScope ps(c, PNP_PROF_BLOCKDIAG, 68.0 * c->n_nodes + c->conn_bytes(), block_diag_flops(c->dim) * c->n_elem);
    ElemArgs<float> A = elem_args<float>(c, c->U32, nullptr, c->hs32, c->adv32, nullptr);
    A.rec = c->rec32;
    CK(launch_block_diag_lanes<float>(c->dim, A, D, c->stream));
  }
  CK(launch_diag_rows<float>(c->rows(), D, c->stream));
  return PNP_OK;
}

int ctx_norm(pnp_ctx* c, const double* x, double* out) {
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 8;
  CK(launch_norm2(c->n3(), x, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = c->hpin[0];
  return PNP_OK;
}

int ctx_dot(pnp_ctx* c, const double* x, const double* y, double* out) {
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 10;
  CK(launch_dot(c->n3(), x, y, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = c->hpin[0];
  return PNP_OK;
}

// 3x3 block-Jacobi preconditioner at U, built in the precision of the Jv
static int build_preconditioner(pnp_ctx* c, const double* U, int prec) {
  CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
  if (prec == PNP_F32) {
    RC(ctx_prepare_f32(c, U));
    RC(ctx_block_diag32(c, c->D32));
    CK(launch_block_invert<float>(c->n_nodes, c->D32, c->Dinv, c->dflag, c->stream));
    if (c->prm.gmres_inner > 0) {
      RC(ctx_alloc_inner(c, c->prm.gmres_restart, c->prm.gmres_inner));
      CK(launch_to_f32(9 * c->n_nodes, c->Dinv, c->Dinv32, c->stream));
    }
  } else {
    RC(ctx_block_diag(c, U, c->Dinv));
    CK(launch_block_invert<double>(c->n_nodes, c->Dinv, c->Dinv, c->dflag, c->stream));
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) PNP_FAIL(PNP_ERR_NAN, "block-Jacobi preconditioner: singular or non-finite 3x3 block");
  return PNP_OK;
}

// w = J x  in the requested precision (FP32 path: U32/hs32/adv32 must be prepared)
static int apply_op(pnp_ctx* c, const double* U, const double* x, double* w, int prec) {
  if (prec == PNP_F64) return ctx_jv64(c, U, x, w);
  CK(launch_to_f32(c->n3(), x, c->V32, c->stream));
  RC(ctx_jv32(c, c->V32, c->JV32));
  CK(launch_to_f64(c->n3(), c->JV32, w, c->stream));
  return PNP_OK;
}

// PNP_ERR_DEVICE_FLAG when a wait of the staged J V gave up (its copies never landed)
int ctx_check_staged_waits(pnp_ctx* c) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) PNP_FAIL(PNP_ERR_DEVICE_FLAG, "J V: a staged copy of the stored linearisation did not complete");
  return PNP_OK;
}

// FP32 J V of the inner solve: the direction padded to 16 bytes per node (one load), the
// output accumulated with one vector atomic per node, then packed to [N][3] with the
// Dirichlet and hanging rows of J V.  Lane-group kernel only.
// With from_state, the state's Gauss-point quantities come from the linearisation stored
// by launch_lane_state for the current Krylov solve.
static int ctx_jv32_pad(pnp_ctx* c, const float4* V4, float* out, bool from_state) {
  // a memset: clearing the accumulator inside the pack, right after the vector atomics
  // that filled it, measured several times slower on GB300
  CK(cudaMemsetAsync(c->JV4, 0, sizeof(float4) * c->n_nodes, c->stream));
  {
    ElemArgs<float> A = elem_args<float>(c, c->U32, nullptr, c->hs32, c->adv32, nullptr);
    A.rec = c->rec32;
    A.V4 = V4;
    A.out4 = c->JV4;
    if (from_state) {
      // direction in, result out (12 B per node each), the stored state (64 B per lane)
      ProfScope ps(c, PNP_PROF_JV32,
                   24.0 * c->n_nodes + 16.0 * c->lin_rows * (double)(c->n_elem << c->dim) + c->conn_bytes(),
                   jv_from_state_flops(c->dim) * c->n_elem);
      CK(launch_jv_from_state(c->dim, A, c->qp32, c->lin_rows, c->dflag + 1, c->wait_polls, c->stream));
    } else if (use_jv_pair(c)) {
      ProfScope ps(c, PNP_PROF_JV32, 56.0 * c->n_nodes + c->conn_bytes(), jv_pair_flops(!c->adv_zero) * c->n_elem);
      CK(launch_jv_pair(A, !c->adv_zero, c->stream));
    } else {
      ProfScope ps(c, PNP_PROF_JV32, 56.0 * c->n_nodes + c->conn_bytes(),
                   element_kernel_flops(c->dim, true) * c->n_elem);
      CK(launch_element_lanes<float>(c->dim, true, A, c->stream));
    }
  }
  CK(launch_pack_jv4(c->rows(), V4, c->JV4, out, c->stream));
  c->jv_count++;
  return PNP_OK;
}

// Gauss-point linearisation of the FP32 J V at the prepared FP32 state (ctx_prepare_f32)
int ctx_linearize32(pnp_ctx* c) {
  if (!c->qp32) {
    const cudaError_t e = cudaMalloc((void**)&c->qp32, sizeof(float4) * 4 * ((size_t)c->n_elem << c->dim));
    if (e != cudaSuccess) {
      c->qp32 = nullptr;
      PNP_FAIL(e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA,
               "stored linearisation: allocation failed: %s", cudaGetErrorString(e));
    }
  }
  // a new linearisation clears the give-up flag of the staged J V's waits
  CK(cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), c->stream));
  // a zero advection field (pure PNP) leaves v out of the stored state: three rows
  double vn = 0.0;
  RC(ctx_norm(c, c->adv, &vn));
  c->lin_rows = vn == 0.0 ? 3 : 4;
  ElemArgs<float> A = elem_args<float>(c, c->U32, nullptr, c->hs32, c->adv32, nullptr);
  A.rec = c->rec32;
  ProfScope ps(c, PNP_PROF_PRECOND,
               32.0 * c->n_nodes + 16.0 * c->lin_rows * (double)(c->n_elem << c->dim) + c->conn_bytes());
  CK(launch_lane_state(c->dim, A, c->qp32, c->lin_rows, c->stream));
  c->lin_user = false;
  return PNP_OK;
}

// JV = J V (FP32 [n][3]) from the stored linearisation
int ctx_jv32_linearized(pnp_ctx* c, const float* V, float* JV) {
  CK(launch_pad4(c->n_nodes, V, c->V4, c->stream));
  return ctx_jv32_pad(c, c->V4, JV, true);
}

// z = P(u): d steps of right-preconditioned FP32 GMRES on (J M^-1) t = u from t = 0, then
// z = M^-1 t (M: the block diagonal).  A fixed number of steps with the Hessenberg
// bookkeeping on the device: no host round trip.  P is homogeneous, P(a u) = a P(u).
// d steps of the inner solve on the basis row Q_0 already written: normalisation,
// Arnoldi with the device-side bookkeeping, and t = sum_i y_i q_i into c->JV32.  Every
// launch depends only on the context's buffers, sizes and parameters (no host round
// trip), so the sequence can be captured as a graph.
static int inner_gmres32_body(pnp_ctx* c, bool from_state) {
  const int d = c->prm.gmres_inner;
  const int64_t n = c->n3(), N = c->n_nodes, ldq = c->ldq;
  cudaStream_t s = c->stream;
  float* Q = c->Qin;  // rows of ldq floats, the entries past n stay zero
  double* sc = c->isc;                           // rotated Hessenberg, rotations, g, count
  double* sv = sc + inner_scalar_doubles(d);     // [d+1] norms s_i of the basis vectors
  double* dinv = sv + (d + 2);                   // [d+1] 1 / s_i^2
  double* dd = dinv + (d + 2);                   // [d+1] projections
  double* coef = dd + (d + 2);                   // [d] combination coefficients
  float* inv_s = c->iinv;
  {
    ProfScope ps(c, PNP_PROF_INNER, 4.0 * n, 2.0 * n);
    CK(launch_multi_axpy_norm_f32(ldq, 0, Q, ldq, dd, dinv, Q, c->part, s));
  }
  CK(launch_inner_start(d, c->part, sv, dinv, inv_s, sc, s));
  const bool pad = !c->use_patches && element_kernel_is_lanes();
  for (int j = 0; j < d; ++j) {
    float* w = Q + (size_t)(j + 1) * ldq;
    if (pad) {
      {
        ProfScope ps(c, PNP_PROF_PRECOND, 60.0 * N, 18.0 * N);
        CK(launch_block_apply32_pad(N, c->Dinv32, Q + (size_t)j * ldq, inv_s + j, c->V4, s));
      }
      RC(ctx_jv32_pad(c, c->V4, w, from_state));
    } else {
      {
        ProfScope ps(c, PNP_PROF_PRECOND, 60.0 * N, 18.0 * N);
        CK(launch_block_apply32(N, c->Dinv32, Q + (size_t)j * ldq, inv_s + j, c->V32, s));
      }
      RC(ctx_jv32(c, c->V32, w));
    }
    {
      const double nj = (double)n * (j + 1);
      ProfScope ps(c, PNP_PROF_INNER, 4.0 * (nj + n) + 4.0 * (nj + 2.0 * n), 4.0 * nj + 2.0 * n);
      CK(launch_multi_dot_f32(ldq, j + 1, Q, ldq, w, c->part, dd, s));
      CK(launch_multi_axpy_norm_f32(ldq, j + 1, Q, ldq, dd, dinv, w, c->part, s));
    }
    CK(launch_inner_col(j, d, dd, c->part, sv, dinv, inv_s, sc, s));
  }
  CK(launch_inner_lsq(d, sv, sc, coef, s));
  CK(launch_combine_f32(n, d, Q, ldq, coef, c->JV32, s));
  return PNP_OK;
}

// what the captured inner solve depends on: sizes, buffers, parameters, boundary table
static std::vector<unsigned char> inner_graph_key(const pnp_ctx* c, bool from_state) {
  struct Key {
    int d, dim, from_state, pad, use_patches, steady, lin_rows, adv_zero;
    int64_t n_nodes, n_elem, ldq;
    const void* bufs[14];
    double phys[4];
    double bc_val[6][3];
    uint8_t dir_faces[4];
  } k;
  std::memset(&k, 0, sizeof(k));
  k.d = c->prm.gmres_inner;
  k.dim = c->dim;
  k.from_state = from_state;
  k.pad = element_kernel_is_lanes();
  k.use_patches = c->use_patches;
  k.lin_rows = c->lin_rows;
  k.adv_zero = c->adv_zero;
  k.n_nodes = c->n_nodes;
  k.n_elem = c->n_elem;
  k.ldq = c->ldq;
  const void* b[14] = {c->Qin, c->isc, c->iinv, c->Dinv32, c->V4, c->JV4, c->qp32, c->part, c->JV32,
                       c->V32, c->U32, c->hs32, c->adv32, c->rec32};
  std::memcpy(k.bufs, b, sizeof(b));
  const PhysParams P = c->phys();
  k.phys[0] = P.eps2x2;
  k.phys[1] = P.kappa;
  k.phys[2] = P.tau_t;
  k.phys[3] = P.C_I;
  k.steady = P.steady;
  const BcTable bc = c->bc_table();
  for (int f = 0; f < 3; ++f) k.dir_faces[f] = bc.dir_faces[f];
  for (int face = 0; face < 6; ++face)
    for (int f = 0; f < 3; ++f) k.bc_val[face][f] = bc.val[face][f];
  std::vector<unsigned char> v(sizeof(k));
  std::memcpy(v.data(), &k, sizeof(k));
  return v;
}

// replays of the captured inner solve while profiling is off (the per-kernel event pairs
// of the profile need eager launches); PNP_INNER_GRAPH=0 turns the graph off
static bool inner_graph_enabled(const pnp_ctx* c) {
  static const bool env_off = [] {
    const char* e = getenv("PNP_INNER_GRAPH");
    return e && std::strcmp(e, "0") == 0;
  }();
  return !env_off && !c->prof_on && c->inner_eager_done && !c->inner_graph_off;
}

// true when the graph was captured; on false the caller runs the solve eagerly (a capture
// that the runtime refuses turns the graph off for the context, with no error latched)
static bool inner_graph_capture(pnp_ctx* c, bool from_state) {
  if (c->inner_exec) {
    cudaGraphExecDestroy(c->inner_exec);
    c->inner_exec = nullptr;
  }
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    c->inner_graph_off = true;
    return false;
  }
  cudaStream_t saved = c->stream;
  const cudaError_t latched0 = c->latched;
  c->stream = c->cap_stream;
  const int64_t l0 = launch_count();
  const int jv0 = c->jv_count;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? inner_gmres32_body(c, from_state) : PNP_OK;
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) {
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  c->stream = saved;
  if (rc == PNP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->inner_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  // the capture counted its launches and J V calls once; replays add them per run
  c->inner_graph_launches = launch_count() - l0;
  note_launches(-c->inner_graph_launches);
  c->inner_graph_jv = c->jv_count - jv0;
  c->jv_count = jv0;
  if (rc != PNP_OK || e != cudaSuccess) {
    cudaGetLastError();
    if (c->inner_exec) cudaGraphExecDestroy(c->inner_exec);
    c->inner_exec = nullptr;
    c->inner_graph_off = true;
    c->latched = latched0;  // a refused capture is not a device error
    return false;
  }
  c->inner_key = inner_graph_key(c, from_state);
  note_capture();
  return true;
}

// z = P(u): d steps of right-preconditioned FP32 GMRES on (J M^-1) t = u from t = 0, then
// z = M^-1 t (M: the block diagonal).  A fixed number of steps with the Hessenberg
// bookkeeping on the device: no host round trip.  P is homogeneous, P(a u) = a P(u).
static int inner_gmres32(pnp_ctx* c, const double* u, float* z32, bool from_state) {
  const int64_t n = c->n3(), N = c->n_nodes;
  cudaStream_t s = c->stream;
  CK(launch_to_f32(n, u, c->Qin, s));
  bool replay = inner_graph_enabled(c);
  if (replay && (!c->inner_exec || c->inner_key != inner_graph_key(c, from_state)))
    replay = inner_graph_capture(c, from_state);
  if (replay) {
    CK(cudaGraphLaunch(c->inner_exec, s));
    note_launches(c->inner_graph_launches);
    c->jv_count += c->inner_graph_jv;
  } else {
    RC(inner_gmres32_body(c, from_state));
    c->inner_eager_done = true;
  }
  ProfScope ps(c, PNP_PROF_PRECOND, 60.0 * N, 18.0 * N);
  CK(launch_block_apply32(N, c->Dinv32, c->JV32, nullptr, z32, s));
  return PNP_OK;
}

// z = P(u) in FP64: d steps of right-preconditioned FP64 GMRES on (J M^-1) t = u from
// t = 0, then z = M^-1 t.  The FP64 counterpart of inner_gmres32 (the same algorithm with
// FP64 J V, basis and dot products), driven from the host: one round trip per step for
// the projections, the Hessenberg system and its Givens rotations on the host.
static int inner_gmres64(pnp_ctx* c, const double* U, const double* u, double* z) {
  const int d = c->prm.gmres_inner;
  const int64_t n = c->n3(), N = c->n_nodes;
  cudaStream_t s = c->stream;
  double* Q = c->Qin64;            // unnormalised basis u_i (v_i = u_i / s_i)
  double* dd = c->isc64;           // [d+2] projections of one pass
  double* dinv = dd + (d + 2);     // [d+2] 1 / s_i^2
  double* coef = dinv + (d + 2);   // [d+2] combination coefficients
  double* dnrm = coef + (d + 2);   // [2]  w . w after the pass
  CK(cudaMemcpyAsync(Q, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  double beta;
  RC(ctx_norm(c, Q, &beta));
  if (!std::isfinite(beta)) PNP_FAIL(PNP_ERR_NAN, "inner gmres: vector norm is not finite");
  if (beta == 0.0) {
    CK(cudaMemsetAsync(z, 0, sizeof(double) * n, s));
    return PNP_OK;
  }
  std::vector<double> H((size_t)(d + 1) * d, 0.0), cs(d), sn(d), g(d + 1, 0.0), y(d), sv(d + 1), hp(d + 2), up(d + 2);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * d + j]; };
  sv[0] = beta;
  g[0] = beta;
  up[0] = 1.0 / (beta * beta);
  CK(cudaMemcpyAsync(dinv, up.data(), sizeof(double), cudaMemcpyHostToDevice, s));
  int k = 0;
  for (int j = 0; j < d; ++j) {
    double* w = Q + (size_t)(j + 1) * n;
    {
      ProfScope ps(c, PNP_PROF_PRECOND, 120.0 * N, 18.0 * N);
      CK(launch_block_apply(N, c->Dinv, Q + (size_t)j * n, 1.0 / sv[j], c->zin64, nullptr, s));
    }
    RC(ctx_jv64(c, U, c->zin64, w));
    const double nj = (double)n * (j + 1);
    {
      ProfScope ps(c, PNP_PROF_ORTHO, 8.0 * (nj + n), 2.0 * nj);
      CK(launch_multi_dot_ext(n, j + 1, false, Q, n, w, c->part, dd, s));
    }
    {
      ProfScope ps(c, PNP_PROF_ORTHO_UPDATE, 8.0 * (nj + 2.0 * n), 2.0 * (nj + n));
      CK(launch_multi_axpy_norm(n, j + 1, Q, n, dd, dinv, w, c->part, dnrm, s));
    }
    CK(cudaMemcpyAsync(hp.data(), dd, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp.data() + (d + 1), dnrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i <= j; ++i) Hij(i, j) = hp[i] / sv[i];
    const double nrm = std::sqrt(hp[d + 1]);
    if (!std::isfinite(nrm)) PNP_FAIL(PNP_ERR_NAN, "inner gmres: Krylov vector norm is not finite");
    sv[j + 1] = nrm;
    Hij(j + 1, j) = nrm;
    if (nrm > 0) {
      up[j + 1] = 1.0 / (nrm * nrm);
      CK(cudaMemcpyAsync(dinv + j + 1, up.data() + j + 1, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
      Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
      Hij(i, j) = t;
    }
    const double rr = std::hypot(Hij(j, j), Hij(j + 1, j));
    if (rr == 0.0) PNP_FAIL(PNP_ERR_NAN, "inner gmres: singular Hessenberg matrix");
    cs[j] = Hij(j, j) / rr;
    sn[j] = Hij(j + 1, j) / rr;
    Hij(j, j) = rr;
    Hij(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    k = j + 1;
    if (nrm <= 1e-300 * beta) break;
  }
  // t = sum_i y_i u_i / s_i with H y = g, then z = M^-1 t
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
    y[i] = t / Hij(i, i);
  }
  for (int i = 0; i < k; ++i) up[i] = -y[i] / sv[i];
  CK(cudaMemcpyAsync(coef, up.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(c->zin64, 0, sizeof(double) * n, s));
  CK(launch_multi_axpy(n, k, Q, n, coef, c->zin64, nullptr, s));
  ProfScope ps(c, PNP_PROF_PRECOND, 120.0 * N, 18.0 * N);
  CK(launch_block_apply(N, c->Dinv, c->zin64, 1.0, z, nullptr, s));
  CK(cudaStreamSynchronize(s));  // the host vectors above go out of scope
  return PNP_OK;
}

// Right-preconditioned GMRES(m), or flexible GMRES(m) when an inner FP32 GMRES(d) is the
// preconditioner (PNP_F32 with gmres_inner > 0).  The Krylov vectors are stored
// unnormalised (v_i = u_i / s_i, s_i kept on the host) so no normalisation pass is
// needed; each iteration does one classical Gram-Schmidt pass (multi-dot, then
// multi-axpy fused with the new norm), two with gmres_cgs2.  Dots, basis and the
// Hessenberg system are FP64.
constexpr int kMgCheck = 20;  // iterations after which a multigrid cycle must have halved the residual

int ctx_gmres(pnp_ctx* c, const double* U, const double* b, double* x, double rtol, int prec, int max_it, int* its_out,
              double* rel_out, bool have_precond) {
  const int m = c->prm.gmres_restart;
  RC(ctx_alloc_krylov(c, m));
  const int64_t n = c->n3();
  cudaStream_t s = c->stream;
  if (!have_precond) RC(build_preconditioner(c, U, prec));
  if (prec == PNP_F32) RC(ctx_prepare_f32(c, U));
  // multigrid preconditioner (FP32 V-cycle) of a flexible outer solve; a solve in which
  // it stagnates continues with the inner FP32 GMRES (block Jacobi) preconditioner
  const bool use_mg = prec == PNP_F32 && c->prm.mg_levels > 0;
  bool mg_on = use_mg;
  const int inner_saved = c->prm.gmres_inner;
  const int inner_fb = inner_saved > 0 ? inner_saved : 24;
  if (use_mg) {
    RC(ctx_mg_setup(c, c->prm.mg_levels));
    RC(ctx_mg_prepare(c, U));
  }
  const bool flex = prec == PNP_F32 && (c->prm.gmres_inner > 0 || use_mg);
  if (flex) RC(ctx_alloc_inner(c, m, std::max(inner_fb, c->prm.gmres_inner)));
  if (use_mg && inner_saved == 0) CK(launch_to_f32(9 * c->n_nodes, c->Dinv, c->Dinv32, s));
  struct InnerRestore {  // the fallback switches gmres_inner for the rest of this solve
    pnp_ctx* c;
    int v;
    ~InnerRestore() { c->prm.gmres_inner = v; }
  } inner_restore{c, inner_saved};
  // the same flexible scheme entirely in FP64 (inner FP64 GMRES, FP64 J V)
  const bool flex64 = prec == PNP_F64 && c->prm.gmres_inner > 0;
  if (flex64) RC(ctx_alloc_inner64(c, m, c->prm.gmres_inner));
  // the inner J V reads the state's Gauss-point quantities stored once for this solve
  const bool from_state = flex && !use_mg && !c->use_patches && element_kernel_is_lanes();
  c->lin_user = false;  // a solve replaces any linearisation stored by pnp_linearize
  if (from_state) RC(ctx_linearize32(c));
  double* V = c->basis;
  double* dd = c->dsc;                    // [m+2] dot products of one pass
  double* dinv = c->dsc + (m + 2);        // [m+2] 1 / s_i^2
  double* dnrm = c->dsc + 2 * (m + 2);    // [1]  w . w after a pass
  double* dcoef = c->dsc + 2 * (m + 2) + 2;  // [m+1] solution-update coefficients
  double* dd2 = c->dsc + 3 * (m + 2) + 2;    // [m+2] projections of the second pass
  double* hp = c->hpin;                     // [0, m+2): D2H scratch
  double* hup = c->hpin + (m + 2);          // [m+2]: H2D slots for 1/s_i^2
  double* hco = c->hpin + 2 * (m + 2) + 2;  // [m+1]: H2D slots for the update coefficients
  double* hp2 = c->hpin + 3 * (m + 2) + 2;  // [m+2]: D2H of the second pass
  *its_out = 0;
  double bn;
  RC(ctx_norm(c, b, &bn));
  if (!std::isfinite(bn)) PNP_FAIL(PNP_ERR_NAN, "gmres: right-hand side is not finite");
  if (bn == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *rel_out = 0;
    return PNP_OK;
  }
  const double tol = rtol * bn;
  // u_0 = b - J x
  RC(apply_op(c, U, x, c->w, prec));
  CK(launch_axpbyz(n, 1.0, b, -1.0, c->w, V, s));
  double beta;
  RC(ctx_norm(c, V, &beta));
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), sv(m + 1), h(m + 1);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int total = 0;
  double beta_cycle = beta;  // true residual at the start of the current cycle
  while (true) {
    if (!std::isfinite(beta)) PNP_FAIL(PNP_ERR_NAN, "gmres: residual norm is not finite");
    if (beta <= tol) break;
    if (total >= max_it) {
      *its_out = total;
      *rel_out = beta / bn;
      PNP_FAIL(PNP_ERR_KRYLOV_MAXIT, "gmres: %d iterations, relative residual %.3e > %.3e", total, beta / bn, rtol);
    }
    sv[0] = beta;
    CK(cudaStreamSynchronize(s));  // the pinned upload slots are free again
    hup[0] = 1.0 / (beta * beta);
    CK(cudaMemcpyAsync(dinv, hup, sizeof(double), cudaMemcpyHostToDevice, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    double res = beta;
    bool breakdown = false;
    bool mg_slow = false;  // the multigrid cycle is not converging: give up on it early
    for (int j = 0; j < m && total < max_it; ++j) {
      const double* uj = V + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      // z = M^-1 (u_j / s_j) ; w = J z   (flexible: z_j = P(u_j) / s_j kept in Zb)
      if (flex) {
        float* zj = c->Zb + (size_t)j * n;
        if (mg_on) RC(ctx_mg_apply(c, uj, zj));
        else RC(inner_gmres32(c, uj, zj, from_state));
        // the outer J V applies the same linearisation as the inner one
        if (from_state) RC(ctx_jv32_linearized(c, zj, c->JV32));
        else RC(ctx_jv32(c, zj, c->JV32));
        ProfScope ps(c, PNP_PROF_PRECOND, 20.0 * (double)n);
        CK(launch_to_f64_scaled(n, c->JV32, 1.0 / sv[j], w, s));
      } else if (flex64) {
        // z_j = P(u_j) (unscaled, kept in Z64), w = J z_j / s_j
        double* zj = c->Z64 + (size_t)j * n;
        RC(inner_gmres64(c, U, uj, zj));
        RC(ctx_jv64(c, U, zj, c->w));
        CK(launch_axpbyz(n, 1.0 / sv[j], c->w, 0.0, c->w, w, s));
      } else if (prec == PNP_F64) {
        {
          ProfScope ps(c, PNP_PROF_PRECOND, 120.0 * c->n_nodes, 18.0 * c->n_nodes);
          CK(launch_block_apply(c->n_nodes, c->Dinv, uj, 1.0 / sv[j], c->z, nullptr, s));
        }
        RC(ctx_jv64(c, U, c->z, w));
      } else {
        {
          ProfScope ps(c, PNP_PROF_PRECOND, 108.0 * c->n_nodes, 18.0 * c->n_nodes);
          CK(launch_block_apply(c->n_nodes, c->Dinv, uj, 1.0 / sv[j], nullptr, c->V32, s));
        }
        RC(ctx_jv32(c, c->V32, c->JV32));
        ProfScope ps(c, PNP_PROF_PRECOND, 36.0 * c->n_nodes);
        CK(launch_to_f64(n, c->JV32, w, s));
      }
      double w1sq;
      {
        // classical Gram-Schmidt (a second pass when gmres_cgs2), one host round trip
        // per iteration; the projections of the two passes go to separate device slots
        const bool two = c->prm.gmres_cgs2 != 0;
        const double nj = (double)n * (j + 1);
        for (int pass = 0; pass < (two ? 2 : 1); ++pass) {
          double* dp = pass == 0 ? dd : dd2;
          {
            ProfScope ps(c, PNP_PROF_ORTHO, 8.0 * (nj + n), 2.0 * nj);
            CK(launch_multi_dot_ext(n, j + 1, false, V, n, w, c->part, dp, s));
          }
          ProfScope ps(c, PNP_PROF_ORTHO_UPDATE, 8.0 * (nj + 2.0 * n), 2.0 * (nj + n));
          CK(launch_multi_axpy_norm(n, j + 1, V, n, dp, dinv, w, c->part, dnrm, s));
        }
        if (two) CK(cudaMemcpyAsync(hp2, dd2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hp, dd, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hp + (m + 1), dnrm, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!two)
          for (int i = 0; i <= j; ++i) hp2[i] = 0.0;
      }
      for (int i = 0; i <= j; ++i) h[i] = (hp[i] + hp2[i]) / sv[i];
      w1sq = hp[m + 1];
      const double nrm = std::sqrt(w1sq);
      if (!std::isfinite(nrm)) PNP_FAIL(PNP_ERR_NAN, "gmres: Krylov vector norm is not finite");
      sv[j + 1] = nrm;
      if (nrm > 0) {
        hup[j + 1] = 1.0 / w1sq;
        CK(cudaMemcpyAsync(dinv + j + 1, hup + j + 1, sizeof(double), cudaMemcpyHostToDevice, s));
      }
      for (int i = 0; i <= j; ++i) Hij(i, j) = h[i];
      Hij(j + 1, j) = nrm;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double rr = std::hypot(Hij(j, j), Hij(j + 1, j));
      if (rr == 0.0) PNP_FAIL(PNP_ERR_NAN, "gmres: singular Hessenberg matrix");
      cs[j] = Hij(j, j) / rr;
      sn[j] = Hij(j + 1, j) / rr;
      Hij(j, j) = rr;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      res = std::fabs(g[j + 1]);
      ++total;
      k = j + 1;
      if (nrm <= 1e-300 * bn) breakdown = true;
      if (res <= tol || breakdown) break;
      // a multigrid-preconditioned cycle that has not halved the residual in 20
      // iterations ends here (its partial solution is kept) and the solve goes on with
      // the inner GMRES preconditioner
      if (mg_on && j + 1 == kMgCheck && res > 0.5 * beta) {
        mg_slow = true;
        break;
      }
    }
    // y = H^-1 g ; x += M^-1 (sum_i y_i u_i / s_i)
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
      y[i] = t / Hij(i, i);
    }
    if (flex) {
      // x += sum_i y_i z_i with z_i = P(u_i) / s_i
      for (int i = 0; i < k; ++i) hco[i] = y[i] / sv[i];
      CK(cudaMemcpyAsync(dcoef, hco, sizeof(double) * k, cudaMemcpyHostToDevice, s));
      CK(launch_combine_f32_add_f64(n, k, c->Zb, n, dcoef, x, s));
    } else if (flex64) {
      for (int i = 0; i < k; ++i) hco[i] = -y[i] / sv[i];
      CK(cudaMemcpyAsync(dcoef, hco, sizeof(double) * k, cudaMemcpyHostToDevice, s));
      CK(launch_multi_axpy(n, k, c->Z64, n, dcoef, x, nullptr, s));
    } else {
      for (int i = 0; i < k; ++i) hco[i] = -y[i] / sv[i];
      CK(cudaMemcpyAsync(dcoef, hco, sizeof(double) * k, cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(c->w, 0, sizeof(double) * n, s));
      CK(launch_multi_axpy(n, k, V, n, dcoef, c->w, nullptr, s));
      CK(launch_block_apply(c->n_nodes, c->Dinv, c->w, 1.0, c->z, nullptr, s));
      CK(launch_axpby(n, 1.0, c->z, 1.0, x, s));
    }
    // true residual (restart vector); when the Arnoldi estimate claims convergence it is
    // accepted only if the true residual agrees (the estimate drifts when the Krylov
    // basis loses orthogonality)
    RC(apply_op(c, U, x, c->w, prec));
    CK(launch_axpbyz(n, 1.0, b, -1.0, c->w, V, s));
    RC(ctx_norm(c, V, &beta));
    if ((res <= tol || breakdown) && beta <= 2.0 * tol) break;
    if (c->prm.monitor >= 2)
      fprintf(stderr, "[pnp gmres] its %5d  estimate %.3e  true %.3e (relative)\n", total, res / bn, beta / bn);
    // a whole cycle that cut the true residual by less than 5%: the operator's rounding
    // floor (FP32 J V) or a stalled flexible preconditioner; stop with the iterate
    if (std::isfinite(beta) && (beta > 0.95 * beta_cycle || mg_slow) && mg_on) {
      mg_on = false;
      c->prm.gmres_inner = inner_fb;
      c->mg_fallbacks++;
      if (c->prm.monitor >= 1)
        fprintf(stderr, "[pnp gmres] multigrid stagnated at relative residual %.3e: inner GMRES(%d)\n", beta / bn,
                inner_fb);
      beta_cycle = beta;
      continue;
    }
    if (std::isfinite(beta) && beta > 0.95 * beta_cycle) {
      CK(cudaStreamSynchronize(s));
      if (from_state) RC(ctx_check_staged_waits(c));
      *its_out = total;
      *rel_out = beta / bn;
      PNP_FAIL(PNP_ERR_KRYLOV_MAXIT, "gmres: stagnated after %d iterations at relative residual %.3e > %.3e", total,
               beta / bn, rtol);
    }
    beta_cycle = beta;
  }
  CK(cudaStreamSynchronize(s));
  *its_out = total;
  *rel_out = beta / bn;
  if (from_state) RC(ctx_check_staged_waits(c));
  return PNP_OK;
}

int ctx_newton(pnp_ctx* c, pnp_solve_stats* st, const double* ref_state) {
  const double t0 = now_ms();
  std::memset(st, 0, sizeof(*st));
  const pnp_params& p = c->prm;
  const int64_t n = c->n3();
  cudaStream_t s = c->stream;
  c->jv_count = 0;
  c->res_count = 0;
  c->mg_fallbacks = 0;
  RC(ctx_prepare_history(c));
  CK(launch_make_consistent(c->rows(), c->U, s));
  RC(ctx_residual(c, c->U, c->F));
  double f0;
  RC(ctx_norm(c, c->F, &f0));
  st->res0 = f0;
  if (!std::isfinite(f0)) {
    st->status = PNP_ERR_NAN;
    PNP_FAIL(PNP_ERR_NAN, "newton: initial residual is not finite");
  }
  // the relative tolerance refers to ||F(ref_state)|| when given (the time step's
  // previous-step state), else to the start's own residual
  double f_ref = f0;
  c->start_fell_back = false;
  if (ref_state) {
    CK(cudaMemcpyAsync(c->Ut, ref_state, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(launch_make_consistent(c->rows(), c->Ut, s));
    RC(ctx_residual(c, c->Ut, c->Ft));
    RC(ctx_norm(c, c->Ft, &f_ref));
    // a start whose residual exceeds the previous state's (an extrapolation that overshoots
    // after a fast transient) is replaced by the previous state
    if (std::isfinite(f_ref) && !(f0 <= f_ref)) {
      std::swap(c->U, c->Ut);
      std::swap(c->F, c->Ft);
      f0 = f_ref;
      st->res0 = f0;
      c->start_fell_back = true;
    }
  }
  st->res_ref = f_ref;
  const double target = std::max(p.newton_rtol * f_ref, p.newton_atol);
  double f = f0, f_prev = f0, eta_prev = p.ew_eta_max;
  int it = 0, kry = 0;
  int rc = PNP_OK;
  while (f > target) {
    if (it >= p.newton_max_it) {
      rc = PNP_ERR_NEWTON_DIVERGED;
      pnp_set_error("newton: %d iterations, ||F|| = %.3e > target %.3e", it, f, target);
      break;
    }
    RC(build_preconditioner(c, c->U, p.precision));
    CK(launch_axpby(n, -1.0, c->F, 0.0, c->rhs, s));
    double eta;
    if (p.precision == PNP_F64 && !p.newton_ew_f64) {
      eta = p.gmres_rtol;
    } else {
      // Eisenstat-Walker, choice 2 (gamma = 0.9, alpha = 2) with safeguards
      if (it == 0) {
        eta = 0.5;
      } else {
        eta = 0.9 * (f / f_prev) * (f / f_prev);
        const double sg = 0.9 * eta_prev * eta_prev;
        if (sg > 0.1) eta = std::max(eta, sg);
      }
      eta = std::max(eta, 0.5 * target / f);
      eta = std::min(std::max(eta, p.ew_eta_min), p.ew_eta_max);
    }
    eta_prev = eta;
    // one attempt = linear solve in precision `prec` + backtracking line search on ||F||;
    // returns 0 accepted, 1 no decrease, <0 hard error (-status)
    double alpha = 1.0, ft = 0.0;
    int its = 0, lrc = PNP_OK;
    double rel = 0;
    auto attempt = [&](int prec, double tol) -> int {
      CK(cudaMemsetAsync(c->dU, 0, sizeof(double) * n, s));
      its = 0;
      lrc = ctx_gmres(c, c->U, c->rhs, c->dU, tol, prec, p.gmres_max_it, &its, &rel, true);
      kry += its;
      if (lrc != PNP_OK && lrc != PNP_ERR_KRYLOV_MAXIT) return -lrc;
      alpha = 1.0;
      while (true) {
        CK(launch_axpbyz(n, 1.0, c->U, alpha, c->dU, c->Ut, s));
        RC(ctx_residual(c, c->Ut, c->Ft));
        RC(ctx_norm(c, c->Ft, &ft));
        if (!p.line_search) return std::isfinite(ft) ? 0 : 1;
        if (std::isfinite(ft) && ft <= (1.0 - 1e-4 * alpha) * f) return 0;
        alpha *= 0.5;
        if (alpha < 1.0 / 1024) return 1;
      }
    };
    int prec_used = p.precision;
    int ar = attempt(p.precision, eta);
    if (ar > 0 && p.precision == PNP_F32 && p.f64_fallback) {
      if (p.monitor)
        fprintf(stderr, "[pnp newton %2d] FP32 step rejected (gmres its %d rel %.2e alpha %.3g ||F_t|| %.3e)\n",
                it, its, rel, alpha, ft);
      prec_used = PNP_F64;
      st->f64_fallbacks++;
      ar = attempt(PNP_F64, std::min(eta, p.gmres_rtol > 0 ? std::max(p.gmres_rtol, 1e-12) : 1e-8));
    }
    if (p.monitor)
      fprintf(stderr, "[pnp newton %2d] ||F|| %.6e -> %.6e  eta %.2e  %s gmres its %4d rel %.2e  alpha %.4g\n", it,
              f, ft, eta, prec_used == PNP_F32 ? "f32" : "f64", its, rel, alpha);
    if (ar < 0) {
      rc = -ar;
      break;
    }
    if (ar > 0) {
      rc = std::isfinite(ft) ? PNP_ERR_NEWTON_DIVERGED : PNP_ERR_NAN;
      pnp_set_error("newton: %s at iteration %d (||F|| = %.3e)",
                    std::isfinite(ft) ? "line search failed" : "residual became non-finite", it + 1, f);
      break;
    }
    std::swap(c->U, c->Ut);
    std::swap(c->F, c->Ft);
    f_prev = f;
    f = ft;
    ++it;
  }
  CK(cudaStreamSynchronize(s));
  st->status = rc;
  st->newton_its = it;
  st->krylov_its = kry;
  st->res_final = f;
  st->jv_evals = c->jv_count;
  st->residual_evals = c->res_count;
  st->mg_fallbacks = c->mg_fallbacks;
  st->wall_ms = now_ms() - t0;
  return rc;
}

int pnp_learned_start(pnp_ctx* c, pnp_solve_stats* st);  // mlp.cu

// One Newton solve over `dt` (BDF2 or BDF1) from the start already in U, to a tolerance
// relative to ||F(ref)|| (NULL: to the start's own residual); on success the history
// shifts (U^{k-1} <- U^k <- U).  A failed solve with split depth left is redone as two
// BDF1 half steps, each started from (and measured against) the previous state.
// BDF2 (3/2, -2, 1/2) or BDF1 (1, -1, 0) coefficients of the time derivative (Def. 1)
static void set_bdf(pnp_params& p, bool bdf2) {
  if (bdf2) {
    p.beta0 = 1.5; p.beta1 = -2.0; p.beta2 = 0.5;
  } else {
    p.beta0 = 1.0; p.beta1 = -1.0; p.beta2 = 0.0;
  }
}

static int advance(pnp_ctx* c, double dt, bool bdf2, int depth, const double* ref, pnp_solve_stats* tot) {
  const int64_t n = c->n3();
  cudaStream_t s = c->stream;
  pnp_params& p = c->prm;
  p.dt = dt;
  set_bdf(p, bdf2);
  pnp_solve_stats one;
  std::memset(&one, 0, sizeof(one));
  const int rc = ctx_newton(c, &one, ref);
  if (depth == 0) {
    tot->res0 = one.res0;
    tot->res_ref = one.res_ref;
  }
  tot->newton_its += one.newton_its;
  tot->krylov_its += one.krylov_its;
  tot->f64_fallbacks += one.f64_fallbacks;
  tot->jv_evals = one.jv_evals;
  tot->residual_evals = one.residual_evals;
  tot->mg_fallbacks += one.mg_fallbacks;
  tot->res_final = one.res_final;
  tot->status = rc;
  if (rc == PNP_OK) {
    CK(cudaMemcpyAsync(c->Ukm1, c->Uk, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->Uk, c->U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    tot->substeps++;
    return PNP_OK;
  }
  const bool recoverable = rc == PNP_ERR_NEWTON_DIVERGED || rc == PNP_ERR_KRYLOV_MAXIT || rc == PNP_ERR_NAN;
  if (!recoverable || depth >= p.dt_retries) return rc;
  if (p.monitor) fprintf(stderr, "[pnp step] Newton failed (status %d) at dt %.3e: two half steps\n", rc, dt);
  for (int h = 0; h < 2; ++h) {
    CK(cudaMemcpyAsync(c->U, c->Uk, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    RC(advance(c, 0.5 * dt, false, depth + 1, nullptr, tot));
  }
  return PNP_OK;
}

int ctx_time_step(pnp_ctx* c, pnp_solve_stats* st) {
  const double t0 = now_ms();
  const int64_t n = c->n3();
  cudaStream_t s = c->stream;
  pnp_params& p = c->prm;
  // BDF2 needs U^{k-1} one full step behind U^k
  const bool bdf2 = !(c->step == 0 || p.bdf_order == 1 || c->history_split);
  // advection at t^{k+1}: v~ = 2 v^k - v^{k-1} (Eq. averaging1); in a coupled step the
  // NS block has set v^{k+1}
  if (!c->coupled) CK(launch_axpbyz(n, 2.0, c->vel, -1.0, c->vel_prev, c->adv, s));
  int start = p.start_mode;
  if (c->history_split) start = PNP_START_PREVIOUS;  // extrapolation assumes equal spacing
  if (c->start_given) start = -1;  // a repeated block iteration: U holds the start
  double r_extra = 0, r_learn = 0;
  if (start == PNP_START_LEARNED) {
    // the judge's residuals use this step's BDF formula
    set_bdf(p, bdf2);
    pnp_solve_stats tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    const int lrc = pnp_learned_start(c, &tmp);
    if (lrc == PNP_OK) {
      start = tmp.start_used;
      r_extra = tmp.res_start_extrapolated;
      r_learn = tmp.res_start_learned;
    } else if (lrc == PNP_ERR_STATE) {
      start = PNP_START_EXTRAPOLATE;  // no trained network: plain extrapolation
    } else {
      return lrc;
    }
  }
  if (start == PNP_START_EXTRAPOLATE && c->step == 0) start = PNP_START_PREVIOUS;  // no history yet
  if (start == PNP_START_PREVIOUS) {
    CK(cudaMemcpyAsync(c->U, c->Uk, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else if (start == PNP_START_EXTRAPOLATE) {
    CK(launch_axpbyz(n, 2.0, c->Uk, -1.0, c->Ukm1, c->U, s));
  }  // learned: U already holds the judged start
  const double dt = p.dt;
  pnp_solve_stats tot;
  std::memset(&tot, 0, sizeof(tot));
  // Newton's relative tolerance refers to the residual of the previous-step state U^k
  // (the paper's start), so that every start is held to the same absolute tolerance
  const int rc = advance(c, dt, bdf2, 0, start == PNP_START_PREVIOUS ? nullptr : c->Uk, &tot);
  p.dt = dt;
  if (c->start_fell_back) start = PNP_START_PREVIOUS;
  tot.start_used = start;
  tot.res_start_extrapolated = r_extra;
  tot.res_start_learned = r_learn;
  *st = tot;
  if (rc != PNP_OK) {
    st->wall_ms = now_ms() - t0;
    return rc;
  }
  if (!c->coupled) CK(cudaMemcpyAsync(c->vel_prev, c->vel, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  c->step++;
  c->history_split = tot.substeps > 1;
  st->wall_ms = now_ms() - t0;
  return PNP_OK;
}

// One NS-PNP step by block iteration (Sec. 4.1): the linear NS block first (body force
// from U^k, then from the latest U^{k+1}), then the PNP Newton solve with v^{k+1} as the
// advection; a repeated iteration restores the PNP history and restarts Newton from the
// latest U^{k+1}.
int ctx_coupled_step(pnp_ctx* c, pnp_solve_stats* st, pnp_ns_stats* nst) {
  const double t0 = now_ms();
  std::memset(st, 0, sizeof(*st));
  std::memset(nst, 0, sizeof(*nst));
  RC(ctx_ns_alloc(c));
  pnp_params& p = c->prm;
  const int64_t n = c->n3();
  cudaStream_t s = c->stream;
  const bool bdf2 = !(c->step == 0 || p.bdf_order == 1);
  const int nb = p.ns_blocks;
  const int64_t step0 = c->step;
  const bool split0 = c->history_split;
  double* save = nb > 1 ? ctx_ns_history_save(c) : nullptr;  // [2][3N]: U^k, U^{k-1}
  if (nb > 1) {
    if (!save) PNP_FAIL(PNP_ERR_NOMEM, "coupled step: no memory for the PNP history");
    CK(cudaMemcpyAsync(save, c->Uk, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(save + n, c->Ukm1, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  for (int b = 0; b < nb; ++b) {
    if (b > 0) {
      CK(cudaMemcpyAsync(c->Uk, save, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(c->Ukm1, save + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      c->step = step0;
      c->history_split = split0;
    }
    set_bdf(p, bdf2);
    pnp_ns_stats one;
    int rc = ctx_ns_solve(c, b == 0 ? c->Uk : c->U, &one);
    nst->status = rc;
    nst->refinements += one.refinements;
    nst->inner_its += one.inner_its;
    nst->matvecs32 += one.matvecs32;
    nst->matvecs64 += one.matvecs64;
    nst->singular_blocks |= one.singular_blocks;
    nst->floor_stop |= one.floor_stop;
    nst->mg_fallbacks += one.mg_fallbacks;
    nst->krylov_fallbacks += one.krylov_fallbacks;
    if (b == 0) nst->res0 = one.res0;
    nst->res_final = one.res_final;
    nst->wall_ms += one.wall_ms;
    if (rc != PNP_OK) {
      st->status = rc;  // the step failed in its NS block
      return rc;
    }
    RC(ctx_ns_velocity(c, c->adv));
    pnp_solve_stats ps;
    c->coupled = true;
    c->start_given = b > 0;
    rc = ctx_time_step(c, &ps);
    c->coupled = false;
    c->start_given = false;
    const int start_used = b == 0 ? ps.start_used : st->start_used;
    const double rse = b == 0 ? ps.res_start_extrapolated : st->res_start_extrapolated;
    const double rsl = b == 0 ? ps.res_start_learned : st->res_start_learned;
    const int nits = st->newton_its + ps.newton_its, kits = st->krylov_its + ps.krylov_its;
    const int revs = st->residual_evals + ps.residual_evals, jvs = st->jv_evals + ps.jv_evals;
    const int f64 = st->f64_fallbacks + ps.f64_fallbacks, mgf = st->mg_fallbacks + ps.mg_fallbacks;
    *st = ps;
    st->start_used = start_used;
    st->res_start_extrapolated = rse;
    st->res_start_learned = rsl;
    st->newton_its = nits;
    st->krylov_its = kits;
    st->residual_evals = revs;
    st->jv_evals = jvs;
    st->f64_fallbacks = f64;
    st->mg_fallbacks = mgf;
    if (rc != PNP_OK) return rc;
  }
  // velocity history: v^{k-1} <- v^k <- v^{k+1}
  CK(cudaMemcpyAsync(c->vel_prev, c->vel, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  RC(ctx_ns_velocity(c, c->vel));
  CK(cudaStreamSynchronize(s));
  st->wall_ms = now_ms() - t0;
  return PNP_OK;
}
