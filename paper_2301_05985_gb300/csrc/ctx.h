// ctx.h -- the context object behind the opaque pnp_ctx handle.
#pragma once

#include "kernels.h"

// One level of the multigrid hierarchy (mg.cu): the level's context and the transfers
// between the next finer level (rows Nf) and this level (rows Nc), on the device.
struct MgLevel {
  pnp_ctx* sub = nullptr;             // the level's context (null for level 0: the owner)
  // transfer between the next finer level (rows Nf) and this level (rows Nc)
  int64_t* p_ptr = nullptr;
  int32_t* p_col = nullptr;
  float* p_w = nullptr;
  int64_t* r_ptr = nullptr;
  int32_t* r_col = nullptr;
  float* r_w = nullptr;
  int32_t* inject = nullptr;
  float *b = nullptr, *x = nullptr, *Ax = nullptr, *Dinv32 = nullptr;
};

struct pnp_ctx {
  int dim = 0, L = 0;
  int64_t n_elem = 0, n_nodes = 0, n_hanging = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  pnp_params prm{};
  int bc_type[6][3] = {};
  double bc_val[6][3] = {};
  cudaError_t latched = cudaSuccess;
  int64_t step = 0;
  bool start_fell_back = false;  // the last Newton solve started from its reference state
  bool history_split = false;  // U^{k-1} is not one full step behind U^k (after a split)

  // mesh (device)
  int32_t* d_conn = nullptr;
  int32_t* d_anchor = nullptr;  // [E][dim] element anchors, uploaded on first use (plane integrals)
  uint8_t* d_level = nullptr;
  uint8_t* d_faces = nullptr;  // boundary-face bits, bit 7 = hanging
  int32_t* d_hnode = nullptr;
  int32_t* d_hpar = nullptr;
  uint8_t* d_hnp = nullptr;

  // Morton patches for the shared-memory element kernels (device), their partial buffers
  bool use_patches = true;
  DevPatches pt;
  std::vector<void*> pt_alloc;
  double* part64 = nullptr;
  float* part32 = nullptr;

  // fields, FP64, [N][3]
  double *U = nullptr, *Uk = nullptr, *Ukm1 = nullptr;
  double *adv = nullptr, *vel = nullptr, *vel_prev = nullptr;
  double* hs = nullptr;  // [N][2]

  // FP32 mirrors for the mixed-precision Jv
  float *U32 = nullptr, *adv32 = nullptr, *hs32 = nullptr, *V32 = nullptr, *JV32 = nullptr;

  // Newton / Krylov scratch
  double *F = nullptr, *dU = nullptr, *Ut = nullptr, *Ft = nullptr, *rhs = nullptr;
  double* Dinv = nullptr;  // [N][9]
  float* D32 = nullptr;    // [N][9] FP32 block diagonal (mixed-precision preconditioner)
  double* basis = nullptr; // [(m+1)][3N]
  double *w = nullptr, *z = nullptr, *r = nullptr;
  double* part = nullptr;  // reduction partials [kRedBlocks][m+2]
  double* dsc = nullptr;   // small device scalars [2*(m+2) + 8]
  double* hpin = nullptr;  // pinned host mirror of dsc
  int* dflag = nullptr;
  int m_alloc = 0;
  // flexible outer GMRES with an inner FP32 GMRES(d) preconditioner
  float* Zb = nullptr;      // [m][3N] preconditioned Krylov vectors
  float* Qin = nullptr;     // [(d+1)][ldq] inner basis (unnormalised), rows padded with zeros
  int64_t ldq = 0;          // row length of Qin: 3N rounded up to a multiple of 4
  float* Dinv32 = nullptr;  // [N][9] FP32 copy of the inverted block diagonal
  double* isc = nullptr;    // inner Hessenberg [(d+1) x d] and scalars
  float* iinv = nullptr;    // [d+2] inverse norms of the inner basis vectors
  int inner_m = 0, inner_d = 0;
  // flexible outer GMRES with an inner FP64 GMRES(d) preconditioner (PNP_F64, gmres_inner > 0)
  double* Z64 = nullptr;    // [m][3N] preconditioned Krylov vectors
  double* Qin64 = nullptr;  // [(d+1)][3N] inner basis (unnormalised)
  double* zin64 = nullptr;  // [3N] block-Jacobi image of an inner basis vector
  double* isc64 = nullptr;  // [3 (d+2) + 2] inner projections, 1 / s_i^2, norm, combination
  int inner64_m = 0, inner64_d = 0;
  float4* rec32 = nullptr;  // [N][2] FP32 node records of the state for the FP32 J V
  float4* V4 = nullptr;     // [N] padded FP32 direction of the inner solve's J V
  float4* JV4 = nullptr;    // [N] padded FP32 J V accumulator
  float4* qp32 = nullptr;   // [4][2^dim E] stored Gauss-point linearisation of the FP32 J V
  bool lin_user = false;    // qp32 holds the linearisation of the last pnp_linearize
  int lin_rows = 4;         // float4 rows per lane in qp32 (3 without advection)
  bool adv_zero = false;    // the advection field was zero at the last ctx_prepare_f32
  int wait_polls = -1;      // poll limit of the staged J V's waits (< 0: the kernel's default)
  // the inner FP32 GMRES captured as a CUDA graph (replayed while profiling is off): the
  // launches depend only on the key below, captured on a stream of the context's own
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t inner_exec = nullptr;
  std::vector<unsigned char> inner_key;
  int64_t inner_graph_launches = 0;  // kernels one replay runs
  int inner_graph_jv = 0;            // J V applications one replay runs
  bool inner_eager_done = false;     // one eager solve ran (launchers' one-time set-up done)
  bool inner_graph_off = false;      // a capture was refused: eager from then on
  int64_t basis_bytes = 0;

  // geometric multigrid preconditioner (mg.cu): level hierarchy, built on first use
  std::vector<struct MgLevel>* mg = nullptr;
  int mg_built = 0;

  // Navier-Stokes block (ns.cu): state allocated on first use, boundary conditions per
  // face and slot (v_x, v_y, v_z, p)
  struct NsState* ns = nullptr;
  int ns_bc_type[6][4] = {};
  double ns_bc_val[6][4] = {};
  // pnp_coupled_step: the PNP step takes the advection as set (v^{k+1}) and leaves the
  // velocity history alone; a repeated block iteration starts from the U already set
  bool coupled = false;
  bool start_given = false;

  // statistics of the last solve (for the time stepper)
  int jv_count = 0, res_count = 0, mg_fallbacks = 0;

  // learned start (optional) and the host copy of the mesh it needs for point location
  struct Mlp* mlp = nullptr;
  pnp_mesh host_mesh;

  // profiling: event pairs per kernel class, resolved on read
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[PNP_PROF_KINDS] = {};
  int64_t prof_cnt[PNP_PROF_KINDS] = {};
  double prof_bytes[PNP_PROF_KINDS] = {};
  double prof_flops[PNP_PROF_KINDS] = {};
  // algorithmic bytes of one element-kernel launch: connectivity + level (+ hanging tables)
  double conn_bytes() const {
    return (double)n_elem * (4.0 * (1 << dim) + 1.0) + (double)n_hanging * 17.0;
  }
  cudaEvent_t take_event() {
    cudaEvent_t e = nullptr;
    if (!ev_pool.empty()) {
      e = ev_pool.back();
      ev_pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }

  int64_t n3() const { return 3 * n_nodes; }
  RowArgs rows() const {
    RowArgs R;
    R.n_nodes = n_nodes;
    R.n_hanging = n_hanging;
    R.faces = d_faces;
    R.hnode = d_hnode;
    R.hpar = d_hpar;
    R.hnp = d_hnp;
    R.bc = bc_table();
    return R;
  }
  BcTable bc_table() const {
    BcTable t{};
    for (int f = 0; f < 3; ++f) {
      uint8_t m = 0;
      for (int face = 0; face < 2 * dim; ++face)
        if (bc_type[face][f] == PNP_DIRICHLET) m |= (uint8_t)(1u << face);
      t.dir_faces[f] = m;
    }
    for (int face = 0; face < 6; ++face)
      for (int f = 0; f < 3; ++f) t.val[face][f] = bc_val[face][f];
    return t;
  }
  PhysParams phys() const {
    PhysParams P;
    P.eps2x2 = 2.0 * prm.eps * prm.eps;
    P.kappa = prm.steady ? 0.0 : prm.beta0 / prm.dt;
    P.tau_t = prm.steady ? 0.0 : 4.0 / (prm.dt * prm.dt);
    P.C_I = prm.C_I;
    P.steady = prm.steady;
    return P;
  }
};

// Records a CUDA event pair around the enclosed launches when profiling is on.
struct ProfScope {
  pnp_ctx* c;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(pnp_ctx* c_, int k, double bytes, double flops = 0.0) : c(c_), kind(k) {
    if (c->prof_on && kind >= 0) {  // kind < 0: not recorded
      c->prof_bytes[kind] += bytes;
      c->prof_flops[kind] += flops;
      a = c->take_event();
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = c->take_event();
      cudaEventRecord(b, c->stream);
      c->ev_pending.push_back({kind, {a, b}});
    }
  }
};

// Internal operations (return pnp_status).
int ctx_check(pnp_ctx* c, cudaError_t e, const char* what);
int ctx_prepare_history(pnp_ctx* c);
int ctx_residual(pnp_ctx* c, const double* U, double* F);
int ctx_jv64(pnp_ctx* c, const double* U, const double* V, double* JV);
int ctx_prepare_f32(pnp_ctx* c, const double* U);
int ctx_jv32(pnp_ctx* c, const float* V32, float* JV32);
// PNP_ERR_DEVICE_FLAG once a wait of the staged J V has given up (the flag is latched)
int ctx_check_staged_waits(pnp_ctx* c);
int ctx_block_diag(pnp_ctx* c, const double* U, double* D);
// FP32 blocks at the prepared FP32 state (ctx_prepare_f32 first)
int ctx_block_diag32(pnp_ctx* c, float* D);
int ctx_norm(pnp_ctx* c, const double* x, double* out);
int ctx_dot(pnp_ctx* c, const double* x, const double* y, double* out);
int ctx_gmres(pnp_ctx* c, const double* U, const double* b, double* x, double rtol, int precision, int max_it,
              int* its, double* relres, bool have_precond);
int ctx_newton(pnp_ctx* c, pnp_solve_stats* st, const double* ref_state = nullptr);
int ctx_alloc_inner(pnp_ctx* c, int m, int d);
int ctx_alloc_inner64(pnp_ctx* c, int m, int d);
int ctx_linearize32(pnp_ctx* c);
int ctx_jv32_linearized(pnp_ctx* c, const float* V, float* JV);
int ctx_time_step(pnp_ctx* c, pnp_solve_stats* st);
int ctx_alloc_krylov(pnp_ctx* c, int m);
void pnp_mlp_release(pnp_ctx* c);
// geometric multigrid (mg.cu): hierarchy of `levels` coarse octrees, per-solve state and
// blocks, one V-cycle z32 = M^-1 u
int ctx_mg_setup(pnp_ctx* c, int levels);
int ctx_mg_prepare(pnp_ctx* c, const double* U);
int ctx_mg_apply(pnp_ctx* c, const double* u, float* z32);
void ctx_mg_release(pnp_ctx* c);
int ctx_mg_level_count(const pnp_ctx* c);
// Navier-Stokes block (ns.cu)
int ctx_ns_alloc(pnp_ctx* c);
void ctx_ns_release(pnp_ctx* c);
double* ctx_ns_field(pnp_ctx* c);
int ctx_ns_prepare(pnp_ctx* c);
int ctx_ns_apply64(pnp_ctx* c, const double* X, const double* Ubody, double* F, bool data);
int ctx_ns_apply32(pnp_ctx* c, const float4* x, float4* y);
int ctx_ns_block_diag(pnp_ctx* c, double* Dg);
int ctx_ns_solve(pnp_ctx* c, const double* Ubody, pnp_ns_stats* st);
int ctx_ns_velocity(pnp_ctx* c, double* v3);
// [2][3N] scratch for the PNP history of repeated block iterations (allocated on first use)
double* ctx_ns_history_save(pnp_ctx* c);
int ctx_coupled_step(pnp_ctx* c, pnp_solve_stats* st, pnp_ns_stats* nst);
double now_ms();
