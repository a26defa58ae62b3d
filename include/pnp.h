/*
 * pnp.h -- C ABI of the GB300 library for the VMS-stabilised Poisson-Nernst-Planck block
 * on 2:1-balanced octrees (Kim, Saurabh, Khanwale, Mani, Anand,
 * Ganapathysubramanian, arXiv 2301.05985).
 *
 * What the library computes
 * -------------------------
 * Unknowns per mesh node: c+, c-, phi (valences +1, -1).  Non-dimensional PNP of
 * Sec. 2.2 (Eqs. nondim_poisson, nondim_np):
 *     -2 eps^2 lap(phi) = c+ - c-,      dc/dt + v.grad c = div(grad c + z c grad phi),
 * eps = Lambda (Debye length / domain length).  Time discretisation: BDF with
 * coefficients beta0..beta2 (Def. 1, Sec. 3).  Space: trilinear (bilinear in 2D) Q1
 * elements on octree leaves, 2x2x2 Gauss quadrature, VMS fine-scale closure
 * c^f = -tau_c R_c with tau_c = (4/dt^2 + (2/h)^2 |v|^2 + C_I d (2/h)^4)^(-1/2)
 * (Sec. 3.1), giving the discrete residual of Def. 3 (Poisson and Nernst-Planck rows).
 * Newton's method with the analytic Jacobian (Sec. 4.1, Eq. newton_linear_system) is
 * applied matrix-free: the library evaluates J(U) V directly.
 *
 * Conventions
 * -----------
 * - Domain: unit square (dim 2) or cube (dim 3).  Octant anchors and node coordinates
 *   are integers in units of 2^-max_level.  Faces: 2*axis + side (x-=0, x+=1, y-=2,
 *   y+=3, z-=4, z+=5).  Fields: c+ = 0, c- = 1, phi = 2.
 * - Vectors of unknowns are node-major FP64 arrays [n_nodes][3] (c+, c-, phi
 *   interleaved) in the library's node order (Morton order of node coordinates; use
 *   pnp_mesh_node_coords to map).  Velocities are [n_nodes][dim].
 * - Hanging nodes (edge midpoints / face centres of a coarser neighbour) are kept in
 *   every vector; their rows are the constraints U_h - sum_p w_p U_p (weights 1/2 or
 *   1/4) and their values never enter element computations.  Dirichlet rows are
 *   U_i - g_i in the residual and V_i in J V.  A node on several Dirichlet faces takes
 *   the value of the highest-numbered one; hanging nodes are never Dirichlet rows.
 * - Pointers marked "device" must be CUDA device pointers valid on the context's
 *   device; "host" pointers are ordinary host memory.  The caller owns every pointer it
 *   passes; the library owns its handles and internal scratch, released by the
 *   *_destroy calls.  All device work of a context is issued on the stream given at
 *   pnp_ctx_create; calls return after that work is complete unless stated otherwise.
 * - Every call returns PNP_OK (0) or an error code; nothing aborts.  After a CUDA
 *   error the context is latched: later calls on it return PNP_ERR_CUDA.
 *   pnp_last_error() gives a message for the calling thread's last failure.
 * - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef PNP_H
#define PNP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pnp_status {
  PNP_OK = 0,
  PNP_ERR_ARG = 1,               /* bad argument (null pointer, size, enum value) */
  PNP_ERR_MESH = 2,              /* octants overlap, leave gaps or are misaligned */
  PNP_ERR_MESH_UNBALANCED = 3,   /* neighbours (face, edge or corner) differ by > 1 level */
  PNP_ERR_NAN = 4,               /* a norm became NaN or Inf */
  PNP_ERR_KRYLOV_MAXIT = 5,      /* GMRES hit its iteration limit, or a restart cycle cut the
                                    true residual by less than 5% (stagnation) */
  PNP_ERR_NEWTON_DIVERGED = 6,   /* Newton hit its iteration limit or line search failed */
  PNP_ERR_CUDA = 7,              /* a CUDA call failed; the context is latched */
  PNP_ERR_DEVICE_FLAG = 8,       /* a kernel's own check failed (bad index / input), or a
                                    bounded wait of a kernel on its own copies gave up */
  PNP_ERR_NOMEM = 9,             /* host or device allocation failed */
  PNP_ERR_STATE = 10             /* call not valid in the current state */
};

enum { PNP_C_PLUS = 0, PNP_C_MINUS = 1, PNP_PHI = 2 };
enum { PNP_NATURAL = 0, PNP_DIRICHLET = 1 };
enum { PNP_F64 = 0, PNP_F32 = 1 };
enum { PNP_DEVICE = 0, PNP_HOST = 1 };
enum {
  PNP_FIELD_U = 0,             /* U^{k+1} iterate / current state      [n][3] */
  PNP_FIELD_U_PREV = 1,        /* U^k                                  [n][3] */
  PNP_FIELD_U_PREV2 = 2,       /* U^{k-1}                              [n][3] */
  PNP_FIELD_ADVECTION = 3,     /* advection velocity v~ of the residual [n][dim] */
  PNP_FIELD_VELOCITY = 4,      /* fluid velocity v^k                    [n][dim] */
  PNP_FIELD_VELOCITY_PREV = 5, /* fluid velocity v^{k-1}                [n][dim] */
  PNP_FIELD_NS = 6             /* Navier-Stokes unknown (v_x, v_y, v_z, p) at the latest
                                  solve (start of the next one)       [n][4]; 2D: v_z = 0 */
};
enum { PNP_NS_VX = 0, PNP_NS_VY = 1, PNP_NS_VZ = 2, PNP_NS_P = 3 };
enum { PNP_START_PREVIOUS = 0, PNP_START_EXTRAPOLATE = 1, PNP_START_LEARNED = 2 };

typedef struct pnp_mesh pnp_mesh;
typedef struct pnp_ctx pnp_ctx;

/* Parameters.  Fill with pnp_params_default, then override. */
typedef struct pnp_params {
  double eps;            /* Lambda; Poisson coefficient is 2*eps^2 (Eq. nondim_poisson) */
  double dt;             /* time step (ignored when steady) */
  double C_I;            /* tau_c constant (6, Sec. 3.1) */
  double beta0, beta1, beta2; /* BDF coefficients used by pnp_residual / pnp_jv /
                                 pnp_newton_solve; pnp_time_step sets them itself */
  int32_t steady;        /* 1: drop the d/dt terms and the 4/dt^2 term of tau_c */
  int32_t bdf_order;     /* pnp_time_step: 1 or 2 (first step is always BDF1) */
  double newton_rtol;    /* stop when ||F(U^m)||_2 <= newton_rtol ||F(U^0)||_2; in
                            pnp_time_step the reference is ||F(U^k)||_2 of the
                            previous-step state whatever the start, so that all starts
                            meet one absolute tolerance */
  double newton_atol;    /* ... or ||F(U^m)||_2 <= newton_atol */
  int32_t newton_max_it;
  int32_t line_search;   /* 1: backtracking (halving, Armijo 1e-4) on ||F||_2 */
  int32_t gmres_restart; /* Krylov basis size m (<= 200) */
  int32_t gmres_max_it;  /* total Krylov iterations per linear solve */
  double gmres_rtol;     /* linear tolerance (plain mode) */
  int32_t precision;     /* PNP_F64: FP64 J V in Krylov (plain); PNP_F32: FP32 J V
                            inside an inexact Newton (Eisenstat-Walker forcing) */
  int32_t start_mode;    /* pnp_time_step Newton start: PNP_START_* */
  double ew_eta_max;     /* Eisenstat-Walker: largest forcing term (0.9) */
  double ew_eta_min;     /* Eisenstat-Walker: smallest forcing term (1e-4) */
  int32_t monitor;       /* 1: one line per Newton iteration on stderr */
  int32_t f64_fallback;  /* 1: when an FP32-J V Newton iteration fails to decrease
                            ||F||, redo it with FP64 J V (default 1) */
  int32_t gmres_cgs2;    /* 0: one classical Gram-Schmidt pass per Krylov vector (PETSc's
                            default, used by the paper's solver); 1: always a second pass */
  int32_t dt_retries;    /* pnp_time_step: when Newton fails, redo the step as two BDF1
                            half steps, recursively up to this depth (0: report the
                            failure; the next full step after a split is BDF1 and starts
                            from the previous state, because the history spacing changed) */
  int32_t gmres_inner;   /* PNP_F32 Krylov solves: 0 = right-preconditioned GMRES(m) with
                            the block diagonal; d in 1..64 = flexible GMRES(m) whose
                            preconditioner is d steps of FP32 GMRES on J M^-1 (M the
                            block diagonal), with FP64 outer dots and orthogonalisation;
                            with PNP_F64 the same flexible scheme with d steps of FP64 GMRES
                            (FP64 J V, basis and dots) as the preconditioner */
  int32_t newton_ew_f64; /* PNP_F64 Newton: 0 = each linear solve to gmres_rtol (exact Newton,
                            the default); 1 = Eisenstat-Walker forcing as in PNP_F32 */
  int32_t mg_levels;     /* PNP_F32 Krylov solves: 0 = off; L > 0 = flexible GMRES(m) in FP64
                            preconditioned by one FP32 V-cycle of geometric multigrid over up to
                            L coarser octrees, each the previous one with its finest level
                            capped (in place of the paper's GAMG, App. A); a solve in which the
                            cycle falls behind (see mg_fallbacks) continues with the inner FP32
                            GMRES of gmres_inner (24 steps when 0).  Non-periodic meshes. */
  int32_t mg_smooth;     /* damped block-Jacobi sweeps before and after the coarse correction (2) */
  double mg_omega;       /* damping of the sweeps (0.5) */
  int32_t mg_coarse_its; /* block-Jacobi sweeps on the coarsest level (16) */
  /* Navier-Stokes block (semi-implicit VMS momentum and solenoidality, Def. 3 and Sec. 3.1) */
  int32_t ns_blocks;     /* pnp_coupled_step: NS -> PNP block iterations per step (1; Sec. 4.1) */
  double ns_Sc;          /* Schmidt number Sc: inertia coefficient 1/Sc, 1/Re = Sc in tau_m (1) */
  double ns_kappa;       /* electrohydrodynamic coupling constant kappa: body force
                            kappa / (2 Lambda^2) (c+ - c-) grad phi (0.5) */
  double ns_rtol;        /* NS linear solve: ||F(X)||_2 <= max(ns_rtol ||F(X^0)||_2, ns_atol)
                            (1e-8 and 1e-10, the tolerances of App. A) */
  double ns_atol;
  double ns_inner_rtol;  /* relative residual reduction of the FP32 BiCGStab of each FP64
                            refinement step (1e-3) */
  int32_t ns_max_it;     /* total FP32 BiCGStab iterations per NS solve (4000) */
  int32_t ns_pin;        /* 1: the pressure of the node at the origin is pinned to 0 unless a
                            pressure Dirichlet face holds it (1) */
  int32_t ns_mg_levels;  /* 0: BiCGStab preconditioned by the inverted 4x4 nodal blocks; L > 0:
                            by one FP32 V-cycle of geometric multigrid over up to L coarser
                            octrees (the hierarchy of mg_levels, shared with it: mg_levels wins
                            when both are set), damped block-Jacobi sweeps (mg_smooth, mg_omega,
                            mg_coarse_its), rediscretised NS operators at the injected v~.
                            Non-periodic meshes (0) */
  int32_t ns_inner_max_it; /* BiCGStab iterations per FP64 refinement step (200) */
  int32_t ns_fgmres;     /* 0: FP32 BiCGStab under FP64 defect correction; m in 1..200: FGMRES(m)
                            in FP64 (basis, dots, matrix action) right-preconditioned in FP32 by
                            the same V-cycle or blocks, restarted to the tolerance (30) */
  int32_t pad4_;
} pnp_params;

typedef struct pnp_solve_stats {
  int32_t status;        /* pnp_status of the solve */
  int32_t newton_its;
  int32_t krylov_its;    /* total over the Newton iterations */
  int32_t residual_evals;
  int32_t jv_evals;
  int32_t start_used;    /* PNP_START_* actually used (learned start may fall back) */
  int32_t f64_fallbacks; /* Newton iterations redone with FP64 J V */
  int32_t substeps;      /* pnp_time_step: Newton solves that completed the step
                            (1 unless dt_retries split it) */
  double res0;           /* ||F(U^0)||_2 */
  double res_final;      /* ||F(U^m)||_2 */
  double res_start_extrapolated; /* learned start only: ||F|| of the extrapolated start */
  double res_start_learned;      /* learned start only: ||F|| of the best network-based start */
  double wall_ms;        /* host wall time of the call */
  double res_ref;        /* ||F|| the relative Newton tolerance refers to: res0, or in
                            pnp_time_step ||F(U^k)|| of the previous-step state */
  int32_t mg_fallbacks;  /* Krylov solves in which the multigrid preconditioner fell behind (20
                            iterations without halving the residual, or a restart cycle that cut
                            it by less than 5%) and the solve went on with the inner FP32 GMRES
                            (gmres_inner, or 24 steps) */
  int32_t pad_;
} pnp_solve_stats;

/* Statistics of one Navier-Stokes linear solve. */
typedef struct pnp_ns_stats {
  int32_t status;        /* pnp_status of the solve */
  int32_t refinements;   /* FGMRES restart cycles, plus FP64 refinement steps (one FP32
                            BiCGStab each) */
  int32_t inner_its;     /* total Krylov iterations (FGMRES, then BiCGStab) */
  int32_t matvecs32;     /* FP32 operator applications on the finest mesh: 2 per BiCGStab
                            iteration and 2 mg_smooth per V-cycle */
  int32_t matvecs64;     /* FP64 operator applications (FGMRES matrix actions and residuals) */
  int32_t singular_blocks; /* 1 when a 4x4 diagonal block was singular (replaced by I) */
  int32_t floor_stop;    /* 1 when the solve stopped at the rounding floor of the FP64 residual
                            (three refinement steps without progress, ||F|| <= 1e-9 ||F(X^0)||)
                            above the requested tolerance */
  int32_t mg_fallbacks;  /* refinement steps whose multigrid-preconditioned correction raised
                            ||F||: undone, the rest of the solve used the inverted blocks */
  int32_t krylov_fallbacks; /* 1 when FGMRES stagnated (three restart cycles cutting ||F|| by
                            less than 5 %) and the solve continued with BiCGStab refinement */
  int32_t pad_;
  double res0;           /* ||F(X^0)||_2 */
  double res_final;      /* ||F(X)||_2 */
  double wall_ms;        /* host wall time of the call */
} pnp_ns_stats;

/* Message for the calling thread's most recent failure ("" if none).  Static storage. */
const char* pnp_last_error(void);

/* Library version string. */
const char* pnp_version(void);

void pnp_params_default(pnp_params* p);

/* ---------------------------------------------------------------- mesh (host) ---- */
/* Build the Q1 mesh of a complete linear octree (Sec. 4.2: octree leaves are the
 * elements).  anchors: host int32 [n_oct][dim] (units of 2^-max_level, aligned to the
 * octant size), levels: host uint8 [n_oct] (0..max_level), max_level <= 16.  The
 * octants must tile the unit domain without overlap (PNP_ERR_MESH) and be 2:1 balanced
 * across faces, edges and corners (PNP_ERR_MESH_UNBALANCED).  Elements are reordered
 * by Morton order; nodes are the unique element corners in Morton order.  *out is
 * owned by the caller and released by pnp_mesh_destroy. */
int pnp_mesh_create(int dim, int max_level, int64_t n_oct, const int32_t* anchors,
                    const uint8_t* levels, pnp_mesh** out);
/* The same with periodic sides: bit k of `periodic` (0 <= periodic < 2^dim) identifies the
 * faces x_k = 0 and x_k = 1 (the periodic side walls of the paper's electroconvection
 * setup, Sec. 5.2).  A node on an identified face is one node, stored with coordinate 0;
 * those faces carry no boundary condition; hanging constraints, conformity and the 2:1
 * balance are taken across the identification (PNP_ERR_MESH_UNBALANCED otherwise).
 * pnp_mesh_create is the case periodic = 0.  The learned start (pnp_mlp_init) rejects
 * periodic meshes (PNP_ERR_ARG). */
int pnp_mesh_create_periodic(int dim, int max_level, int64_t n_oct, const int32_t* anchors,
                             const uint8_t* levels, int periodic, pnp_mesh** out);
/* The same after refinement (the paper builds its octrees top-down with a refinement
 * predicate on coordinates and field values, Sec. 4.2, and refines near the membrane and
 * where the fields vary fastest, Sec. 5.2): every input octant is split until it reaches
 * target_levels[e] (host uint8 [n_oct], <= max_level; NULL = no targets), then leaves are
 * split until the octree is 2:1 balanced across faces, edges and corners (across the
 * identified faces of periodic axes too).  The result is the coarsest balanced octree
 * refining each octant to at least its target; pnp_mesh_elements returns its leaves.
 * The input octants must tile the domain without overlap (PNP_ERR_MESH otherwise). */
int pnp_mesh_create_refined(int dim, int max_level, int64_t n_oct, const int32_t* anchors,
                            const uint8_t* levels, const uint8_t* target_levels, int periodic,
                            pnp_mesh** out);
/* The coarse octrees of the multigrid preconditioner (mg_levels): the same octree with
 * every leaf finer than cap_level replaced by its ancestor at cap_level (2:1 balance is
 * kept).  Its Q1 space is contained in the mesh's, and every coarse node is a point of
 * the fine mesh.  *out is released by pnp_mesh_destroy. */
int pnp_mesh_coarsen(const pnp_mesh* m, int cap_level, pnp_mesh** out);
/* The grid transfer between a mesh and a coarsening of it (pnp_mesh_coarsen): the
 * prolongation P, fine node values of a coarse Q1 field (trilinear interpolation in the
 * coarse element holding the node, coarse hanging corners expanded to their parents), as
 * CSR host arrays ptr int64 [n_fine_nodes + 1], col int32 [nnz] (independent coarse
 * nodes), w float [nnz]; the restriction is its transpose.  inject int32 [n_coarse_nodes]:
 * the fine node at each coarse node's point.  *nnz is always set; the array pointers may
 * be NULL (call once with NULL to size them).  Non-periodic meshes only. */
int pnp_mesh_transfer(const pnp_mesh* fine, const pnp_mesh* coarse, int64_t* nnz, int64_t* ptr,
                      int32_t* col, float* w, int32_t* inject);
void pnp_mesh_destroy(pnp_mesh* m);
int pnp_mesh_info(const pnp_mesh* m, int* dim, int* max_level, int64_t* n_elem,
                  int64_t* n_nodes, int64_t* n_hanging);
/* Integer node coordinates, host int32 [n_nodes][dim]. */
int pnp_mesh_node_coords(const pnp_mesh* m, int32_t* ijk);
/* Hanging flags, host uint8 [n_nodes] (1 = hanging). */
int pnp_mesh_hanging(const pnp_mesh* m, uint8_t* flags);
/* Element anchors host int32 [n_elem][dim] and levels host uint8 [n_elem] in the
 * library's (Morton) element order. */
int pnp_mesh_elements(const pnp_mesh* m, int32_t* anchors, uint8_t* levels);
/* Statistics of the Morton patches the element kernels use (host int64 [7]): patches,
 * most nodes in a patch, most colours, nodes shared between patches, partial rows,
 * total patch slots, and the number of violated layout invariants (0 when valid). */
int pnp_mesh_patch_stats(const pnp_mesh* m, int64_t* stats);

/* ---------------------------------------------------------------- context -------- */
/* Create a context on the current CUDA device: uploads the mesh (the mesh may be
 * destroyed afterwards), allocates fields and solver scratch.  stream: a cudaStream_t
 * (NULL = legacy default stream) on which all of this context's work runs.  All
 * fields start at zero; all faces start with natural (zero-flux) conditions. */
int pnp_ctx_create(const pnp_mesh* m, const pnp_params* p, void* stream, pnp_ctx** out);
void pnp_ctx_destroy(pnp_ctx* c);
int pnp_set_params(pnp_ctx* c, const pnp_params* p);
int pnp_get_params(const pnp_ctx* c, pnp_params* p);
/* Boundary condition of one field on one face (Table tab:BC-AliMani style): type
 * PNP_DIRICHLET (value g) or PNP_NATURAL (zero total flux for c+-, zero normal
 * derivative for phi). */
int pnp_set_bc(pnp_ctx* c, int face, int field, int type, double value);
/* Copy a field in (set) or out (get).  where = PNP_DEVICE or PNP_HOST selects the kind
 * of pointer; layout per the PNP_FIELD_* comments, FP64. */
int pnp_set_field(pnp_ctx* c, int which, const double* src, int where);
int pnp_get_field(pnp_ctx* c, int which, double* dst, int where);
/* Impose Dirichlet values and hanging-node interpolation on PNP_FIELD_U. */
int pnp_make_consistent(pnp_ctx* c);

/* ---------------------------------------------------------------- operators ------ */
/* F = residual of Def. 3 at U (device [n][3] FP64 each), using the context's
 * U_PREV / U_PREV2 (BDF history), ADVECTION, parameters and boundary conditions. */
int pnp_residual(pnp_ctx* c, const double* U, double* F);
/* JV = J(U) V, the directional derivative of the residual (device pointers).
 * precision PNP_F64: V, JV are FP64 [n][3]; PNP_F32: V, JV are FP32 [n][3] and the
 * element arithmetic runs in FP32 (U is rounded to FP32 once per call). */
int pnp_jv(pnp_ctx* c, const double* U, const void* V, void* JV, int precision);
/* FP32 J V through a stored linearisation, for many directions at one state (the
 * inner Krylov solve of the flexible GMRES uses the same kernels).  pnp_linearize
 * evaluates at U (device FP64 [n][3]), with the context's history, advection, parameters
 * and boundary conditions at this call, the state's quantities at every element's
 * Gauss points that J V needs (Def. 3 linearised: v, grad phi, grad c+-, tau_c and
 * z (c - tau_c R) per Gauss point, FP32, 64 B each, held by the context; 48 B when the
 * advection field is zero: v and tau_c are then not stored, tau_c follows from the level).
 * pnp_jv_linearized then returns JV = J V for FP32 device vectors V, JV [n][3], equal to
 * pnp_jv(..., PNP_F32) at that U up to FP32 summation order.  A later solver call
 * (pnp_gmres, pnp_newton_solve, pnp_time_step) replaces the stored linearisation;
 * pnp_jv_linearized then returns PNP_ERR_STATE until pnp_linearize is called again.
 * The J V kernel streams the stored quantities through shared memory with bulk copies;
 * if one of its bounded waits on them gives up, the block waits (with a longer bound) for
 * the copies it issued, exits, and the call raises PNP_ERR_DEVICE_FLAG (here, and from the
 * solver calls that use it).  The flag stays set until the next linearisation (a
 * pnp_linearize, or the start of the next flexible Krylov solve). */
int pnp_linearize(pnp_ctx* c, const double* U);
int pnp_jv_linearized(pnp_ctx* c, const float* V, float* JV);
/* The poll limit of each bounded wait of the staged J V above (polls < 0: the default,
 * 2^22 polls, about a second; at most 2^30).  A limit of 0 makes every wait give up at
 * once while the copies still land: it exercises the failure path on a healthy GPU. */
int pnp_set_wait_limit(pnp_ctx* c, int64_t polls);
/* 3x3 diagonal blocks of J(U): D device FP64 [n][3][3] (row-major per node), exact
 * for the assembled operator including hanging-node coupling.  Dirichlet rows are
 * identity rows, hanging rows identity blocks. */
int pnp_block_diag(pnp_ctx* c, const double* U, double* D);
/* The same blocks in FP32 arithmetic at U rounded to FP32 (D device FP32 [n][3][3]):
 * the blocks the mixed-precision solver inverts for its block-Jacobi preconditioner. */
int pnp_block_diag_f32(pnp_ctx* c, const double* U, float* D);
/* Species fluxes through boundary face `face` (0 <= face < 2 dim; axis face/2, the high
 * side when face is odd): flux[s] = int_face n . (grad c_s + z_s c_s grad phi) dS for
 * s = +, - (z = +1, -1), n the outward unit normal, U a device FP64 [n][3] state (hanging
 * entries ignored, taken from their constraints).  Each element side on the face is
 * integrated with the 2^(d-1)-point Gauss rule; the sum is reduced in a fixed order.
 * These are the terms of the boundary current of Sec. 5.2, the net species flux
 * through the top boundary: j_T = -(flux[0] - flux[1]) / L_T, L_T the face's length
 * (area in 3D; 1 on the unit domain).  A periodic face gives 0.  flux: host double[2]. */
int pnp_boundary_flux(pnp_ctx* c, const double* U, int face, double* flux);
/* Refinement indicator: |grad c+|, |grad c-|, |grad phi| of the Q1 fields of U (device FP64
 * [n][3], hanging entries taken from their constraints) at the centre of every element,
 * G device FP64 [n_elem][3] in the library's element order (pnp_mesh_elements).  With
 * pnp_mesh_create_refined it refines where the fields vary fastest (Sec. 5.2 refines the
 * electroconvection meshes where the concentration gradients are largest). */
int pnp_element_gradient(pnp_ctx* c, const double* U, double* G);
/* Averages of (c+, c-, phi) over the plane x_axis = coord * 2^-max_level (0 <= coord <=
 * 2^max_level; coord < 2^max_level on a periodic axis) of the unit domain: the integral
 * of each Q1 field over the plane, each element's cross-section integrated with the
 * 2^(d-1)-point Gauss rule (exact), U a device FP64 [n][3] state.  Evaluated at every node
 * level along the wall-normal axis these are the x-averaged profiles of Sec. 5.2.  The
 * first call uploads the element anchors (4 dim bytes per element).  avg: host double[3]. */
int pnp_plane_average(pnp_ctx* c, const double* U, int axis, int64_t coord, double* avg);
/* ||x||_2 of a device FP64 vector of n entries, the reduction Newton and GMRES use
 * (fixed grid, fixed summation order: bitwise reproducible); result on the host.
 * x may be NULL when n == 0.  Uses the context's scratch and stream. */
int pnp_norm2(pnp_ctx* c, const double* x, int64_t n, double* result);

/* ---------------------------------------------------------------- solvers -------- */
/* The linear solve of each Newton iteration (Sec. 4.1, Eq. newton_linear_system), by the
 * Krylov method of the paper's PNP solver options (App. A: PETSc FGMRES, relative
 * tolerance 1e-8), with a 3x3 block-Jacobi preconditioner in place of its GAMG.
 * Solve J(U) x = b by right-preconditioned GMRES(m) (3x3 block-Jacobi preconditioner,
 * classical Gram-Schmidt, a second pass when gmres_cgs2, FP64 basis and dot products;
 * convergence accepted after a true-residual check).
 * U, b, x: device FP64 [n][3]; x is the initial guess on entry.  rtol relative to
 * ||b||; precision selects the J V arithmetic. */
int pnp_gmres(pnp_ctx* c, const double* U, const double* b, double* x, double rtol,
              int precision, pnp_solve_stats* st);
/* Newton solve of F(U) = 0 for PNP_FIELD_U in place (Sec. 4.1: Newton's method on the
 * fully discrete PNP residual of Def. 3 with the analytic Jacobian, Eq.
 * newton_linear_system, here applied matrix-free), starting from its current value (made
 * consistent first), with the context's parameters: stop when ||F|| <= newton_rtol
 * ||F(U^0)|| or newton_atol; PNP_F64 solves each linear system with pnp_gmres to
 * gmres_rtol (App. A's 1e-8), PNP_F32 inexactly (Eisenstat-Walker forcing) with FP32 J V;
 * optional backtracking line search.  Returns PNP_ERR_NEWTON_DIVERGED when newton_max_it
 * is reached or the line search fails, PNP_ERR_NAN on a non-finite norm. */
int pnp_newton_solve(pnp_ctx* c, pnp_solve_stats* st);
/* One BDF time step (Def. 1): BDF1 on the first step, then bdf_order; advection
 * v~ = 2 v^k - v^{k-1} (Eq. averaging1) from the VELOCITY fields; Newton start per
 * start_mode, Newton tolerance relative to ||F(U^k)|| (see newton_rtol); a start whose
 * residual norm exceeds ||F(U^k)|| is replaced by U^k (st->start_used then reports
 * PNP_START_PREVIOUS); on success
 * U_PREV2 <- U_PREV <- U^{k+1} = U and VELOCITY_PREV <- VELOCITY.  With dt_retries > 0
 * a step whose Newton solve fails is redone as two BDF1 half steps (recursively);
 * st->substeps counts the solves that completed it.  On failure the context keeps the
 * last completed (sub)step as U_PREV.  The BDF coefficients and dt used last are left
 * in the context's parameters except dt, which is restored. */
int pnp_time_step(pnp_ctx* c, pnp_solve_stats* st);
/* Number of steps taken so far by pnp_time_step (0 after pnp_ctx_create or
 * pnp_reset_history). */
int pnp_step_count(const pnp_ctx* c, int64_t* k);
/* Resume a trajectory (e.g. from a checkpoint written with pnp_get_field): declare that
 * U_PREV and U_PREV2 hold the states of steps k and k-1 of equally spaced steps.  The next
 * pnp_time_step is BDF2 when k >= 1 (and bdf_order is 2) and may extrapolate its start;
 * k = 0 makes it a first step (BDF1, previous-step start). */
int pnp_set_step_count(pnp_ctx* c, int64_t k);
/* Start a new trajectory: U_PREV and U_PREV2 <- U, step count <- 0. */
int pnp_reset_history(pnp_ctx* c);

/* ---------------------------------------------------------------- Navier-Stokes -- */
/* The semi-implicit VMS Navier-Stokes block (Def. 3 momentum and solenoidality with the
 * closure v^f = -tau_m R_m, p^f = -tau_sol R_sol of Sec. 3.1), linear in X = (v, p) at
 * t^{k+1}: with v~ = 2 v^k - v^{k-1} (Eq. averaging1) from VELOCITY / VELOCITY_PREV,
 *   momentum, test N_a e_i:  N_a R_m,i + grad N_a . grad v_i
 *                            + (1/Sc) tau_m (v~ . grad N_a) R_m,i + d_i N_a tau_sol div v
 *   solenoidality, test N_a: N_a div v + tau_m grad N_a . R_m
 *   R_m,i = (1/Sc)((beta0 v_i + beta1 v_i^k + beta2 v_i^{k-1})/dt + v~ . grad v_i) + d_i p
 *           + kappa / (2 Lambda^2) (c+ - c-) d_i phi,
 *   tau_m = (4/dt^2 + (2/h)^2 |v~|^2 + C_I Sc^2 d (2/h)^4)^(-1/2), tau_sol = 1/(d (2/h)^2 tau_m)
 * (parameters ns_Sc, ns_kappa, eps, dt, beta0..2, C_I, steady).  The solenoidality row
 * takes +tau_m grad N_a . R_m, the sign v^f = -tau_m R_m gives (the printed form has a
 * minus and a misprinted test function there).  Unknowns node-major [n][4] = (v_x, v_y,
 * v_z, p), 2D: slot v_z inactive (its row is X = 0).  Rows: hanging-node constraints,
 * Dirichlet rows X - g from pnp_ns_set_bc, and with ns_pin the pressure of the node at
 * the origin fixed to 0.  The PNP state of the body force is PNP_FIELD_U. */
/* Boundary condition of slot PNP_NS_* on one face: PNP_DIRICHLET (value g; a no-slip wall
 * is g = 0 on the three velocity slots) or PNP_NATURAL (the boundary terms of the weak
 * form vanish). */
int pnp_ns_set_bc(pnp_ctx* c, int face, int slot, int type, double value);
/* F = the NS rows at X (device FP64 [n][4] each): the residual of the linear system,
 * A X - b, with b from the history, the body force and the Dirichlet values. */
int pnp_ns_residual(pnp_ctx* c, const double* X, double* F);
/* Y = A X: the matrix of the linear system (the residual without its data terms), with
 * identity rows on Dirichlet / pin rows and the constraint rows of hanging nodes.
 * precision PNP_F64: double [n][4]; PNP_F32: float [n][4] (16-byte aligned). */
int pnp_ns_matvec(pnp_ctx* c, const void* X, void* Y, int precision);
/* The 4x4 nodal diagonal blocks of A (device FP64 [n][16], row-major per node) before the
 * row substitutions; a hanging corner contributes w_p^2 times its own block to each
 * parent p (the cross pairs through hanging corners are left out).  The preconditioner
 * of pnp_ns_solve inverts them (identity rows on constrained rows). */
int pnp_ns_block_diag(pnp_ctx* c, double* D);
/* Solve the linear NS system for PNP_FIELD_NS in place, starting from its value, until
 * ||F(X)|| <= max(ns_rtol ||F(X^0)||, ns_atol), right-preconditioned in FP32 by the inverted
 * diagonal blocks or (ns_mg_levels) a multigrid V-cycle.  ns_fgmres = m > 0 (default):
 * FGMRES(m) with an FP64 basis, FP64 dots and FP64 matrix action, restarted (three restart
 * cycles in a row that cut ||F|| by less than 5 % hand the solve, from its iterate, to the
 * BiCGStab refinement below: st->krylov_fallbacks).  ns_fgmres = 0: FP64 defect
 * correction around FP32 BiCGStab (App. A solves this block with BiCGStab) of at most
 * ns_inner_max_it iterations each (a step that raises ||F|| is undone, and with multigrid the
 * solve continues with the blocks).  PNP_ERR_KRYLOV_MAXIT after ns_max_it Krylov
 * iterations, 60 refinement steps, or when progress stops above 1e-9 ||F(X^0)|| (at or below
 * it the solve ends as converged with st->floor_stop = 1); PNP_ERR_NAN on a non-finite
 * norm.  st->inner_its counts the Krylov iterations, st->refinements the FGMRES restart
 * cycles or refinement steps.  Uses the context's beta0..2. */
int pnp_ns_solve(pnp_ctx* c, pnp_ns_stats* st);
/* One NS-PNP time step by block iteration (Sec. 4.1): ns_blocks times, the NS system
 * (body force from U^k in the first pass, then from the latest U^{k+1}) and then the PNP
 * Newton solve of pnp_time_step with the new velocity v^{k+1} as the advection; BDF1 on the
 * first step, then bdf_order, for both blocks.  On success VELOCITY_PREV <- VELOCITY <-
 * v^{k+1}, PNP_FIELD_NS holds (v, p)^{k+1} and the PNP history is shifted as in
 * pnp_time_step.  pst: the last PNP solve (Newton / Krylov counts summed over the block
 * iterations), nst: the NS solves (iterations summed). */
int pnp_coupled_step(pnp_ctx* c, pnp_solve_stats* pst, pnp_ns_stats* nst);

/* ---------------------------------------------------------------- learned start -- */
/* The library's addition to the paper (which has no learned component): a per-node
 * network proposes the Newton start of pnp_time_step (start_mode PNP_START_LEARNED);
 * plain Newton judges it -- the start with the smallest ||F|| of {learned U_l,
 * extrapolated U_e = 2 U^k - U^{k-1}, blend U_e + a (U_l - U_e)} is used, with a in
 * [0, 2] the minimiser of ||F_e + a (F_l - F_e)|| (one extra residual).  After three
 * steps in a row won by U_e the network and the judge's residuals are skipped for the
 * next four steps (U_e is used; st->res_start_learned = -1), then tried again.
 *
 * Input (216 features per non-hanging node): the fields c+, c-, phi and the last-axis
 * velocity component at t^k and t^{k-1}, sampled at the 3x3x3 lattice around the node
 * with spacing equal to the finest element that has the node as a corner (points
 * clamped to the domain; Q1 interpolation where a point is not a node); feature index
 * ((step*4 + field)*27 + point), point index x fastest over offsets {-1,0,1}^3.
 * Each (step, field) group is standardised with the training data's per-field mean and
 * standard deviation.  Network: 216 -> 128 -> 128 -> 128 -> 3, GELU x Phi(x) after the
 * hidden layers, BF16 weights and activations, FP32 accumulation on the tensor cores.
 * Output: the standardised correction U^{k+1} - (2 U^k - U^{k-1}) per field.
 * Parameters (FP32 master copy) are packed as W1[216][128], b1[128], W2[128][128], b2,
 * W3[128][128], b3, W4[128][3], b4[3]: PNP_MLP_PARAMS floats.  3D meshes only. */
#define PNP_MLP_PARAMS 61187

typedef struct pnp_train_cfg {
  int32_t steps;       /* Adam steps */
  int32_t batch;       /* samples (node, time) per step, <= 65536 */
  double lr;           /* Adam learning rate (1e-3) */
  double beta1, beta2, adam_eps; /* 0.9, 0.999, 1e-8 */
  uint64_t seed;       /* sampling seed */
} pnp_train_cfg;

typedef struct pnp_train_stats {
  double loss_first;   /* mean-squared error (standardised units) of the first batch */
  double loss_last;    /* ... of the last batch */
  double wall_ms;
  int64_t samples;     /* (node, time) pairs available */
  int32_t steps;
  int32_t pad_;
} pnp_train_stats;

/* Allocate the network of a context: He-normal weights from seed, zero biases, Adam
 * state cleared, identity standardisation; builds the stencil tables of the mesh. */
int pnp_mlp_init(pnp_ctx* c, uint64_t seed);
/* Host FP32 parameters in the packed order, n = PNP_MLP_PARAMS. */
int pnp_mlp_set_weights(pnp_ctx* c, const float* params, int64_t n);
int pnp_mlp_get_weights(pnp_ctx* c, float* params, int64_t n);
/* Standardisation (host arrays): input mean/std per field (c+, c-, phi, u) [4] each,
 * output mean/std per field [3] each. */
int pnp_mlp_set_normalization(pnp_ctx* c, const double* in_mean, const double* in_std, const double* out_mean,
                              const double* out_std);
int pnp_mlp_get_normalization(pnp_ctx* c, double* in_mean, double* in_std, double* out_mean, double* out_std);
/* Append a trajectory produced by the solver: states device FP64 [T][n_nodes][3]
 * (consecutive time levels, T >= 3), uz device FP64 [T][n_nodes] or NULL (zero).
 * The data are copied. */
int pnp_mlp_add_trajectory(pnp_ctx* c, const double* states, int64_t T, const double* uz);
int pnp_mlp_clear_data(pnp_ctx* c);
/* Train with Adam on the appended trajectories (standardisation computed from them
 * first).  Marks the network as trained. */
int pnp_mlp_train(pnp_ctx* c, const pnp_train_cfg* cfg, pnp_train_stats* st);
/* Raw (unstandardised) features of every non-hanging node, node order: device FP64
 * [n_free][216]; nodes: device int32 [n_free] (may be NULL).  n_free is the number of
 * non-hanging nodes. */
int pnp_mlp_features(pnp_ctx* c, const double* Uk, const double* Ukm1, const double* uz_k, const double* uz_km1,
                     double* X, int32_t* nodes);
/* Network output for B standardised input rows: X device FP32 [B][216] (rounded to
 * BF16 inside), Y device FP32 [B][3]. */
int pnp_mlp_forward(pnp_ctx* c, const float* X, int64_t B, float* Y);
/* Mean-squared-error loss and its gradient with respect to the packed parameters for
 * B rows: X device FP32 [B][216], Yt device FP32 [B][3], grad device FP32
 * [PNP_MLP_PARAMS]; *loss on the host.  B <= 65536. */
int pnp_mlp_loss_grad(pnp_ctx* c, const float* X, const float* Yt, int64_t B, float* grad, double* loss);
/* One Adam update (Kingma and Ba, "Adam: a method for stochastic optimization", ICLR
 * 2015, Algorithm 1, with bias correction) of the FP32 master parameters with a given
 * gradient, the same update pnp_mlp_train applies after each batch:
 *     t += 1;  m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *     p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 * in FP32 per parameter, then the BF16 weights are refreshed.  grad: device FP32
 * [PNP_MLP_PARAMS] in the packed order; cfg: lr, beta1, beta2, adam_eps (steps, batch and
 * seed are ignored).  The moments and t carry over between calls and pnp_mlp_train
 * steps; pnp_mlp_init clears them.  Lets a caller run its own training loop with the
 * library's gradients (pnp_mlp_loss_grad). */
int pnp_mlp_adam_step(pnp_ctx* c, const float* grad, const pnp_train_cfg* cfg);
/* Adam state: first and second moments host FP32 [PNP_MLP_PARAMS] each (packed order)
 * and the step count t.  Any pointer may be NULL. */
int pnp_mlp_get_adam_state(pnp_ctx* c, float* m, float* v, int64_t* t);

/* Allocation-free network forward (no counterpart in the paper; a service of this
 * library).  Same result as pnp_mlp_forward, but needs no context and never allocates
 * device memory: for callers that cannot call cudaMalloc -- e.g. a host application
 * that reserves its whole device-memory budget up front and forbids later allocations,
 * or code that must not introduce allocation (and its implicit synchronisation) into
 * a latency-critical stream.  The BF16 weights, activations and output rows live in one
 * fixed file-scope device array (about 5 MB) that every GPU loading the library keeps
 * until the process exits.
 *   params: device FP32 [PNP_MLP_PARAMS] packed parameters (layout above);
 *   X: device FP32 [B][216] standardised inputs; Y: device FP32 [B][3] outputs;
 *   B <= PNP_NOALLOC_MAX_ROWS (larger B: PNP_ERR_ARG, split the call);
 *   stream: cudaStream_t (NULL = legacy default stream); returns after the work is done.
 * The array is part of the library's device code: CUDA commits it on a device when it
 * loads that code there, which under lazy module loading (CUDA's default) can be the
 * first call of this or another network entry point on that device -- a caller with a
 * fixed device budget should count these 5 MB in it.  Later calls allocate nothing.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * for that device; make that first call before any stream capture.  All calls share the
 * array, so calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. */
#define PNP_NOALLOC_MAX_ROWS 4096
int pnp_mlp_forward_noalloc(const float* params, const float* X, int64_t B, float* Y, void* stream);

/* ---------------------------------------------------------------- profiling ------ */
/* Kernel classes timed with CUDA events recorded on the context's stream around each
 * launch while profiling is on. */
enum {
  PNP_PROF_RESIDUAL = 0,   /* FP64 residual element kernel */
  PNP_PROF_JV64 = 1,       /* FP64 J V element kernel */
  PNP_PROF_JV32 = 2,       /* FP32 J V element kernel */
  PNP_PROF_BLOCKDIAG = 3,  /* block-diagonal element kernel + 3x3 inversion */
  PNP_PROF_ORTHO = 4,      /* Gram-Schmidt projections: the multi-dot kernel */
  PNP_PROF_PRECOND = 5,    /* block-Jacobi apply (and FP32 conversion) */
  PNP_PROF_MLP = 6,        /* learned-start network kernels */
  PNP_PROF_ORTHO_UPDATE = 7, /* Gram-Schmidt update: the multi-axpy + norm kernel */
  PNP_PROF_INNER = 8,      /* FP32 Gram-Schmidt of the inner GMRES (flexible mode) */
  PNP_PROF_MG = 9,         /* multigrid: everything on the coarse levels of a V-cycle */
  PNP_PROF_NS = 10,        /* Navier-Stokes FP64-data element kernels (residual, FGMRES matrix
                              action, blocks) */
  PNP_PROF_NS32 = 11,      /* Navier-Stokes FP32 matrix action (V-cycle, BiCGStab) */
  PNP_PROF_NS_KRYLOV = 12, /* Navier-Stokes Krylov vector work (FGMRES Gram-Schmidt, BiCGStab),
                              block-Jacobi and finest-level smoothing kernels */
  PNP_PROF_KINDS = 13
};
/* on != 0: clear the accumulated times and start recording; on == 0: stop. */
int pnp_profile_enable(pnp_ctx* c, int on);
/* Accumulated device time (ms), number of timed regions, algorithmic HBM bytes (each
 * operand read once and each result written once, as the launches' sizes dictate)
 * and algorithmic floating-point operations (an FMA counts 2; the operation count of
 * the formulation the kernel evaluates, 0 where not tracked) of one class since
 * profiling was enabled; synchronises the stream.  Any output pointer may be NULL. */
int pnp_profile_read(pnp_ctx* c, int kind, double* total_ms, int64_t* count, double* alg_bytes,
                     double* alg_flops);
/* Kernels launched by this process through the library since it was loaded (a graph
 * replay counts the kernels it runs). */
int64_t pnp_kernel_launches(void);
/* Captures of the inner Krylov solve as a CUDA graph since the library was loaded (one
 * per change of its sizes, buffers or parameters; replays run while profiling is off). */
int64_t pnp_graph_captures(void);

#ifdef __cplusplus
}
#endif
#endif /* PNP_H */
