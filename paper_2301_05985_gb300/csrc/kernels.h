// kernels.h -- launch interfaces of the library's CUDA kernels.
#pragma once

#include "patches.h"
#include "pnp_internal.h"

// Arguments of the fused element kernels (residual / Jv / block diagonal).
template <typename T>
struct ElemArgs {
  int64_t n_elem;
  const int32_t* conn;     // [E][2^dim]
  const uint8_t* level;    // [E]
  const int32_t* hang_par; // [H][4]
  const uint8_t* hang_np;  // [H]
  const T* U;              // [N][3]
  const T* V;              // [N][3] direction (Jv only)
  const T* hs;             // [N][2] (beta1 c^k + beta2 c^{k-1}) / dt
  const T* adv;            // [N][3] advection velocity
  T* out;                  // [N][3] accumulated (must be zeroed first)
  PhysParams P;
  // FP32 lane kernel only (may be null): per node {c+, c-, phi, h+, h-, v0, v1, v2}, 32 B
  // aligned, the same values as U, hs and adv in one sector
  const float4* rec = nullptr;
  // FP32 J V only (may be null): direction and accumulated output padded to [N] float4,
  // read with one 16-byte load and added with one vector atomic per node
  const float4* V4 = nullptr;
  float4* out4 = nullptr;
};

// Arguments of the Dirichlet / hanging row kernels.
struct RowArgs {
  int64_t n_nodes, n_hanging;
  const uint8_t* faces;    // [N] boundary-face bits; bit 7 = hanging
  const int32_t* hnode;
  const int32_t* hpar;
  const uint8_t* hnp;
  BcTable bc;
};

// Counts every kernel the library launches (read by pnp_kernel_launches).
void note_launch();
// adds n launches (a replayed graph's kernels) and reads the counter
void note_launches(int64_t n);
int64_t launch_count();
// counts a capture of the inner solve (read by pnp_graph_captures)
void note_capture();

// Arguments of the shared-memory patch kernels (residual / Jv over Morton patches).
template <typename T>
struct PatchArgs {
  DevPatches pt;
  const uint8_t* level;    // [E]
  const uint8_t* faces;    // [N]
  BcTable bc;
  const T* U;              // [N][3]
  const T* V;              // [N][3] (Jv)
  const T* hs;             // [N][2]
  const T* adv;            // [N][3]
  T* out;                  // [N][3]: every non-hanging row written (no zeroing needed)
  T* partial;              // [n_partials][3]
  PhysParams P;
};
template <typename T>
cudaError_t launch_patch(int dim, bool jv, const PatchArgs<T>& A, cudaStream_t s);

template <typename T>
cudaError_t launch_element(int dim, bool jv, const ElemArgs<T>& A, cudaStream_t s);
// the same operator with 2^dim lanes per element (element_lanes.cu)
template <typename T>
cudaError_t launch_element_lanes(int dim, bool jv, const ElemArgs<T>& A, cudaStream_t s);
// floating-point operations per element (an FMA counts 2) of the element kernel that
// launch_element runs, counted from the formulation it evaluates
double element_kernel_flops(int dim, bool jv);
// the FP64 residual of the lane-group kernel evaluated in double-float arithmetic (pairs
// of floats, about 48 bits, on the FP32 pipe); FP64 inputs and output as launch_element
cudaError_t launch_residual_df(int dim, const ElemArgs<double>& A, cudaStream_t s);
// true when launch_element runs the lane-group kernel (not PNP_ELEMENT_KERNEL=thread)
bool element_kernel_is_lanes();
// true when the FP64 residual runs in double-float arithmetic (lane-group kernel, unless
// PNP_RESIDUAL_ARITH=f64 selects FP64 arithmetic)
bool residual_double_float();
// FP32 operations per FP64 operation of the double-float arithmetic: a sum costs 20, a
// product 10, a fused multiply-add (2 FP64 flops) 30, so 15 per flop for the FMA-dominated
// element formulation
constexpr double kDfFlopsPerFlop = 15.0;
// FP32 J V from a stored linearisation (element_lanes.cu): launch_lane_state computes, per
// element lane, the state's Gauss-point quantities J V needs (qp: rows * 2^dim * n_elem
// float4, A.rec set; rows = 4, or 3 when the advection field is zero); launch_jv_from_state
// applies J V with them (A.V or A.V4, A.out or A.out4; qp and A.conn 16-byte aligned).
// err[0] |= 1 when a staged copy's wait gave up.
cudaError_t launch_lane_state(int dim, const ElemArgs<float>& A, float4* qp, int rows, cudaStream_t s);
// polls: the limit of each bounded wait on a stage (< 0: the default, about a second)
cudaError_t launch_jv_from_state(int dim, const ElemArgs<float>& A, const float4* qp, int rows, int* err,
                                 int polls, cudaStream_t s);
double jv_from_state_flops(int dim);
// FP32 J V on hexahedra with two lanes per element (jv_pair.cu): the state from the node
// records (A.rec), the direction A.V4 (with A.out4) or A.V (with A.out); `advection`
// false when the advection field is zero (tau_c then depends on the level only)
cudaError_t launch_jv_pair(const ElemArgs<float>& A, bool advection, cudaStream_t s);
double jv_pair_flops(bool advection);
// Dout [N][9] += the 3x3 diagonal blocks of the Jacobian (lane-group kernel; Dout zeroed
// first, Dirichlet and hanging rows left to launch_diag_rows)
template <typename T>
cudaError_t launch_block_diag_lanes(int dim, const ElemArgs<T>& A, T* Dout, cudaStream_t s);
double block_diag_flops(int dim);
template <typename T>
cudaError_t launch_row_fixups(const RowArgs& R, const T* in, T* out, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_diag_rows(const RowArgs& R, T* Dg, cudaStream_t s);

// ------------------------------------------------------------------ vector kernels
// All reductions are deterministic: fixed grid, per-block partials, one final block.
constexpr int kRedBlocks = 608;  // 4 x 152 SMs
// persistent grid of the inner FP32 Gram-Schmidt kernels: 8 blocks of 256 per SM, enough
// loads in flight for a streaming kernel with few registers
constexpr int kInnerBlocks = 8 * 152;
constexpr int kRedThreads = 256;

// history h_s = (b1 c^k + b2 c^{k-1}) / dt, [N][2]
cudaError_t launch_history(int64_t N, const double* Uk, const double* Ukm1, double b1, double b2, double dt,
                           double* hs, cudaStream_t s);
// y[i] = (float) x[i]
cudaError_t launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t s);
// rec[i] = {U[i][0..2], hs[i][0..1], adv[i][0..2]} in FP32 (two float4 per node)
cudaError_t launch_node_records(int64_t N, const double* U, const double* hs, const double* adv, float4* rec,
                                cudaStream_t s);
cudaError_t launch_to_f64(int64_t n, const float* x, double* y, cudaStream_t s);
// y = a x + b y
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s);
// z = a x + b y
cudaError_t launch_axpbyz(int64_t n, double a, const double* x, double b, const double* y, double* z, cudaStream_t s);
// partial sums of x.y into part[kRedBlocks], then result[0] = sum (device)
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* part, double* result, cudaStream_t s);
cudaError_t launch_norm2(int64_t n, const double* x, double* part, double* result, cudaStream_t s);
// w -= sum_i h[i] Vb[i*ld + .], i < k ; optionally hacc[i] += h[i]
cudaError_t launch_multi_axpy(int64_t n, int k, const double* Vb, int64_t ld, const double* h, double* w,
                              double* hacc, cudaStream_t s);
// z_i = Dinv_i v_i per node (3x3 blocks); optionally also a float copy z32 (may be null)
cudaError_t launch_block_apply(int64_t N, const double* Dinv, const double* v, double scale, double* z, float* z32,
                               cudaStream_t s);
// blocks (= partial rows) of the multi-dot for vectors of n entries
int multi_dot_blocks(int64_t n);
// d[i] = V_i . w for i < k, plus d[k] = w . w when with_self (part: [multi_dot_blocks(n)][k+1])
cudaError_t launch_multi_dot_ext(int64_t n, int k, bool with_self, const double* Vb, int64_t ld, const double* w,
                                 double* part, double* d, cudaStream_t s);
// w -= sum_i d[i] dinv[i] V_i (i < k);  nrm2[0] = w . w afterwards
cudaError_t launch_multi_axpy_norm(int64_t n, int k, const double* Vb, int64_t ld, const double* d, const double* dinv,
                                   double* w, double* part, double* nrm2, cudaStream_t s);
// Dinv = inverse of the 3x3 blocks of D (Gauss-Jordan with partial pivoting, FP64);
// flag[0] |= 1 on a singular or non-finite block.  D may alias Dinv when T = double.
template <typename T>
cudaError_t launch_block_invert(int64_t N, const T* D, double* Dinv, int* flag, cudaStream_t s);
// hanging interpolation + Dirichlet values on U
cudaError_t launch_make_consistent(const RowArgs& R, double* U, cudaStream_t s);
// out[j] = sum_b part[b*k + j] for j < k (one block per output, fixed order)
cudaError_t launch_reduce_parts(int nparts, int k, const double* part, double* out, cudaStream_t s);

// ---------------------------------------------- inner FP32 GMRES (inner_krylov.cu)
int inner_dot_blocks(int64_t n);
int inner_max_depth();
// d_i = U_i . w (FP32 vectors, i < k); part: [inner_dot_blocks(n)][k].  n and ld are
// multiples of 4 and the vectors 16-byte aligned (rows padded with zeros)
cudaError_t launch_multi_dot_f32(int64_t n, int k, const float* Ub, int64_t ld, const float* w, double* part, double* d,
                                 cudaStream_t s);
// w -= sum_i d_i dinv_i U_i (i < k, FP32) and the per-block partials of w . w in part
// (summed by launch_inner_start / launch_inner_col); n, ld multiples of 4 as above
cudaError_t launch_multi_axpy_norm_f32(int64_t n, int k, const float* Ub, int64_t ld, const double* d,
                                       const double* dinv, float* w, double* part, cudaStream_t s);
// y = Dinv32 (inv_s[0] u) per node (inv_s may be null: scale 1); y4: the same, padded
cudaError_t launch_block_apply32(int64_t N, const float* Dinv32, const float* u, const float* inv_s, float* y,
                                 cudaStream_t s);
cudaError_t launch_block_apply32_pad(int64_t N, const float* Dinv32, const float* u, const float* inv_s, float4* y4,
                                     cudaStream_t s);
// out [N][3] <- acc4 with the Dirichlet rows set to V4 and the hanging rows to
// V4_h - sum_p w_p V4_p (the J V row fix-ups of the padded FP32 path)
cudaError_t launch_pack_jv4(const RowArgs& R, const float4* V4, const float4* acc4, float* out, cudaStream_t s);
// y4[i] = (x[3i], x[3i+1], x[3i+2], 0)
cudaError_t launch_pad4(int64_t N, const float* x, float4* y4, cudaStream_t s);
// inner Arnoldi bookkeeping; sc holds the rotated Hessenberg, the rotations, g and the
// number of columns before a breakdown: inner_scalar_doubles(d) doubles
inline size_t inner_scalar_doubles(int d) { return (size_t)(d + 1) * d + 2 * (size_t)d + (size_t)(d + 1) + 1; }
cudaError_t launch_inner_start(int d, const double* part, double* sv, double* dinv, float* inv_s, double* sc,
                               cudaStream_t s);
cudaError_t launch_inner_col(int j, int d, const double* dd, const double* part, double* sv, double* dinv, float* inv_s,
                             double* sc, cudaStream_t s);
cudaError_t launch_inner_lsq(int d, const double* sv, double* sc, double* coef, cudaStream_t s);
// out = sum_i coef_i U_i (FP32); x += sum_i coef_i Z_i (FP32 vectors into FP64)
cudaError_t launch_combine_f32(int64_t n, int k, const float* Ub, int64_t ld, const double* coef, float* out,
                               cudaStream_t s);
cudaError_t launch_combine_f32_add_f64(int64_t n, int k, const float* Zb, int64_t ld, const double* coef, double* x,
                                       cudaStream_t s);
// y = scale * x
cudaError_t launch_to_f64_scaled(int64_t n, const float* x, double scale, double* y, cudaStream_t s);
// out[s] = int_face n . (grad c_s + z_s c_s grad phi) dS (s = +, -) over boundary face
// `face` (boundary.cu); part: kRedBlocks x 2 partials; out: 2 device doubles
cudaError_t launch_element_gradient(int dim, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                    const int32_t* hpar, const uint8_t* hnp, const double* U, double* out,
                                    cudaStream_t s);
cudaError_t launch_boundary_flux(int dim, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                 const uint8_t* faces, const int32_t* hnode, const int32_t* hpar, const uint8_t* hnp,
                                 const double* U, int face, double* part, double* out, cudaStream_t s);
// out[f] = integral of field f over the plane x_ax = coord 2^-L (boundary.cu); anchor:
// element anchors [E][dim] on the device; part: kRedBlocks x 3 partials
cudaError_t launch_plane_integral(int dim, int L, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                  const int32_t* anchor, const int32_t* hnode, const int32_t* hpar, const uint8_t* hnp,
                                  const double* U, int ax, int64_t coord, double* part, double* out, cudaStream_t s);
// copy with layout change: [N][dim] <-> [N][3]
cudaError_t launch_vel_pack(int64_t N, int dim, const double* src, double* dst3, cudaStream_t s);
cudaError_t launch_vel_unpack(int64_t N, int dim, const double* src3, double* dst, cudaStream_t s);
