// ns.cu -- the semi-implicit VMS Navier-Stokes block of arXiv 2301.05985 and its solver.
//
// Rows (Def. 3 momentum and solenoidality, with the closure v^f = -tau_m R_m,
// p^f = -tau_sol R_sol of Sec. 3.1), linear in X = (v, p) at t^{k+1} because the
// advection v~ = 2 v^k - v^{k-1} (Eq. averaging1) is known:
//   momentum, test N_a e_i:
//     N_a R_m,i + grad N_a . grad v_i + (1/Sc) tau_m (v~ . grad N_a) R_m,i + d_i N_a tau_sol div v
//   solenoidality, test N_a:
//     N_a div v + tau_m grad N_a . R_m
//   R_m,i = (1/Sc)(beta0 v_i / dt + h_i + v~ . grad v_i) + d_i p + kappa/(2 Lambda^2) rho d_i phi
// (lap v = 0 for a Q1 field on an axis-aligned cube; h = (beta1 v^k + beta2 v^{k-1}) / dt;
// rho = c+ - c- and phi from the PNP state; the Galerkin terms other than the viscous one
// equal N_a R_m,i), tau_m = (4/dt^2 + (2/h)^2 |v~|^2 + C_I Sc^2 d (2/h)^4)^(-1/2) with
// 1/Re = Sc (the velocity scale D/L of Sec. 2.2), tau_sol = 1 / (d (2/h)^2 tau_m).  The
// solenoidality row takes +tau_m grad N_a . R_m, the sign that v^f = -tau_m R_m gives.
//
// Unknowns node-major [N][4] = (v_x, v_y, v_z, p); in 2D slot 2 is inactive (row X_2 = 0).
// Rows of hanging nodes are their constraints, Dirichlet rows X - g (per face and slot,
// the highest Dirichlet face containing the node wins) and, with ns_pin and no pressure
// Dirichlet face at that node, the pressure row of the node at the origin is X_3 = 0.
//
// Solver (App. A solves this block with BiCGStab): FP64 defect correction around FP32
// BiCGStab preconditioned by the inverted 4x4 nodal diagonal blocks.  Each refinement
// step evaluates F(X) = A X - b in FP64 (one kernel with the data terms), solves
// A d = -F(X) / ||F(X)|| in FP32 to ns_inner_rtol, and adds ||F|| d to X.  The BiCGStab
// scalars stay on the device (one small reduction kernel updates them); the host reads
// the residual norm every kCheck iterations.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "kernels.h"
#include "lane_ops.cuh"

#define CK(x)                                          \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) return ctx_check(c, e_, #x); \
  } while (0)
#define RC(x)                    \
  do {                           \
    int r_ = (x);                \
    if (r_ != PNP_OK) return r_; \
  } while (0)

namespace {

constexpr int kNsThreads = 256;
constexpr int kCheck = 8;          // BiCGStab iterations between host reads of ||r||
constexpr int kMaxRefine = 60;     // FP64 refinement steps per solve

template <typename T>
struct NsArgs {
  int64_t n_elem;
  const int32_t* conn;
  const uint8_t* level;
  const int32_t* hang_par;
  const uint8_t* hang_np;
  const T* X;          // [N][4] unknown / direction
  const T* adv;        // [N][4] v~ (slot 3 unused)
  const double* hv;    // [N][4] history (beta1 v^k + beta2 v^{k-1}) / dt (data kernel only)
  const double* U;     // [N][3] PNP state (c+, c-, phi) of the body force (data kernel only)
  T* out;              // [N][4] accumulated
  double isc, kap, tau_t, cid, fb;  // 1/Sc, beta0/dt, 4/dt^2, C_I Sc^2 d, kappa / (2 Lambda^2)
};

struct NsBc {
  uint8_t dir[4];      // per slot: bit f = Dirichlet on face f
  double val[6][4];
  int64_t pin;         // node whose pressure row is X_3 = 0 (-1: none)
  int dim;
};

// nodal values of a 4-slot field at node id (hanging: the parents' weighted sum)
template <typename T>
__device__ __forceinline__ void load4(const int32_t* __restrict__ hpar, const uint8_t* __restrict__ hnp,
                                      const T* __restrict__ src, int32_t id, bool valid, T (&d)[4]) {
#pragma unroll
  for (int f = 0; f < 4; ++f) d[f] = T(0);
  if (!valid) return;
  if (id >= 0) {
#pragma unroll
    for (int f = 0; f < 4; ++f) d[f] = __ldg(src + 4 * (int64_t)id + f);
  } else {
    const int32_t h = -id - 1;
    const int np = hnp[h];
    const T wgt = np == 2 ? T(0.5) : T(0.25);
    for (int p = 0; p < np; ++p) {
      const int64_t pid = hpar[4 * h + p];
#pragma unroll
      for (int f = 0; f < 4; ++f) d[f] += wgt * __ldg(src + 4 * pid + f);
    }
  }
}
__device__ __forceinline__ void load4(const int32_t* __restrict__ hpar, const uint8_t* __restrict__ hnp,
                                      const float* __restrict__ src, int32_t id, bool valid, float (&d)[4]) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    if (id >= 0) {
      v = __ldg(s4 + id);
    } else {
      const int32_t h = -id - 1;
      const int np = hnp[h];
      const float wgt = np == 2 ? 0.5f : 0.25f;
      for (int p = 0; p < np; ++p) {
        const float4 a = __ldg(s4 + hpar[4 * h + p]);
        v.x += wgt * a.x; v.y += wgt * a.y; v.z += wgt * a.z; v.w += wgt * a.w;
      }
    }
  }
  d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}

__device__ __forceinline__ void add4(double* out, int64_t id, const double (&r)[4], double wgt) {
#pragma unroll
  for (int f = 0; f < 4; ++f) atomicAdd(out + 4 * id + f, wgt * r[f]);
}
__device__ __forceinline__ void add4(float* out, int64_t id, const float (&r)[4], float wgt) {
  atomicAdd(reinterpret_cast<float4*>(out) + id, make_float4(wgt * r[0], wgt * r[1], wgt * r[2], wgt * r[3]));
}

template <typename T>
__device__ __forceinline__ void scatter_rows(const NsArgs<T>& A, int32_t id, const T (&r)[4]) {
  if (id >= 0) {
    add4(A.out, id, r, T(1));
  } else {
    const int32_t h = -id - 1;
    const int np = A.hang_np[h];
    const T wgt = np == 2 ? T(0.5) : T(0.25);
    for (int p = 0; p < np; ++p) add4(A.out, A.hang_par[4 * h + p], r, wgt);
  }
}

// physical constants in the kernel's arithmetic type
template <typename C>
struct NsK {
  C isc, kap, tau_t, cid, fb;  // 1/Sc, beta0/dt, 4/dt^2, C_I Sc^2 d, kappa / (2 Lambda^2)
};

// One lane per (element, corner): the lane's Gauss point is the one next to its corner.
// DATA adds the history and body-force terms (the residual F = A X - b); without them
// the kernel applies the matrix.  T: storage type of the vectors; C: arithmetic type (T,
// or double-float for FP64 data: GB300 runs FP64 at 1/64 of the FP32 rate).
template <typename T, typename C, int D, bool DATA>
__global__ void __launch_bounds__(kNsThreads) k_ns_lanes(NsArgs<T> A, NsK<C> K) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;  // shuffles need the whole warp
  const int64_t e = t / NC;
  const int c = (int)(t & (NC - 1));
  const bool valid = e < A.n_elem;
  const int32_t id = valid ? __ldg(A.conn + e * NC + c) : 0;
  const int lev = valid ? A.level[e] : 0;
  const C inv_h = pow2i(lev, C(0));
  const C w = pow2i(-D * (lev + 1), C(0));  // (h/2)^D
  const C nb = C(-0.5 * (1.0 - kG));
  C sh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[k] = ((c >> k) & 1) ? inv_h : -inv_h;
  const C G2 = pow2i(2 * lev + 2, C(0));        // (2/h)^2
  const C iG2d = pow2i(-2 * lev - 2, C(0)) * C(1.0 / D);  // 1 / (d (2/h)^2)

  T xs[4], as[4];
  load4(A.hang_par, A.hang_np, A.X, id, valid, xs);
  load4(A.hang_par, A.hang_np, A.adv, id, valid, as);
  C xn[4], an[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    xn[f] = to_compute<C>(xs[f]);
    an[f] = to_compute<C>(as[f]);
  }
  C v[3] = {C(0), C(0), C(0)}, gv[3][3], gp[3], va[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < D; ++i) interp_vg<C, D>(xn[i], nb, sh, v[i], gv[i]);
#pragma unroll
  for (int i = D; i < 3; ++i) gv[i][0] = gv[i][1] = gv[i][2] = C(0);
  interp_g<C, D>(xn[3], nb, sh, gp);
  C vv = C(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    va[i] = interp_v<C, D>(an[i], nb);
    vv = fma(va[i], va[i], vv);
  }
  const C arg = fma(K.cid * G2, G2, fma(G2, vv, K.tau_t));
  const C tau_m = inv_sqrt(arg);
  const C tau_s = (arg * tau_m) * iG2d;  // 1 / (tr(G) tau_m) = sqrt(arg) / (d (2/h)^2)
  C div = C(0);
#pragma unroll
  for (int i = 0; i < D; ++i) div += gv[i][i];
  C Rm[3] = {C(0), C(0), C(0)};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    C a = K.kap * v[i];
#pragma unroll
    for (int j = 0; j < D; ++j) a = fma(va[j], gv[i][j], a);
    Rm[i] = fma(K.isc, a, gp[i]);
  }
  if constexpr (DATA) {
    // history h_i and the body force kappa/(2 Lambda^2) (c+ - c-) grad phi of the PNP state
    double hs[4], u3[3] = {0.0, 0.0, 0.0};
    load4(A.hang_par, A.hang_np, A.hv, id, valid, hs);
    if (valid) {
      if (id >= 0) {
#pragma unroll
        for (int f = 0; f < 3; ++f) u3[f] = __ldg(A.U + 3 * (int64_t)id + f);
      } else {
        const int32_t h = -id - 1;
        const int np = A.hang_np[h];
        const double wgt = np == 2 ? 0.5 : 0.25;
        for (int p = 0; p < np; ++p) {
          const int64_t pid = A.hang_par[4 * h + p];
#pragma unroll
          for (int f = 0; f < 3; ++f) u3[f] += wgt * __ldg(A.U + 3 * pid + f);
        }
      }
    }
    const C rho = interp_v<C, D>(to_compute<C>(u3[0] - u3[1]), nb);
    C gphi[3];
    interp_g<C, D>(to_compute<C>(u3[2]), nb, sh, gphi);
    const C frho = K.fb * rho;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const C hq = interp_v<C, D>(to_compute<C>(hs[i]), nb);
      Rm[i] += fma(K.isc, hq, frho * gphi[i]);
    }
  }
  C r[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < D) {
      C Phi[3];
      const C su = K.isc * tau_m * Rm[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) Phi[j] = fma(su, va[j], gv[i][j]);
      Phi[i] = fma(tau_s, div, Phi[i]);
      r[i] = w * test_t<C, D>(Rm[i], Phi, nb, sh);
    } else {
      r[i] = C(0);
    }
  }
  {
    C Phi[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) Phi[j] = tau_m * Rm[j];
    r[3] = w * test_t<C, D>(div, Phi, nb, sh);
  }
  if (!valid) return;
  T ro[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) ro[f] = to_storage<T>(r[f]);
  scatter_rows(A, id, ro);
}

// Dirichlet / pin rows (mode 0: X - g, the residual; 1: X, the matrix) of free nodes.
template <typename T>
__global__ void k_ns_rows(int64_t N, const uint8_t* __restrict__ faces, NsBc bc, const T* __restrict__ X,
                          T* __restrict__ out, int mode) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint8_t fm = faces[i];
  if (fm & 0x80) return;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const unsigned msk = fm & bc.dir[f] & 0x3F;
    bool dir = msk != 0;
    double g = dir ? bc.val[31 - __clz(msk)][f] : 0.0;
    if (f == 2 && bc.dim == 2) { dir = true; g = 0.0; }
    if (f == 3 && !dir && i == bc.pin) dir = true;  // g = 0
    if (dir) out[4 * i + f] = mode == 0 ? T(double(X[4 * i + f]) - g) : X[4 * i + f];
  }
}

// constraint rows of hanging nodes: out_h = X_h - sum_p w_p X_p
template <typename T>
__global__ void k_ns_hanging_rows(int64_t H, const int32_t* __restrict__ hnode, const int32_t* __restrict__ hpar,
                                  const uint8_t* __restrict__ hnp, const T* __restrict__ X, T* __restrict__ out) {
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= H) return;
  const int np = hnp[h];
  const T wgt = np == 2 ? T(0.5) : T(0.25);
  const int64_t id = hnode[h];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T s = X[4 * id + f];
    for (int p = 0; p < np; ++p) s -= wgt * X[4 * (int64_t)hpar[4 * h + p] + f];
    out[4 * id + f] = s;
  }
}

// 4x4 diagonal block of the lane's own node: sum over the element's Gauss points q of
// the rows of test N_c against trial N_c (tau and v~ of q fetched from lane q); a
// hanging corner adds w_p^2 times it to each parent (its cross pairs are left out: the
// blocks only precondition).
template <int D>
__global__ void __launch_bounds__(kNsThreads) k_ns_diag(NsArgs<double> A, double* __restrict__ Dg) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;
  const int64_t e = t / NC;
  const int c = (int)(t & (NC - 1));
  const int lane = threadIdx.x & 31, gb = lane & ~(NC - 1);
  const bool valid = e < A.n_elem;
  const int32_t id = valid ? __ldg(A.conn + e * NC + c) : 0;
  const int lev = valid ? A.level[e] : 0;
  const double inv_h = pow2i(lev, 0.0);
  const double w = pow2i(-D * (lev + 1), 0.0);
  const double nb = -0.5 * (1.0 - kG);
  const double G2 = pow2i(2 * lev + 2, 0.0);
  double an[4];
  load4(A.hang_par, A.hang_np, A.adv, id, valid, an);
  double va[3] = {0.0, 0.0, 0.0}, vv = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    va[i] = interp_v<double, D>(an[i], nb);
    vv = fma(va[i], va[i], vv);
  }
  const double tm = inv_sqrt(fma(A.cid * G2, G2, fma(G2, vv, A.tau_t)));
  const double ts = 1.0 / (double(D) * G2 * tm);
  double B[4][4] = {};
#pragma unroll 1
  for (int q = 0; q < NC; ++q) {
    double vq[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) vq[j] = __shfl_sync(kFull, va[j], gb + q);
    const double tmq = __shfl_sync(kFull, tm, gb + q), tsq = __shfl_sync(kFull, ts, gb + q);
    double N, dN[3];
    shape_at<double, D>(c, q, inv_h, N, dN);
    double a = 0.0, dd = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      a = fma(vq[j], dN[j], a);
      dd = fma(dN[j], dN[j], dd);
    }
    const double Rv = A.isc * fma(A.kap, N, a);
    const double diag = N * Rv + dd + A.isc * tmq * a * Rv;
#pragma unroll
    for (int f = 0; f < D; ++f) {
#pragma unroll
      for (int g = 0; g < D; ++g) B[f][g] += tsq * dN[f] * dN[g] + (f == g ? diag : 0.0);
      B[f][3] += (N + A.isc * tmq * a) * dN[f];
      B[3][f] += (N + tmq * Rv) * dN[f];
    }
    B[3][3] += tmq * dd;
  }
  if (!valid) return;
  int32_t tg[4] = {id, -1, -1, -1};
  double wt = 1.0;
  int nt = 1;
  if (id < 0) {
    const int32_t h = -id - 1;
    nt = A.hang_np[h];
    wt = nt == 2 ? 0.5 : 0.25;
    for (int p = 0; p < nt; ++p) tg[p] = A.hang_par[4 * h + p];
  }
  for (int p = 0; p < nt; ++p)
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int g = 0; g < 4; ++g) atomicAdd(Dg + 16 * (int64_t)tg[p] + 4 * f + g, w * wt * wt * B[f][g]);
}

// identity rows of the blocks for Dirichlet / pin / inactive / hanging rows, then the
// inverse (Gauss-Jordan, partial pivoting) in FP32 for the preconditioner; a singular
// block (flag bit 2) is replaced by the identity
__global__ void k_ns_block_invert(int64_t N, const uint8_t* __restrict__ faces, NsBc bc, double* __restrict__ Dg,
                                  float* __restrict__ Dinv, int* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double a[4][8];
  const uint8_t fm = faces[i];
  for (int f = 0; f < 4; ++f) {
    bool unit = (fm & 0x80) != 0 || (fm & bc.dir[f] & 0x3F) != 0 || (f == 2 && bc.dim == 2);
    if (f == 3 && i == bc.pin && !(fm & bc.dir[3] & 0x3F)) unit = true;
    for (int g = 0; g < 4; ++g) {
      a[f][g] = unit ? (f == g ? 1.0 : 0.0) : Dg[16 * i + 4 * f + g];
      a[f][4 + g] = f == g ? 1.0 : 0.0;
    }
  }
  bool ok = true;
  for (int k = 0; k < 4 && ok; ++k) {
    int piv = k;
    for (int r = k + 1; r < 4; ++r)
      if (fabs(a[r][k]) > fabs(a[piv][k])) piv = r;
    if (!(fabs(a[piv][k]) > 0.0)) { ok = false; break; }
    if (piv != k)
      for (int g = 0; g < 8; ++g) { const double tmp = a[k][g]; a[k][g] = a[piv][g]; a[piv][g] = tmp; }
    const double inv = 1.0 / a[k][k];
    for (int g = 0; g < 8; ++g) a[k][g] *= inv;
    for (int r = 0; r < 4; ++r)
      if (r != k) {
        const double m = a[r][k];
        for (int g = 0; g < 8; ++g) a[r][g] -= m * a[k][g];
      }
  }
  if (!ok) atomicOr(flag, 4);
  for (int f = 0; f < 4; ++f)
    for (int g = 0; g < 4; ++g) Dinv[16 * i + 4 * f + g] = ok ? float(a[f][4 + g]) : (f == g ? 1.f : 0.f);
}

__global__ void k_ns_block_apply(int64_t N, const float* __restrict__ Dinv, const float4* __restrict__ x,
                                 float4* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 v = x[i];
  const float4* M = reinterpret_cast<const float4*>(Dinv) + 4 * i;
  const float4 m0 = M[0], m1 = M[1], m2 = M[2], m3 = M[3];
  y[i] = make_float4(m0.x * v.x + m0.y * v.y + m0.z * v.z + m0.w * v.w,
                     m1.x * v.x + m1.y * v.y + m1.z * v.z + m1.w * v.w,
                     m2.x * v.x + m2.y * v.y + m2.z * v.z + m2.w * v.w,
                     m3.x * v.x + m3.y * v.y + m3.z * v.z + m3.w * v.w);
}

// ------------------------------------------------------------------ BiCGStab pieces
// device scalars
enum { S_RHO = 0, S_ALPHA, S_OMEGA, S_BETA, S_RR, S_BREAK, S_ITS, kScalars = 8 };

__device__ __forceinline__ double dot4(float4 a, float4 b) {
  return (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z + (double)a.w * b.w;
}

// partials of <a0, b0> (and <a1, b1> when a1 is given) with FP64 accumulation
__global__ void __launch_bounds__(kRedThreads) k_dot4_part(int64_t n, const float4* __restrict__ a0,
                                                          const float4* __restrict__ b0,
                                                          const float4* __restrict__ a1,
                                                          const float4* __restrict__ b1, double* __restrict__ part) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double x0 = 0.0, x1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x0 += dot4(a0[i], b0[i]);
    if (a1) x1 += dot4(a1[i], b1[i]);
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0[0];
    part[gridDim.x + blockIdx.x] = s1[0];
  }
}

// sums the partials (fixed order) and updates the scalars of one BiCGStab stage:
// 0: rho' = <r^, r>, beta = (rho'/rho)(alpha/omega), rho = rho';  1: alpha = rho / <r^, v>;
// 2: omega = <t, s> / <t, t>;  3: rr = <r, r>.  A zero denominator sets S_BREAK.
__global__ void __launch_bounds__(kRedThreads) k_bicg_scalar(int stage, int nparts, const double* __restrict__ part,
                                                            double* __restrict__ sc) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double x0 = 0.0, x1 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    x0 += part[i];
    x1 += part[nparts + i];
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double a = s0[0], b = s1[0];
  if (stage == 0) {
    if (a == 0.0 || sc[S_OMEGA] == 0.0) {
      sc[S_BREAK] = 1.0;
      sc[S_BETA] = 0.0;
    } else {
      sc[S_BETA] = (a / sc[S_RHO]) * (sc[S_ALPHA] / sc[S_OMEGA]);
    }
    sc[S_RHO] = a;
  } else if (stage == 1) {
    if (a == 0.0) {
      sc[S_BREAK] = 1.0;
      sc[S_ALPHA] = 0.0;
    } else {
      sc[S_ALPHA] = sc[S_RHO] / a;
    }
  } else if (stage == 2) {
    sc[S_OMEGA] = b > 0.0 ? a / b : 0.0;
  } else {
    sc[S_RR] = a;
    sc[S_ITS] += 1.0;
  }
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(int64_t n, const float4* __restrict__ r, const float4* __restrict__ v, float4* __restrict__ p,
                         const double* __restrict__ sc) {
  const float b = (float)sc[S_BETA], om = (float)sc[S_OMEGA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = r[i], q = p[i], w = v[i];
    p[i] = make_float4(a.x + b * (q.x - om * w.x), a.y + b * (q.y - om * w.y), a.z + b * (q.z - om * w.z),
                       a.w + b * (q.w - om * w.w));
  }
}

// r -= alpha v  (r becomes s)
__global__ void k_bicg_s(int64_t n, float4* __restrict__ r, const float4* __restrict__ v,
                         const double* __restrict__ sc) {
  const float al = (float)sc[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = r[i], w = v[i];
    r[i] = make_float4(a.x - al * w.x, a.y - al * w.y, a.z - al * w.z, a.w - al * w.w);
  }
}

// x += alpha p^ + omega s^;  r -= omega t;  partials of <r, r>
__global__ void __launch_bounds__(kRedThreads) k_bicg_xr(int64_t n, float4* __restrict__ x,
                                                        const float4* __restrict__ ph, const float4* __restrict__ sh,
                                                        float4* __restrict__ r, const float4* __restrict__ t,
                                                        const double* __restrict__ sc, double* __restrict__ part) {
  __shared__ double s0[kRedThreads];
  const float al = (float)sc[S_ALPHA], om = (float)sc[S_OMEGA];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = x[i], p = ph[i], s = sh[i];
    x[i] = make_float4(a.x + al * p.x + om * s.x, a.y + al * p.y + om * s.y, a.z + al * p.z + om * s.z,
                       a.w + al * p.w + om * s.w);
    const float4 q = r[i], u = t[i];
    const float4 rn = make_float4(q.x - om * u.x, q.y - om * u.y, q.z - om * u.z, q.w - om * u.w);
    r[i] = rn;
    acc += dot4(rn, rn);
  }
  s0[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s0[threadIdx.x] += s0[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0[0];
    part[gridDim.x + blockIdx.x] = 0.0;
  }
}

// out = s * F (FP64 [N][4]) in FP32
__global__ void k_ns_to_f32(int64_t n4, const double* __restrict__ F, double s, float4* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n4) return;
  out[i] = make_float4((float)(s * F[4 * i]), (float)(s * F[4 * i + 1]), (float)(s * F[4 * i + 2]),
                       (float)(s * F[4 * i + 3]));
}

// X += s * x (FP32 correction into the FP64 unknown)
__global__ void k_ns_add_f32(int64_t n4, const float4* __restrict__ x, double s, double* __restrict__ X) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 a = x[i];
  X[4 * i] += s * a.x;
  X[4 * i + 1] += s * a.y;
  X[4 * i + 2] += s * a.z;
  X[4 * i + 3] += s * a.w;
}

// v~ = 2 v^k - v^{k-1} and h = (b1 v^k + b2 v^{k-1}) / dt, padded to 4 slots, and the FP32
// copy of v~; velocities node-major [N][3]
__global__ void k_ns_history(int64_t N, const double* __restrict__ vk, const double* __restrict__ vkm1, double b1,
                             double b2, double inv_dt, double* __restrict__ adv, double* __restrict__ hv,
                             float4* __restrict__ adv32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double a[3], h[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const double x = vk[3 * i + f], y = vkm1[3 * i + f];
    a[f] = 2.0 * x - y;
    h[f] = (b1 * x + b2 * y) * inv_dt;
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    adv[4 * i + f] = a[f];
    hv[4 * i + f] = h[f];
  }
  adv[4 * i + 3] = 0.0;
  hv[4 * i + 3] = 0.0;
  adv32[i] = make_float4((float)a[0], (float)a[1], (float)a[2], 0.f);
}

// x += sum_i coef_i Z_i: FP32 vectors and FP64 coefficients combined in FP64 (the terms of
// a flexible GMRES update can be large and cancel)
__global__ void k_ns_combine(int64_t n, int k, const float* __restrict__ Zb, int64_t ld,
                             const double* __restrict__ coef, double* __restrict__ x) {
  extern __shared__ double cfd[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cfd[i] = coef[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double v0 = 0.0, v1 = 0.0;
    int i = 0;
    for (; i + 2 <= k; i += 2) {
      v0 = fma(cfd[i], (double)Zb[(int64_t)i * ld + t], v0);
      v1 = fma(cfd[i + 1], (double)Zb[(int64_t)(i + 1) * ld + t], v1);
    }
    if (i < k) v0 = fma(cfd[i], (double)Zb[(int64_t)i * ld + t], v0);
    x[t] += v0 + v1;
  }
}

// v^{k+1} of X [N][4] into a node-major [N][3] velocity
__global__ void k_ns_velocity(int64_t N, const double* __restrict__ X, double* __restrict__ v3) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
#pragma unroll
  for (int f = 0; f < 3; ++f) v3[3 * i + f] = X[4 * i + f];
}

// ------------------------------------------------------------------ multigrid pieces
// Dirichlet / pin / inactive row of slot f at a free node (hanging nodes: faces bit 7)
__device__ __forceinline__ bool ns_dir(const NsBc& bc, uint8_t fm, int64_t i, int f) {
  if (f == 2 && bc.dim == 2) return true;
  const bool d = (fm & bc.dir[f] & 0x3F) != 0;
  return d || (f == 3 && i == bc.pin);
}

// x = omega D^-1 b (first sweep) or x += omega D^-1 (b - Ax), 4x4 blocks
__global__ void k_ns_smooth(int64_t N, const float* __restrict__ Dinv, const float4* __restrict__ b,
                            const float4* __restrict__ Ax, float4* __restrict__ x, float om, int first) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float4 r = b[i];
  if (!first) {
    const float4 a = Ax[i];
    r = make_float4(r.x - a.x, r.y - a.y, r.z - a.z, r.w - a.w);
  }
  const float4* M = reinterpret_cast<const float4*>(Dinv) + 4 * i;
  const float4 m0 = M[0], m1 = M[1], m2 = M[2], m3 = M[3];
  const float4 d = make_float4(om * (m0.x * r.x + m0.y * r.y + m0.z * r.z + m0.w * r.w),
                               om * (m1.x * r.x + m1.y * r.y + m1.z * r.z + m1.w * r.w),
                               om * (m2.x * r.x + m2.y * r.y + m2.z * r.z + m2.w * r.w),
                               om * (m3.x * r.x + m3.y * r.y + m3.z * r.z + m3.w * r.w));
  if (first) {
    x[i] = d;
  } else {
    const float4 o = x[i];
    x[i] = make_float4(o.x + d.x, o.y + d.y, o.z + d.z, o.w + d.w);
  }
}

// out[j] = sum_q w_q (b - Ax)[col_q] over the fine rows that are weak-form equations
// (Dirichlet, pin, inactive and hanging rows carry no element contributions); coarse
// constrained rows are zero
__global__ void k_ns_restrict(int64_t Nc, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              const float* __restrict__ w, const float4* __restrict__ b, const float4* __restrict__ Ax,
                              const uint8_t* __restrict__ faces_f, NsBc bcf, const uint8_t* __restrict__ faces_c,
                              NsBc bcc, float4* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= Nc) return;
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) {
    const int64_t i = col[q];
    const uint8_t ff = faces_f[i];
    if (ff & 0x80) continue;
    const float wq = w[q];
    const float4 bi = b[i], ai = Ax[i];
    const float r[4] = {bi.x - ai.x, bi.y - ai.y, bi.z - ai.z, bi.w - ai.w};
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (!ns_dir(bcf, ff, i, f)) s[f] = fmaf(wq, r[f], s[f]);
  }
  const uint8_t fc = faces_c[j];
  float o[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) o[f] = ((fc & 0x80) || ns_dir(bcc, fc, j, f)) ? 0.f : s[f];
  out[j] = make_float4(o[0], o[1], o[2], o[3]);
}

// x[i] += sum_q w_q xc[col_q] on the fine rows that are not constrained by a value
__global__ void k_ns_prolong_add(int64_t Nf, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const float* __restrict__ w, const float4* __restrict__ xc,
                                 const uint8_t* __restrict__ faces_f, NsBc bcf, float4* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Nf) return;
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) {
    const float4 a = xc[col[q]];
    const float wq = w[q];
    s[0] = fmaf(wq, a.x, s[0]); s[1] = fmaf(wq, a.y, s[1]); s[2] = fmaf(wq, a.z, s[2]); s[3] = fmaf(wq, a.w, s[3]);
  }
  const uint8_t ff = faces_f[i];
  float4 o = x[i];
  const bool h = (ff & 0x80) != 0;
  if (h || !ns_dir(bcf, ff, i, 0)) o.x += s[0];
  if (h || !ns_dir(bcf, ff, i, 1)) o.y += s[1];
  if (h || !ns_dir(bcf, ff, i, 2)) o.z += s[2];
  if (h || !ns_dir(bcf, ff, i, 3)) o.w += s[3];
  x[i] = o;
}

// coarse v~ (FP64 [Nc][4] and its FP32 copy) at the coarse nodes' points
__global__ void k_ns_inject_adv(int64_t Nc, const int32_t* __restrict__ map, const double* __restrict__ fine,
                                double* __restrict__ coarse, float4* __restrict__ coarse32) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= Nc) return;
  const int64_t i = map[j];
  double a[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    a[f] = fine[4 * i + f];
    coarse[4 * j + f] = a[f];
  }
  coarse32[j] = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
}

inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }
inline int gsb(int64_t n) { return (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (n + 255) / 256)); }

}  // namespace

// ------------------------------------------------------------------ state
struct NsState {
  double *X = nullptr, *F = nullptr, *adv = nullptr, *hv = nullptr, *Dg = nullptr;
  float4* adv32 = nullptr;
  float* Dinv = nullptr;
  float4 *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *t = nullptr, *ph = nullptr, *sh = nullptr,
         *x = nullptr;
  double *part = nullptr, *sc = nullptr, *hsc = nullptr;
  double* usave = nullptr;  // [2][3N] PNP history of repeated block iterations
  float4* mgAx = nullptr;   // [N] operator scratch of the finest multigrid level
  float4* xbest = nullptr;  // [N] BiCGStab's best iterate
  bool mg_off = false;      // this solve fell back from the V-cycle to the inverted blocks
  int64_t fine32 = 0;       // finest-level FP32 operator applications of this solve's V-cycles
  // FGMRES(m): unnormalised FP64 basis [(m+1)][4N], FP32 preconditioned vectors [m][4N], an
  // FP64 scratch vector, reduction partials and device scalars
  double *Q = nullptr, *z64 = nullptr, *fpart = nullptr, *fsc = nullptr, *fsc2 = nullptr;
  float* Z = nullptr;
  int fg_m = 0;
  int64_t pin = -1;
  std::vector<void*> alloc;
};

void ctx_ns_release(pnp_ctx* c) {
  if (!c->ns) return;
  for (void* p : c->ns->alloc) cudaFree(p);
  if (c->ns->hsc) cudaFreeHost(c->ns->hsc);
  delete c->ns;
  c->ns = nullptr;
}

int ctx_ns_alloc(pnp_ctx* c) {
  if (c->ns) return PNP_OK;
  NsState* S = new NsState();
  c->ns = S;
  const int64_t N = c->n_nodes;
  auto get = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    S->alloc.push_back(*p);
    return true;
  };
  const size_t d4 = sizeof(double) * 4 * N, f4 = sizeof(float4) * N;
  bool ok = get((void**)&S->X, d4) && get((void**)&S->F, d4) && get((void**)&S->adv, d4) && get((void**)&S->hv, d4) &&
            get((void**)&S->Dg, sizeof(double) * 16 * N) &&
            get((void**)&S->adv32, f4) && get((void**)&S->Dinv, sizeof(float) * 16 * N) && get((void**)&S->r, f4) &&
            get((void**)&S->rh, f4) && get((void**)&S->p, f4) && get((void**)&S->v, f4) && get((void**)&S->t, f4) &&
            get((void**)&S->ph, f4) && get((void**)&S->sh, f4) && get((void**)&S->x, f4) &&
            get((void**)&S->part, sizeof(double) * 2 * kRedBlocks) && get((void**)&S->sc, sizeof(double) * kScalars);
  // pinned host scalars: the BiCGStab scalars, or FGMRES projections (m <= 200)
  if (ok) ok = cudaMallocHost((void**)&S->hsc, sizeof(double) * 256) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ctx_ns_release(c);
    PNP_FAIL(PNP_ERR_NOMEM, "ns: device allocation failed");
  }
  if (cudaMemsetAsync(S->X, 0, d4, c->stream) != cudaSuccess) return ctx_check(c, cudaGetLastError(), "ns memset");
  // the node at the origin carries the pressure pin
  const auto& m = c->host_mesh;
  for (int64_t i = 0; i < N && S->pin < 0; ++i) {
    bool o = m.node_hang[i] < 0;
    for (int k = 0; k < m.dim && o; ++k) o = m.node_ijk[(size_t)i * m.dim + k] == 0;
    if (o) S->pin = i;
  }
  return PNP_OK;
}

double* ctx_ns_field(pnp_ctx* c) { return c->ns ? c->ns->X : nullptr; }

double* ctx_ns_history_save(pnp_ctx* c) {
  if (!c->ns) return nullptr;
  if (!c->ns->usave) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * 6 * c->n_nodes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    c->ns->usave = (double*)p;
    c->ns->alloc.push_back(p);
  }
  return c->ns->usave;
}

static NsBc ns_bc(const pnp_ctx* c) {
  NsBc b{};
  for (int f = 0; f < 4; ++f) {
    uint8_t m = 0;
    for (int face = 0; face < 2 * c->dim; ++face)
      if (c->ns_bc_type[face][f] == PNP_DIRICHLET) m |= (uint8_t)(1u << face);
    b.dir[f] = m;
  }
  for (int face = 0; face < 6; ++face)
    for (int f = 0; f < 4; ++f) b.val[face][f] = c->ns_bc_val[face][f];
  b.pin = c->prm.ns_pin ? c->ns->pin : -1;
  b.dim = c->dim;
  return b;
}

template <typename T>
static NsArgs<T> ns_args(const pnp_ctx* c, const T* X, const T* adv, T* out) {
  const pnp_params& p = c->prm;
  NsArgs<T> A{};
  A.n_elem = c->n_elem;
  A.conn = c->d_conn;
  A.level = c->d_level;
  A.hang_par = c->d_hpar;
  A.hang_np = c->d_hnp;
  A.X = X;
  A.adv = adv;
  A.out = out;
  A.isc = 1.0 / p.ns_Sc;
  A.kap = p.steady ? 0.0 : p.beta0 / p.dt;
  A.tau_t = p.steady ? 0.0 : 4.0 / (p.dt * p.dt);
  A.cid = p.C_I * p.ns_Sc * p.ns_Sc * c->dim;
  A.fb = p.ns_kappa / (2.0 * p.eps * p.eps);
  return A;
}

template <typename C, typename T>
static NsK<C> ns_k(const NsArgs<T>& A) {
  return NsK<C>{C(A.isc), C(A.kap), C(A.tau_t), C(A.cid), C(A.fb)};
}

// the FP64 rows in double-float arithmetic (default) or FP64 arithmetic
template <int D, bool DATA>
static void launch_ns64(const NsArgs<double>& A, int blocks, cudaStream_t s) {
  if (residual_double_float()) k_ns_lanes<double, df, D, DATA><<<blocks, kNsThreads, 0, s>>>(A, ns_k<df>(A));
  else k_ns_lanes<double, double, D, DATA><<<blocks, kNsThreads, 0, s>>>(A, ns_k<double>(A));
}

// element-kernel flops per lane (FP counts of the code above, fma = 2)
static double ns_lane_flops(int D, bool data) {
  const double tri = D * (D - 1) / 2.0;
  const double vg = 3 * tri + 4 * D, v = 3 * D, g = vg - 2, tt = 6 * D + 3 * tri + 1;
  double f = D * vg + g + D * v + 2 * D + 12 + D * (2 + 2 * D + 2) + (D + 1) * (3 + 2 * D + tt) + 8;
  if (data) f += 4 * v + g + 8 * D;
  return f;
}

// ||x||_2 of a [N][4] FP64 vector
static int ctx_norm4(pnp_ctx* c, const double* x, double* out) {
  double* slot = c->dsc + 4 * (c->m_alloc + 2) + 8;
  CK(launch_norm2(4 * c->n_nodes, x, c->part, slot, c->stream));
  CK(cudaMemcpyAsync(c->hpin, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = c->hpin[0];
  return PNP_OK;
}

// ------------------------------------------------------------------ operators
int ctx_ns_prepare(pnp_ctx* c) {
  RC(ctx_ns_alloc(c));
  NsState* S = c->ns;
  const pnp_params& p = c->prm;
  const int64_t N = c->n_nodes;
  const double inv_dt = p.steady ? 0.0 : 1.0 / p.dt;
  k_ns_history<<<nblk(N, 256), 256, 0, c->stream>>>(N, c->vel, c->vel_prev, p.beta1, p.beta2, inv_dt, S->adv, S->hv,
                                                     S->adv32);
  note_launch();
  CK(cudaGetLastError());
  return PNP_OK;
}

// F = the NS rows of X (data = true: the residual A X - b, Ubody the PNP state of the body
// force; false: A X), FP64
int ctx_ns_apply64(pnp_ctx* c, const double* X, const double* Ubody, double* F, bool data) {
  NsState* S = c->ns;
  const int64_t N = c->n_nodes;
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(F, 0, sizeof(double) * 4 * N, s));
  NsArgs<double> A = ns_args<double>(c, X, S->adv, F);
  A.hv = S->hv;
  A.U = Ubody;
  const int64_t lanes = c->n_elem << c->dim;
  {
    // flops: the FP64 formulation's, times 15 FP32 operations per double-float operation
    ProfScope ps(c, PNP_PROF_NS, 72.0 * N + (data ? 56.0 * N : 0.0) + 32.0 * N + c->conn_bytes(),
                 ns_lane_flops(c->dim, data) * lanes * (residual_double_float() ? 15.0 : 1.0));
    if (c->n_elem) {
      const int blocks = nblk(lanes, kNsThreads);
      if (c->dim == 2) {
        if (data) launch_ns64<2, true>(A, blocks, s);
        else launch_ns64<2, false>(A, blocks, s);
      } else {
        if (data) launch_ns64<3, true>(A, blocks, s);
        else launch_ns64<3, false>(A, blocks, s);
      }
      note_launch();
    }
  }
  const NsBc bc = ns_bc(c);
  k_ns_rows<double><<<nblk(N, 256), 256, 0, s>>>(N, c->d_faces, bc, X, F, data ? 0 : 1);
  note_launch();
  if (c->n_hanging) {
    k_ns_hanging_rows<double><<<nblk(c->n_hanging, 256), 256, 0, s>>>(c->n_hanging, c->d_hnode, c->d_hpar, c->d_hnp,
                                                                     X, F);
    note_launch();
  }
  CK(cudaGetLastError());
  return PNP_OK;
}

// y = A x, FP32 (x, y padded [N] float4)
int ctx_ns_apply32(pnp_ctx* c, const float4* x, float4* y) {
  NsState* S = c->ns;
  const int64_t N = c->n_nodes;
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(y, 0, sizeof(float4) * N, s));
  NsArgs<float> A = ns_args<float>(c, reinterpret_cast<const float*>(x), reinterpret_cast<const float*>(S->adv32),
                                   reinterpret_cast<float*>(y));
  const int64_t lanes = c->n_elem << c->dim;
  {
    ProfScope ps(c, PNP_PROF_NS32, 48.0 * N + c->conn_bytes(), ns_lane_flops(c->dim, false) * lanes);
    if (c->n_elem) {
      const int blocks = nblk(lanes, kNsThreads);
      if (c->dim == 2) k_ns_lanes<float, float, 2, false><<<blocks, kNsThreads, 0, s>>>(A, ns_k<float>(A));
      else k_ns_lanes<float, float, 3, false><<<blocks, kNsThreads, 0, s>>>(A, ns_k<float>(A));
      note_launch();
    }
  }
  const NsBc bc = ns_bc(c);
  const float* xf = reinterpret_cast<const float*>(x);
  float* yf = reinterpret_cast<float*>(y);
  k_ns_rows<float><<<nblk(N, 256), 256, 0, s>>>(N, c->d_faces, bc, xf, yf, 1);
  note_launch();
  if (c->n_hanging) {
    k_ns_hanging_rows<float><<<nblk(c->n_hanging, 256), 256, 0, s>>>(c->n_hanging, c->d_hnode, c->d_hpar, c->d_hnp,
                                                                    xf, yf);
    note_launch();
  }
  CK(cudaGetLastError());
  return PNP_OK;
}

// the 4x4 diagonal blocks [N][16] (FP64, before the row substitutions) into Dg
int ctx_ns_block_diag(pnp_ctx* c, double* Dg) {
  NsState* S = c->ns;
  const int64_t N = c->n_nodes;
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(Dg, 0, sizeof(double) * 16 * N, s));
  NsArgs<double> A = ns_args<double>(c, nullptr, S->adv, nullptr);
  const int64_t lanes = c->n_elem << c->dim;
  ProfScope ps(c, PNP_PROF_NS, 32.0 * N + 128.0 * N + c->conn_bytes());
  if (c->n_elem) {
    if (c->dim == 2) k_ns_diag<2><<<nblk(lanes, kNsThreads), kNsThreads, 0, s>>>(A, Dg);
    else k_ns_diag<3><<<nblk(lanes, kNsThreads), kNsThreads, 0, s>>>(A, Dg);
    note_launch();
  }
  CK(cudaGetLastError());
  return PNP_OK;
}

// the inverted blocks of the preconditioner, with the identity on constrained rows
int ctx_ns_blocks_row_fix(pnp_ctx* c, double* Dg, float* Dinv) {
  const int64_t N = c->n_nodes;
  CK(cudaMemsetAsync(c->dflag + 3, 0, sizeof(int), c->stream));
  k_ns_block_invert<<<nblk(N, 128), 128, 0, c->stream>>>(N, c->d_faces, ns_bc(c), Dg, Dinv, c->dflag + 3);
  note_launch();
  CK(cudaGetLastError());
  return PNP_OK;
}

// ------------------------------------------------------------------ multigrid
static int ns_mg_levels(const pnp_ctx* c) { return c->prm.mg_levels > 0 ? c->prm.mg_levels : c->prm.ns_mg_levels; }

// Per solve: every coarse level's parameters, boundary table, injected v~ and inverted
// diagonal blocks (level 0 uses the solve's own blocks).
static int ctx_ns_mg_prepare(pnp_ctx* c) {
  RC(ctx_mg_setup(c, ns_mg_levels(c)));
  NsState* S = c->ns;
  if (!S->mgAx) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(float4) * c->n_nodes) != cudaSuccess) {
      cudaGetLastError();
      PNP_FAIL(PNP_ERR_NOMEM, "ns multigrid: device allocation failed");
    }
    S->mgAx = (float4*)q;
    S->alloc.push_back(q);
  }
  auto& lv = *c->mg;
  pnp_ctx* fine = c;
  for (size_t l = 1; l < lv.size(); ++l) {
    pnp_ctx* sc = lv[l].sub;
    pnp_params& q = sc->prm;
    const pnp_params& p = c->prm;
    q.eps = p.eps;
    q.dt = p.dt;
    q.C_I = p.C_I;
    q.beta0 = p.beta0;
    q.beta1 = p.beta1;
    q.beta2 = p.beta2;
    q.steady = p.steady;
    q.ns_Sc = p.ns_Sc;
    q.ns_kappa = p.ns_kappa;
    q.ns_pin = p.ns_pin;
    std::memcpy(sc->ns_bc_type, c->ns_bc_type, sizeof(c->ns_bc_type));
    std::memcpy(sc->ns_bc_val, c->ns_bc_val, sizeof(c->ns_bc_val));
    RC(ctx_ns_alloc(sc));
    const int64_t Nc = sc->n_nodes;
    k_ns_inject_adv<<<nblk(Nc, 256), 256, 0, c->stream>>>(Nc, lv[l].inject, fine->ns->adv, sc->ns->adv,
                                                          sc->ns->adv32);
    note_launch();
    CK(cudaGetLastError());
    RC(ctx_ns_block_diag(sc, sc->ns->Dg));
    RC(ctx_ns_blocks_row_fix(sc, sc->ns->Dg, sc->ns->Dinv));
    fine = sc;
  }
  return PNP_OK;
}

// x = one V-cycle on level l applied to b (level 0: the caller's vectors; coarser levels:
// their contexts' r and x)
static int ns_mg_cycle(pnp_ctx* c, size_t l, const float4* b, float4* x) {
  auto& lv = *c->mg;
  pnp_ctx* lc = l == 0 ? c : lv[l].sub;
  NsState* LS = lc->ns;
  float4* Ax = l == 0 ? c->ns->mgAx : LS->t;
  const int64_t N = lc->n_nodes;
  cudaStream_t s = c->stream;
  const float om = (float)c->prm.mg_omega;
  const NsBc bc = ns_bc(lc);
  auto apply = [&]() -> int {
    RC(ctx_ns_apply32(lc, x, Ax));
    if (l == 0) c->ns->fine32++;
    return PNP_OK;
  };
  auto smooth = [&](bool first) -> int {
    if (!first) RC(apply());
    ProfScope ps(c, l == 0 ? PNP_PROF_NS_KRYLOV : -1, 112.0 * N, 36.0 * N);
    k_ns_smooth<<<nblk(N, 256), 256, 0, s>>>(N, LS->Dinv, b, Ax, x, om, first ? 1 : 0);
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
  RC(apply());
  pnp_ctx* cc = lv[l + 1].sub;
  const MgLevel& C = lv[l + 1];
  {
    ProfScope ps(c, l == 0 ? PNP_PROF_MG : -1, 0.0);
    k_ns_restrict<<<nblk(cc->n_nodes, 256), 256, 0, s>>>(cc->n_nodes, C.r_ptr, C.r_col, C.r_w, b, Ax, lc->d_faces, bc,
                                                         cc->d_faces, ns_bc(cc), cc->ns->r);
    note_launch();
    CK(cudaGetLastError());
    RC(ns_mg_cycle(c, l + 1, cc->ns->r, cc->ns->x));
    k_ns_prolong_add<<<nblk(N, 256), 256, 0, s>>>(N, C.p_ptr, C.p_col, C.p_w, cc->ns->x, lc->d_faces, bc, x);
    note_launch();
    CK(cudaGetLastError());
  }
  for (int k = 0; k < nu; ++k) RC(smooth(false));
  return PNP_OK;
}

// out = M^-1 in: the inverted blocks, or one V-cycle
static int ns_precond(pnp_ctx* c, const float4* in, float4* out) {
  NsState* S = c->ns;
  const int64_t N = c->n_nodes;
  if (ns_mg_levels(c) > 0 && !S->mg_off && c->mg && c->mg->size() > 1) return ns_mg_cycle(c, 0, in, out);
  ProfScope ps(c, PNP_PROF_NS_KRYLOV, 96.0 * N, 32.0 * N);
  k_ns_block_apply<<<nblk(N, 256), 256, 0, c->stream>>>(N, S->Dinv, in, out);
  note_launch();
  CK(cudaGetLastError());
  return PNP_OK;
}

// FP32 BiCGStab on A d = r (r = S->r on entry, d = S->x), right preconditioned by the
// inverted blocks, to ||r|| <= rtol ||r_0|| or `max_it` iterations; returns the iterations
static int ns_bicgstab32(pnp_ctx* c, double rtol, int max_it, int* its_out) {
  NsState* S = c->ns;
  const int64_t N = c->n_nodes;
  cudaStream_t s = c->stream;
  const size_t f4 = sizeof(float4) * N;
  const int G = gsb(N);
  CK(cudaMemsetAsync(S->x, 0, f4, s));
  CK(cudaMemsetAsync(S->p, 0, f4, s));
  CK(cudaMemsetAsync(S->v, 0, f4, s));
  CK(cudaMemcpyAsync(S->rh, S->r, f4, cudaMemcpyDeviceToDevice, s));
  const double init[kScalars] = {1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  std::memcpy(S->hsc, init, sizeof(init));
  CK(cudaMemcpyAsync(S->sc, S->hsc, sizeof(init), cudaMemcpyHostToDevice, s));
  // ||r_0||^2
  k_dot4_part<<<G, kRedThreads, 0, s>>>(N, S->r, S->r, nullptr, nullptr, S->part);
  k_bicg_scalar<<<1, kRedThreads, 0, s>>>(3, G, S->part, S->sc);
  note_launches(2);
  CK(cudaMemcpyAsync(S->hsc, S->sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double rr0 = S->hsc[S_RR];
  int its = 0;
  // the iterate with the smallest recursive residual seen at a check is the result (BiCGStab
  // can diverge late; the zero start is the first candidate)
  if (!S->xbest) {
    void* q = nullptr;
    if (cudaMalloc(&q, f4) != cudaSuccess) {
      cudaGetLastError();
      PNP_FAIL(PNP_ERR_NOMEM, "ns: device allocation failed");
    }
    S->xbest = (float4*)q;
    S->alloc.push_back(q);
  }
  double best = rr0;
  bool x_is_best = true;  // S->x (zero) is the best so far
  *its_out = 0;
  if (!(rr0 > 0.0)) return PNP_OK;
  const double tol2 = rtol * rtol * rr0;
  while (its < max_it) {
    const int batch = std::min(kCheck, max_it - its);
    for (int b = 0; b < batch; ++b) {
      {
        // <r^, r>, p = r + beta (p - omega v)
        ProfScope ps(c, PNP_PROF_NS_KRYLOV, 96.0 * N, 16.0 * N);
        k_dot4_part<<<G, kRedThreads, 0, s>>>(N, S->rh, S->r, nullptr, nullptr, S->part);
        k_bicg_scalar<<<1, kRedThreads, 0, s>>>(0, G, S->part, S->sc);
        k_bicg_p<<<G, 256, 0, s>>>(N, S->r, S->v, S->p, S->sc);
        note_launches(3);
      }
      RC(ns_precond(c, S->p, S->ph));  // p^ = M^-1 p
      RC(ctx_ns_apply32(c, S->ph, S->v));
      {
        // alpha = rho / <r^, v>, s = r - alpha v
        ProfScope ps(c, PNP_PROF_NS_KRYLOV, 80.0 * N, 16.0 * N);
        k_dot4_part<<<G, kRedThreads, 0, s>>>(N, S->rh, S->v, nullptr, nullptr, S->part);
        k_bicg_scalar<<<1, kRedThreads, 0, s>>>(1, G, S->part, S->sc);
        k_bicg_s<<<G, 256, 0, s>>>(N, S->r, S->v, S->sc);
        note_launches(3);
      }
      RC(ns_precond(c, S->r, S->sh));  // s^ = M^-1 s
      RC(ctx_ns_apply32(c, S->sh, S->t));
      {
        // omega = <t, s> / <t, t>, x += alpha p^ + omega s^, r = s - omega t, <r, r>
        ProfScope ps(c, PNP_PROF_NS_KRYLOV, 144.0 * N, 40.0 * N);
        k_dot4_part<<<G, kRedThreads, 0, s>>>(N, S->t, S->r, S->t, S->t, S->part);
        k_bicg_scalar<<<1, kRedThreads, 0, s>>>(2, G, S->part, S->sc);
        k_bicg_xr<<<G, kRedThreads, 0, s>>>(N, S->x, S->ph, S->sh, S->r, S->t, S->sc, S->part);
        k_bicg_scalar<<<1, kRedThreads, 0, s>>>(3, G, S->part, S->sc);
        note_launches(4);
      }
      CK(cudaGetLastError());
    }
    its += batch;
    CK(cudaMemcpyAsync(S->hsc, S->sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double rr = S->hsc[S_RR];
    if (std::isfinite(rr) && rr < best) {
      best = rr;
      x_is_best = true;
      if (rr > tol2) CK(cudaMemcpyAsync(S->xbest, S->x, f4, cudaMemcpyDeviceToDevice, s));
    } else {
      x_is_best = false;
    }
    if (!std::isfinite(rr) || rr <= tol2 || S->hsc[S_BREAK] != 0.0) break;
  }
  if (!x_is_best) {
    if (best < rr0) CK(cudaMemcpyAsync(S->x, S->xbest, f4, cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemsetAsync(S->x, 0, f4, s));
  }
  *its_out = its;
  return PNP_OK;
}

// FGMRES(m) in FP64 on A d = -F(X), right-preconditioned in FP32 (the V-cycle or the
// inverted blocks), restarted until ||F(X)|| <= target.  The preconditioned vectors are
// kept (FP32) so the flexible relation A Z = Q H holds in FP64; the basis is unnormalised
// with its scales on the host (as the PNP solver's outer GMRES).
static int ns_alloc_fgmres(pnp_ctx* c, int m) {
  NsState* S = c->ns;
  if (S->fg_m == m && S->Q) return PNP_OK;
  const int64_t n = 4 * c->n_nodes;
  auto get = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    S->alloc.push_back(*p);
    return true;
  };
  // earlier (smaller) buffers stay in the allocation list until the context is destroyed
  const bool ok = get((void**)&S->Q, sizeof(double) * (size_t)(m + 1) * n) &&
                  get((void**)&S->Z, sizeof(float) * (size_t)m * n) && get((void**)&S->z64, sizeof(double) * n) &&
                  // partials: the multi-dot's blocks x (m + 2), and the update-and-norm kernel's
                  // kRedBlocks (whichever is larger)
                  get((void**)&S->fpart, sizeof(double) *
                                             std::max<size_t>((size_t)kRedBlocks, (size_t)multi_dot_blocks(n)) *
                                             (size_t)(m + 2)) &&
                  get((void**)&S->fsc, sizeof(double) * (size_t)(3 * (m + 2) + 4)) &&
                  get((void**)&S->fsc2, sizeof(double) * (size_t)(m + 2));
  if (!ok) {
    cudaGetLastError();
    S->Q = nullptr;
    PNP_FAIL(PNP_ERR_NOMEM, "ns: no device memory for FGMRES(%d)", m);
  }
  S->fg_m = m;
  return PNP_OK;
}

static int ns_fgmres(pnp_ctx* c, const double* Ubody, double target, double& f, pnp_ns_stats* st) {
  NsState* S = c->ns;
  const pnp_params& p = c->prm;
  const int m = p.ns_fgmres;
  RC(ns_alloc_fgmres(c, m));
  const int64_t N = c->n_nodes, n = 4 * N;
  cudaStream_t s = c->stream;
  double* dd = S->fsc;               // [m+2] projections
  double* dinv = dd + (m + 2);       // [m+2] 1 / s_i^2
  double* dcoef = dinv + (m + 2);    // [m+2] combination coefficients
  double* dnrm = dcoef + (m + 2);    // w . w after the pass
  double* dd2 = S->fsc2;             // [m+2] projections of the second pass
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), sv(m + 1), hp(m + 2);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int total = 0, cycles = 0;
  double f_prev = f;
  int stalls = 0;
  while (f > target) {
    if (total >= p.ns_max_it) {
      pnp_set_error("ns: FGMRES %d iterations, ||F|| = %.3e > %.3e", total, f, target);
      return PNP_ERR_KRYLOV_MAXIT;
    }
    // u_0 = -F, s_0 = ||F||
    CK(launch_axpbyz(n, -1.0, S->F, 0.0, S->F, S->Q, s));
    sv[0] = f;
    hp[0] = 1.0 / (f * f);
    CK(cudaMemcpyAsync(dinv, hp.data(), sizeof(double), cudaMemcpyHostToDevice, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = f;
    int k = 0;
    for (int j = 0; j < m && total < p.ns_max_it; ++j) {
      double* uj = S->Q + (size_t)j * n;
      double* w = S->Q + (size_t)(j + 1) * n;
      float4* zj = reinterpret_cast<float4*>(S->Z + (size_t)j * n);
      // z_j = M^-1 (u_j / s_j) in FP32; w = A z_j in FP64
      k_ns_to_f32<<<nblk(N, 256), 256, 0, s>>>(N, uj, 1.0 / sv[j], S->r);
      note_launch();
      RC(ns_precond(c, S->r, zj));
      CK(launch_to_f64_scaled(n, reinterpret_cast<const float*>(zj), 1.0, S->z64, s));
      RC(ctx_ns_apply64(c, S->z64, nullptr, w, false));
      st->matvecs64++;
      {
        // classical Gram-Schmidt, two passes (the pressure and velocity scales differ by
        // orders of magnitude: one pass loses orthogonality and the Arnoldi estimate with it)
        const double nj = (double)n * (j + 1);
        ProfScope ps(c, PNP_PROF_NS_KRYLOV, 16.0 * (2.0 * nj + 3.0 * n), 8.0 * nj);
        CK(launch_multi_dot_ext(n, j + 1, false, S->Q, n, w, S->fpart, dd, s));
        CK(launch_multi_axpy_norm(n, j + 1, S->Q, n, dd, dinv, w, S->fpart, dnrm, s));
        CK(launch_multi_dot_ext(n, j + 1, false, S->Q, n, w, S->fpart, dd2, s));
        CK(launch_multi_axpy_norm(n, j + 1, S->Q, n, dd2, dinv, w, S->fpart, dnrm, s));
      }
      CK(cudaMemcpyAsync(S->hsc, dd, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(S->hsc + (m + 2), dd2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(S->hsc + (m + 1), dnrm, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) Hij(i, j) = (S->hsc[i] + S->hsc[m + 2 + i]) / sv[i];
      const double nrm = std::sqrt(S->hsc[m + 1]);
      if (!std::isfinite(nrm)) PNP_FAIL(PNP_ERR_NAN, "ns: FGMRES vector norm is not finite");
      sv[j + 1] = nrm;
      Hij(j + 1, j) = nrm;
      if (nrm > 0) {
        hp[j + 1] = 1.0 / (nrm * nrm);
        CK(cudaMemcpyAsync(dinv + j + 1, hp.data() + j + 1, sizeof(double), cudaMemcpyHostToDevice, s));
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      const double rr = std::hypot(Hij(j, j), Hij(j + 1, j));
      if (rr == 0.0) PNP_FAIL(PNP_ERR_NAN, "ns: singular FGMRES Hessenberg matrix");
      cs[j] = Hij(j, j) / rr;
      sn[j] = Hij(j + 1, j) / rr;
      Hij(j, j) = rr;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      k = j + 1;
      if (p.monitor)
        fprintf(stderr, "[pnp ns fgmres %3d] estimated ||F|| %.6e\n", total, std::fabs(g[j + 1]));
      if (std::fabs(g[j + 1]) <= target || nrm <= 1e-300 * f) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
      y[i] = t / Hij(i, i);
    }
    // X += sum_j y_j z_j
    CK(cudaStreamSynchronize(s));  // the pinned slots are free
    for (int i = 0; i < k; ++i) S->hsc[i] = y[i];
    CK(cudaMemcpyAsync(dcoef, S->hsc, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    k_ns_combine<<<gsb(n), 256, k * sizeof(double), s>>>(n, k, S->Z, n, dcoef, S->X);
    note_launch();
    CK(cudaGetLastError());
    RC(ctx_ns_apply64(c, S->X, Ubody, S->F, true));
    st->matvecs64++;
    RC(ctx_norm4(c, S->F, &f));
    if (!std::isfinite(f)) PNP_FAIL(PNP_ERR_NAN, "ns: residual is not finite");
    ++cycles;
    if (p.monitor) fprintf(stderr, "[pnp ns cycle %2d] ||F|| %.6e (%d iterations)\n", cycles, f, total);
    // restart cycles that cut ||F|| by less than 5% three times in a row: the rounding floor
    // (<= 1e-9 ||F(X^0)||, converged) or a failure
    stalls = f < 0.95 * f_prev ? 0 : stalls + 1;
    if (stalls >= 3) {
      if (f <= 1e-9 * st->res0) {
        st->floor_stop = 1;
        break;
      }
      st->inner_its = total;
      st->refinements = cycles;
      return -1;  // stagnated: the caller continues with BiCGStab
    }
    f_prev = f;
  }
  st->inner_its = total;
  st->refinements = cycles;
  return PNP_OK;
}

// Solve the linear NS system for X (start: its current value), body force from Ubody.
int ctx_ns_solve(pnp_ctx* c, const double* Ubody, pnp_ns_stats* st) {
  const double t0 = now_ms();
  std::memset(st, 0, sizeof(*st));
  RC(ctx_ns_prepare(c));
  NsState* S = c->ns;
  const pnp_params& p = c->prm;
  const int64_t N = c->n_nodes;
  cudaStream_t s = c->stream;
  S->fine32 = 0;
  RC(ctx_ns_block_diag(c, S->Dg));
  RC(ctx_ns_blocks_row_fix(c, S->Dg, S->Dinv));
  if (ns_mg_levels(c) > 0) RC(ctx_ns_mg_prepare(c));
  RC(ctx_ns_apply64(c, S->X, Ubody, S->F, true));
  st->matvecs64 = 1;
  double f;
  RC(ctx_norm4(c, S->F, &f));
  if (!std::isfinite(f)) PNP_FAIL(PNP_ERR_NAN, "ns: initial residual is not finite");
  st->res0 = f;
  const double target = std::max(p.ns_rtol * f, p.ns_atol);
  S->mg_off = false;
  int inner_total = 0, ref = 0, stalls = 0;
  if (p.ns_fgmres > 0) {
    const int rc = f > target ? ns_fgmres(c, Ubody, target, f, st) : PNP_OK;
    if (rc >= 0) {
      st->status = rc;
      st->matvecs32 = (int32_t)S->fine32;
      st->res_final = f;
      st->wall_ms = now_ms() - t0;
      return rc;
    }
    // FGMRES stagnated: BiCGStab refinement from its iterate (restart cycles and refinement
    // steps add up in st->refinements, Krylov iterations in st->inner_its)
    st->krylov_fallbacks++;
    inner_total = st->inner_its;
    ref = st->refinements;
    if (p.monitor) fprintf(stderr, "[pnp ns] FGMRES stagnated at ||F|| %.6e: BiCGStab refinement\n", f);
  }
  int rc = PNP_OK;
  double f_prev = f;
  // a refinement step that raises ||F|| is undone (X and F kept in the free block buffer)
  // and, with multigrid, the rest of the solve uses the inverted blocks
  double* Xs = S->Dg;
  double* Fs = S->Dg + 4 * N;
  S->mg_off = false;
  while (f > target) {
    if (ref >= kMaxRefine || inner_total >= p.ns_max_it) {
      rc = PNP_ERR_KRYLOV_MAXIT;
      pnp_set_error("ns: %d refinements, %d BiCGStab iterations, ||F|| = %.3e > %.3e", ref, inner_total, f, target);
      break;
    }
    CK(cudaMemcpyAsync(Xs, S->X, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(Fs, S->F, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, s));
    k_ns_to_f32<<<nblk(N, 256), 256, 0, s>>>(N, S->F, -1.0 / f, S->r);
    note_launch();
    int its = 0;
    RC(ns_bicgstab32(c, p.ns_inner_rtol, std::min(p.ns_inner_max_it, p.ns_max_it - inner_total), &its));
    inner_total += its;
    k_ns_add_f32<<<nblk(N, 256), 256, 0, s>>>(N, S->x, f, S->X);
    note_launch();
    RC(ctx_ns_apply64(c, S->X, Ubody, S->F, true));
    st->matvecs64++;
    double fn;
    RC(ctx_norm4(c, S->F, &fn));
    ++ref;
    const bool worse = !(fn <= f);  // non-finite included
    if (p.monitor)
      fprintf(stderr, "[pnp ns %2d] ||F|| %.6e -> %.6e  bicgstab its %4d%s%s\n", ref, f, fn, its,
              (ns_mg_levels(c) > 0 && !S->mg_off) ? "  multigrid" : "", worse ? "  (undone)" : "");
    if (worse) {
      CK(cudaMemcpyAsync(S->X, Xs, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(S->F, Fs, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, s));
      if (ns_mg_levels(c) > 0 && !S->mg_off) {
        S->mg_off = true;
        st->mg_fallbacks++;
        continue;
      }
    } else {
      f = fn;
    }
    // three refinement steps in a row without reducing ||F|| end the solve: at the
    // rounding floor of the FP64 residual (||F|| <= 1e-9 ||F(X^0)||) as converged
    // (floor_stop), above it as a failure
    stalls = f < f_prev ? 0 : stalls + 1;
    if (stalls >= 3) {
      if (f <= 1e-9 * st->res0) {
        st->floor_stop = 1;
        break;
      }
      rc = PNP_ERR_KRYLOV_MAXIT;
      pnp_set_error("ns: no progress in three refinement steps (||F|| = %.3e)", f);
      break;
    }
    f_prev = f;
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->dflag + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  st->status = rc;
  st->refinements = ref;
  // BiCGStab: two per iteration, and the V-cycles' finest-level applications
  st->matvecs32 += 2 * (inner_total - st->inner_its) + (int32_t)S->fine32;
  st->inner_its = inner_total;
  st->res_final = f;
  st->singular_blocks = (flag & 4) ? 1 : 0;
  st->wall_ms = now_ms() - t0;
  return rc;
}

// copy v^{k+1} of X to a node-major [N][3] velocity
int ctx_ns_velocity(pnp_ctx* c, double* v3) {
  k_ns_velocity<<<nblk(c->n_nodes, 256), 256, 0, c->stream>>>(c->n_nodes, c->ns->X, v3);
  note_launch();
  CK(cudaGetLastError());
  return PNP_OK;
}
