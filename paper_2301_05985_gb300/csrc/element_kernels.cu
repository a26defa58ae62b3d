// element_kernels.cu -- fused gather / Gauss-point physics / test contraction / scatter
// for the VMS PNP residual and its Jacobian action, plus the exact 3x3 block diagonal.
//
// Physics per Gauss point (Def. 3 of arXiv 2301.05985 with c^f = -tau_c R_c, Sec. 3.1):
//   P_s  = v - z_s grad(phi)
//   R_s  = kappa c_s + h_s + P_s . grad c_s          (lap of a Q1 field on a cube is 0)
//   Nernst-Planck row:  q [kappa c_s + h_s + v.grad c_s] + grad q . [grad c_s + z_s c_s grad phi + tau R_s P_s]
//   Poisson row:        2 eps^2 grad q . grad phi - q sum_s z_s c_s + q sum_s z_s tau R_s
// with kappa = beta0/dt, h_s = (beta1 c_s^k + beta2 c_s^{k-1})/dt (both 0 when steady) and
// tau = (4/dt^2 + (2/h)^2 |v|^2 + C_I d (2/h)^4)^(-1/2).  J V is the exact directional
// derivative (the residual is cubic in U; tau does not depend on U).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "element_kernels.cuh"
#include "kernels.h"

using namespace pnpk;

namespace {

template <int Q, int NQ, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (Q < NQ) {
    f(std::integral_constant<int, Q>{});
    static_for<Q + 1, NQ>(f);
  }
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename T, int NF, int NC>
__device__ __forceinline__ void gather(const ElemArgs<T>& A, const int32_t (&conn)[NC], const T* __restrict__ src,
                                       int stride, T (&dst)[NF][NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int32_t id = conn[c];
    if (id >= 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[f][c] = __ldg(src + (int64_t)stride * id + f);
    } else {
      const int32_t hidx = -id - 1;
      const int np = A.hang_np[hidx];
      const T wgt = np == 2 ? T(0.5) : T(0.25);
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[f][c] = T(0);
      for (int p = 0; p < np; ++p) {
        const int32_t pid = A.hang_par[4 * hidx + p];
#pragma unroll
        for (int f = 0; f < NF; ++f) dst[f][c] += wgt * __ldg(src + (int64_t)stride * pid + f);
      }
    }
  }
}

template <typename T, int NC>
__device__ __forceinline__ void scatter(const ElemArgs<T>& A, const int32_t (&conn)[NC], T (&r)[3][NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int32_t id = conn[c];
    if (id >= 0) {
#pragma unroll
      for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)id + f, r[f][c]);
    } else {
      const int32_t hidx = -id - 1;
      const int np = A.hang_np[hidx];
      const T wgt = np == 2 ? T(0.5) : T(0.25);
      for (int p = 0; p < np; ++p) {
        const int32_t pid = A.hang_par[4 * hidx + p];
#pragma unroll
        for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)pid + f, wgt * r[f][c]);
      }
    }
  }
}

// Element vector (3 fields x 2^D corners) of the residual (JV = false) or of J V (JV =
// true) from nodal values u (U), va (advection), hs (history), du (direction), all
// [field][corner]; the inputs are overwritten by their modal coefficients.
template <typename T, int D, bool JV>
__device__ __forceinline__ void element_compute(T (&u)[3][1 << D], T (&va)[3][1 << D], T (&hs)[2][1 << D],
                                                T (&du)[3][1 << D], int lev, const PhysParams& Pp,
                                                T (&acc)[3][1 << D]) {
  constexpr int NC = 1 << D;
  const T h = T(ldexp(1.0, -lev));
  const T inv_h = T(ldexp(1.0, lev));
  const T Gs = T(2.0 / kGauss) * inv_h;     // 2 / (h g)
  const T G2 = T(4.0) * inv_h * inv_h;      // (2/h)^2
  T w = T(1);
#pragma unroll
  for (int k = 0; k < D; ++k) w *= T(0.5) * h;
  const T kappa = T(Pp.kappa);
  const T tau0 = T(Pp.tau_t) + T(Pp.C_I * D) * G2 * G2;
  const T e2 = T(Pp.eps2x2);
#pragma unroll
  for (int f = 0; f < 3; ++f) to_modal<T, D>(u[f]);
#pragma unroll
  for (int f = 0; f < D; ++f) to_modal<T, D>(va[f]);
#pragma unroll
  for (int f = 0; f < 2; ++f) to_modal<T, D>(hs[f]);
  if constexpr (JV) {
#pragma unroll
    for (int f = 0; f < 3; ++f) to_modal<T, D>(du[f]);
  }
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int m = 0; m < NC; ++m) acc[f][m] = T(0);

#pragma unroll 1
  for (int q = 0; q < NC; ++q) {
    QpSign<T, D> sgn;
    qp_sign<T, D>(q, sgn);
    T cv[2], gc[2][3], gp[3], v[3] = {T(0), T(0), T(0)}, hq[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      cv[s] = qpr_value<T, D>(u[s], sgn);
      qpr_grad<T, D>(u[s], sgn, Gs, gc[s]);
      hq[s] = qpr_value<T, D>(hs[s], sgn);
    }
    qpr_grad<T, D>(u[2], sgn, Gs, gp);
    T vv = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = qpr_value<T, D>(va[k], sgn);
      vv += v[k] * v[k];
    }
    const T tau = rsq(tau0 + G2 * vv);
    T R[2], P[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T z = s == 0 ? T(1) : T(-1);
      T pg = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        P[s][k] = v[k] - z * gp[k];
        pg += P[s][k] * gc[s][k];
      }
      R[s] = kappa * cv[s] + hq[s] + pg;
    }
    if constexpr (!JV) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T z = s == 0 ? T(1) : T(-1);
        T vg = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) vg += v[k] * gc[s][k];
        const T S = kappa * cv[s] + hq[s] + vg;
        const T tR = tau * R[s];
        const T zc = z * cv[s];
        T Phi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Phi[k] = gc[s][k] + zc * gp[k] + tR * P[s][k];
        qpr_test_acc<T, D>(acc[s], S, Phi, Gs, sgn);
      }
      const T S = -(cv[0] - cv[1]) + tau * (R[0] - R[1]);
      T Phi[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[k] = e2 * gp[k];
      qpr_test_acc<T, D>(acc[2], S, Phi, Gs, sgn);
    } else {
      T dcv[2], dgc[2][3], dgp[3];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        dcv[s] = qpr_value<T, D>(du[s], sgn);
        qpr_grad<T, D>(du[s], sgn, Gs, dgc[s]);
      }
      qpr_grad<T, D>(du[2], sgn, Gs, dgp);
      T dR[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T z = s == 0 ? T(1) : T(-1);
        T vg = T(0), pg = T(0), gcd = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          vg += v[k] * dgc[s][k];
          pg += P[s][k] * dgc[s][k];
          gcd += gc[s][k] * dgp[k];
        }
        dR[s] = kappa * dcv[s] + pg - z * gcd;
        const T S = kappa * dcv[s] + vg;
        const T tdR = tau * dR[s];
        const T zdc = z * dcv[s];
        const T zc_tR = z * (cv[s] - tau * R[s]);
        T Phi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Phi[k] = dgc[s][k] + zdc * gp[k] + zc_tR * dgp[k] + tdR * P[s][k];
        qpr_test_acc<T, D>(acc[s], S, Phi, Gs, sgn);
      }
      const T S = -(dcv[0] - dcv[1]) + tau * (dR[0] - dR[1]);
      T Phi[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[k] = e2 * dgp[k];
      qpr_test_acc<T, D>(acc[2], S, Phi, Gs, sgn);
    }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) from_modal<T, D>(acc[f], w);
}

template <typename T, int D, bool JV>
__global__ void __launch_bounds__(128) k_element(ElemArgs<T> A) {
  constexpr int NC = 1 << D;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.n_elem) return;
  int32_t conn[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) conn[c] = __ldg(A.conn + e * NC + c);
  T u[3][NC], va[3][NC], hs[2][NC], du[3][NC], acc[3][NC];
  gather<T, 3, NC>(A, conn, A.U, 3, u);
  gather<T, 3, NC>(A, conn, A.adv, 3, va);
  gather<T, 2, NC>(A, conn, A.hs, 2, hs);
  if constexpr (JV) gather<T, 3, NC>(A, conn, A.V, 3, du);
  element_compute<T, D, JV>(u, va, hs, du, A.level[e], A.P, acc);
  scatter<T, NC>(A, conn, acc);
}

// ------------------------------------------------------------------ patch kernels
// One CTA per Morton patch of up to kPatchElems elements: the patch's target nodes are
// staged in shared memory (one coalesced-by-slot pass over the node data), each thread
// computes one element from shared memory, contributions are added colour by colour into
// shared-memory accumulators (elements of one colour share no node: no atomics, fixed
// order), then owned rows are written with the Dirichlet rows applied and shared rows go
// to a partial buffer summed by k_patch_finalize in patch order.  Deterministic.
constexpr int kPatchElems = 256;

template <typename T>
__device__ __forceinline__ T dirichlet_row(const BcTable& bc, uint8_t fm, int f, bool jv, T acc, T u, T v) {
  const unsigned msk = fm & bc.dir_faces[f] & 0x3F;
  if (!msk) return acc;
  return jv ? v : T(double(u) - bc.val[31 - __clz(msk)][f]);
}

template <typename T, int D, bool JV>
__global__ void __launch_bounds__(kPatchElems) k_patch(PatchArgs<T> A) {
  constexpr int NC = 1 << D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int PN = A.pt.max_nodes;
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sA = sU + 3 * PN;
  T* sH = sA + 3 * PN;
  T* acc = sH + 2 * PN;
  T* sV = acc + 3 * PN;  // JV only
  const int p = blockIdx.x;
  const int n0 = A.pt.patch_n0[p], nn = A.pt.patch_n0[p + 1] - n0;
  const int e0 = A.pt.patch_e0[p], ne = A.pt.patch_e0[p + 1] - e0;
  const int h0 = A.pt.patch_h0[p];
  for (int s = threadIdx.x; s < nn; s += blockDim.x) {
    const int64_t id = A.pt.pnode[n0 + s];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      sU[f * PN + s] = A.U[3 * id + f];
      sA[f * PN + s] = A.adv[3 * id + f];
      acc[f * PN + s] = T(0);
      if constexpr (JV) sV[f * PN + s] = A.V[3 * id + f];
    }
    sH[s] = A.hs[2 * id];
    sH[PN + s] = A.hs[2 * id + 1];
  }
  __syncthreads();
  const int t = threadIdx.x;
  int color = -1;
  uint16_t slot[NC];
  T r[3][NC];
  if (t < ne) {
    const int64_t e = e0 + t;
    color = A.pt.el_color[e];
#pragma unroll
    for (int c = 0; c < NC; ++c) slot[c] = A.pt.el_slot[e * NC + c];
    T u[3][NC], va[3][NC], hs[2][NC], du[3][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const uint16_t sl = slot[c];
      if (!(sl & 0x8000)) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          u[f][c] = sU[f * PN + sl];
          va[f][c] = sA[f * PN + sl];
          if constexpr (JV) du[f][c] = sV[f * PN + sl];
        }
        hs[0][c] = sH[sl];
        hs[1][c] = sH[PN + sl];
      } else {
        const int hc = h0 + (sl & 0x7FFF);
        const int np = A.pt.hc_np[hc];
        const T wgt = np == 2 ? T(0.5) : T(0.25);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          u[f][c] = T(0);
          va[f][c] = T(0);
          du[f][c] = T(0);
        }
        hs[0][c] = T(0);
        hs[1][c] = T(0);
        for (int q = 0; q < np; ++q) {
          const int ps = A.pt.hc_par[4 * hc + q];
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            u[f][c] += wgt * sU[f * PN + ps];
            va[f][c] += wgt * sA[f * PN + ps];
            if constexpr (JV) du[f][c] += wgt * sV[f * PN + ps];
          }
          hs[0][c] += wgt * sH[ps];
          hs[1][c] += wgt * sH[PN + ps];
        }
      }
    }
    element_compute<T, D, JV>(u, va, hs, du, A.level[e], A.P, r);
  }
  const int ncol = A.pt.patch_ncol[p];
  for (int col = 0; col < ncol; ++col) {
    if (color == col) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const uint16_t sl = slot[c];
        if (!(sl & 0x8000)) {
#pragma unroll
          for (int f = 0; f < 3; ++f) acc[f * PN + sl] += r[f][c];
        } else {
          const int hc = h0 + (sl & 0x7FFF);
          const int np = A.pt.hc_np[hc];
          const T wgt = np == 2 ? T(0.5) : T(0.25);
          for (int q = 0; q < np; ++q) {
            const int ps = A.pt.hc_par[4 * hc + q];
#pragma unroll
            for (int f = 0; f < 3; ++f) acc[f * PN + ps] += wgt * r[f][c];
          }
        }
      }
    }
    __syncthreads();
  }
  for (int s = threadIdx.x; s < nn; s += blockDim.x) {
    const int64_t id = A.pt.pnode[n0 + s];
    const int32_t q = A.pt.pbslot[n0 + s];
    if (q < 0) {
      const uint8_t fm = A.faces[id];
#pragma unroll
      for (int f = 0; f < 3; ++f)
        A.out[3 * id + f] = dirichlet_row<T>(A.bc, fm, f, JV, acc[f * PN + s], sU[f * PN + s],
                                             JV ? sV[f * PN + s] : T(0));
    } else {
#pragma unroll
      for (int f = 0; f < 3; ++f) A.partial[3 * (int64_t)q + f] = acc[f * PN + s];
    }
  }
}

// shared nodes: sum their partials in patch order, then apply the Dirichlet rows
template <typename T>
__global__ void k_patch_finalize(PatchArgs<T> A, bool jv) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.pt.n_bnodes) return;
  const int64_t id = A.pt.bnode[b];
  T v[3] = {T(0), T(0), T(0)};
  for (int32_t q = A.pt.bptr[b]; q < A.pt.bptr[b + 1]; ++q)
#pragma unroll
    for (int f = 0; f < 3; ++f) v[f] += A.partial[3 * (int64_t)q + f];
  const uint8_t fm = A.faces[id];
#pragma unroll
  for (int f = 0; f < 3; ++f)
    A.out[3 * id + f] = dirichlet_row<T>(A.bc, fm, f, jv, v[f], A.U[3 * id + f], jv ? A.V[3 * id + f] : T(0));
}

// ------------------------------------------------------------------ row fix-ups
// mode 0: F = U - g on Dirichlet rows;  mode 1: out = V on Dirichlet rows.
template <typename T>
__global__ void k_dirichlet_rows(int64_t N, const uint8_t* __restrict__ faces, BcTable bc, const T* __restrict__ in,
                                 T* __restrict__ out, int mode) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint8_t fm = faces[i];
  if (fm & 0x80) return;  // hanging: constraint row written separately
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const unsigned msk = fm & bc.dir_faces[f] & 0x3F;
    if (msk) {
      const int face = 31 - __clz(msk);
      out[3 * i + f] = mode == 0 ? T(double(in[3 * i + f]) - bc.val[face][f]) : in[3 * i + f];
    }
  }
}

// out_h = in_h - sum_p w_p in_p  (constraint rows of hanging nodes)
template <typename T>
__global__ void k_hanging_rows(int64_t H, const int32_t* __restrict__ hnode, const int32_t* __restrict__ hpar,
                               const uint8_t* __restrict__ hnp, const T* __restrict__ in, T* __restrict__ out) {
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= H) return;
  const int np = hnp[h];
  const T wgt = np == 2 ? T(0.5) : T(0.25);
  const int64_t id = hnode[h];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    T s = in[3 * id + f];
    for (int p = 0; p < np; ++p) s -= wgt * in[3 * (int64_t)hpar[4 * h + p] + f];
    out[3 * id + f] = s;
  }
}

// Dirichlet / hanging rows of the block diagonal.
template <typename T>
__global__ void k_diag_rows(int64_t N, const uint8_t* __restrict__ faces, BcTable bc, T* __restrict__ Dg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint8_t fm = faces[i];
  T* B = Dg + 9 * i;
  if (fm & 0x80) {
    for (int k = 0; k < 9; ++k) B[k] = (k % 4 == 0) ? T(1) : T(0);
    return;
  }
  for (int f = 0; f < 3; ++f)
    if (fm & bc.dir_faces[f] & 0x3F)
      for (int g = 0; g < 3; ++g) B[3 * f + g] = (f == g) ? T(1) : T(0);
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ launchers
// Element kernel of launch_element: one lane group per element unless
// PNP_ELEMENT_KERNEL=thread selects one thread per element (modal sum factorisation).
static bool per_thread_elements() {
  static const bool v = [] {
    const char* e = getenv("PNP_ELEMENT_KERNEL");
    return e && strcmp(e, "thread") == 0;
  }();
  return v;
}

bool element_kernel_is_lanes() { return !per_thread_elements(); }

bool residual_double_float() {
  static const bool v = [] {
    const char* e = getenv("PNP_RESIDUAL_ARITH");
    return !(e && strcmp(e, "f64") == 0);
  }();
  return v && !per_thread_elements();
}

double element_kernel_flops(int D, bool jv) {
  const double NC = 1 << D;
  if (per_thread_elements()) {
    // modal form: nodal -> modal transforms, per Gauss point values / gradients from
    // the modal coefficients, physics, test contraction, modal -> nodal
    const double val = 2 * NC, grad = D * (NC + 1);
    const double to_m = D * NC + NC, from_m = D * NC + 2 * NC;
    const double acc = 2 * D + (NC - 1) + 2 * NC;
    const double common = 2 * val + 2 * grad + 2 * val + grad + D * val + 2 * D + 3 + 2 * (3 * D + 3);
    const double poisson = 4 + D + acc;
    if (!jv) return NC * (common + 2 * (6 * D + 4 + acc) + poisson) + 8 * to_m + 3 * from_m;
    return NC * (common + 2 * val + 3 * grad + 2 * (12 * D + 8 + acc) + poisson) + 11 * to_m + 3 * from_m;
  }
  // lane form, per lane: axis stages of the value/gradient interpolation (3 flops per
  // interpolated track, 4 per value + new derivative from one difference), the physics
  // at the lane's Gauss point, and the transposed stages of the three test fields
  const double tri = D * (D - 1) / 2.0;
  const double vg = 3 * tri + 4 * D, g = vg - 2, v = 3 * D, tt = 6 * D + 3 * tri + 1;
  const double state = 2 * vg + 2 * v + g + D * v + 2 * D + 3 + 30;
  const double phys = jv ? 2 * vg + g + 101 : 53;
  return NC * (state + phys + 3 * tt);
}

template <typename T>
cudaError_t launch_element(int dim, bool jv, const ElemArgs<T>& A, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  // default: one lane group per element; PNP_ELEMENT_KERNEL=thread selects one thread
  // per element (modal sum factorisation in registers)
  if (!per_thread_elements()) return launch_element_lanes<T>(dim, jv, A, s);
  const int t = 128;
  if (dim == 2) {
    if (jv) { k_element<T, 2, true><<<nblk(A.n_elem, t), t, 0, s>>>(A); note_launch(); }
    else { k_element<T, 2, false><<<nblk(A.n_elem, t), t, 0, s>>>(A); note_launch(); }
  } else {
    if (jv) { k_element<T, 3, true><<<nblk(A.n_elem, t), t, 0, s>>>(A); note_launch(); }
    else { k_element<T, 3, false><<<nblk(A.n_elem, t), t, 0, s>>>(A); note_launch(); }
  }
  return cudaGetLastError();
}
template cudaError_t launch_element<double>(int, bool, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_element<float>(int, bool, const ElemArgs<float>&, cudaStream_t);

template <typename T>
cudaError_t launch_patch(int dim, bool jv, const PatchArgs<T>& A, cudaStream_t s) {
  if (A.pt.n_patches == 0) return cudaSuccess;
  const size_t smem = (size_t)(jv ? 14 : 11) * A.pt.max_nodes * sizeof(T);
  void (*kern)(PatchArgs<T>);
  if (dim == 2) kern = jv ? k_patch<T, 2, true> : k_patch<T, 2, false>;
  else kern = jv ? k_patch<T, 3, true> : k_patch<T, 3, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)A.pt.n_patches, kPatchElems, smem, s>>>(A); note_launch();
  if (A.pt.n_bnodes) { k_patch_finalize<T><<<nblk(A.pt.n_bnodes, 256), 256, 0, s>>>(A, jv); note_launch(); }
  return cudaGetLastError();
}
template cudaError_t launch_patch<double>(int, bool, const PatchArgs<double>&, cudaStream_t);
template cudaError_t launch_patch<float>(int, bool, const PatchArgs<float>&, cudaStream_t);

template <typename T>
cudaError_t launch_row_fixups(const RowArgs& R, const T* in, T* out, int mode, cudaStream_t s) {
  const int t = 256;
  if (R.n_nodes) { k_dirichlet_rows<T><<<nblk(R.n_nodes, t), t, 0, s>>>(R.n_nodes, R.faces, R.bc, in, out, mode); note_launch(); }
  if (R.n_hanging) { k_hanging_rows<T><<<nblk(R.n_hanging, t), t, 0, s>>>(R.n_hanging, R.hnode, R.hpar, R.hnp, in, out); note_launch(); }
  return cudaGetLastError();
}
template cudaError_t launch_row_fixups<double>(const RowArgs&, const double*, double*, int, cudaStream_t);
template cudaError_t launch_row_fixups<float>(const RowArgs&, const float*, float*, int, cudaStream_t);

template <typename T>
cudaError_t launch_diag_rows(const RowArgs& R, T* Dg, cudaStream_t s) {
  if (R.n_nodes) { k_diag_rows<T><<<nblk(R.n_nodes, 256), 256, 0, s>>>(R.n_nodes, R.faces, R.bc, Dg); note_launch(); }
  return cudaGetLastError();
}
template cudaError_t launch_diag_rows<double>(const RowArgs&, double*, cudaStream_t);
template cudaError_t launch_diag_rows<float>(const RowArgs&, float*, cudaStream_t);
