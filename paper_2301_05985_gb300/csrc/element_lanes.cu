// element_lanes.cu -- the VMS PNP residual and its Jacobian action with one lane group
// per element: 2^d lanes of a warp share an element, lane c holds corner c and the
// Gauss point next to it.
//
// Physics per Gauss point as in Def. 3 of arXiv 2301.05985 with the fine scales
// c^f = -tau_c R_c (Sec. 3.1; the same statement as element_kernels.cu).  Interpolation
// is a tensor product of 1D operators on the two nodes of an axis: at the Gauss point
// next to node b (xi = -g for b = 0, +g for b = 1, g = 1/sqrt 3)
//     value:       a u_b + b' u_{1-b} = u_b - b' (u_b - u_{1-b}),   a = (1 + g)/2, b' = (1 - g)/2
//     derivative:  (u_1 - u_0) / h           (constant along the axis)
// applied axis by axis with the partner value fetched by a lane shuffle (lane ^ 2^k);
// value and derivative share the difference u_b - u_{1-b}.  The FP32 kernels execute no
// FP64 instruction (GB300 runs FP64 at 1/64 of the FP32 rate): powers of two come from
// the exponent bits and the parameters arrive converted.
// The test side (element vector r_c = w sum_q [N_c(q) S_q + grad N_c(q) . Phi_q], w =
// (h/2)^d) is the transpose: the value operator is symmetric and the derivative's
// transpose sends s_b (x_0 + x_1) / h to node b (s_0 = -1, s_1 = +1).
#include <cstdint>

#include "kernels.h"

namespace {

constexpr double kG = 0.57735026918962576450914878050196;  // 1/sqrt(3)
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T flip(T x, int k) {
  return __shfl_xor_sync(kFull, x, 1 << k);
}

// value and gradient at this lane's Gauss point from this lane's nodal value x
// (nb = -b': the value operator is x - b' (x - partner))
template <typename T, int D>
__device__ __forceinline__ void interp_vg(T x, T nb, const T (&sh)[3], T& val, T (&g)[3]) {
  T I = x;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T pI = flip(I, k);
    T pG[3];
#pragma unroll
    for (int j = 0; j < k; ++j) pG[j] = flip(g[j], k);
#pragma unroll
    for (int j = 0; j < k; ++j) g[j] = fma(nb, g[j] - pG[j], g[j]);
    const T d = I - pI;
    g[k] = sh[k] * d;
    I = fma(nb, d, I);
  }
#pragma unroll
  for (int k = D; k < 3; ++k) g[k] = T(0);
  val = I;
}

template <typename T, int D>
__device__ __forceinline__ void interp_g(T x, T nb, const T (&sh)[3], T (&g)[3]) {
  T I = x;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T pI = flip(I, k);
    T pG[3];
#pragma unroll
    for (int j = 0; j < k; ++j) pG[j] = flip(g[j], k);
#pragma unroll
    for (int j = 0; j < k; ++j) g[j] = fma(nb, g[j] - pG[j], g[j]);
    const T d = I - pI;
    g[k] = sh[k] * d;
    if (k + 1 < D) I = fma(nb, d, I);
  }
#pragma unroll
  for (int k = D; k < 3; ++k) g[k] = T(0);
}

template <typename T, int D>
__device__ __forceinline__ T interp_v(T x, T nb) {
#pragma unroll
  for (int k = 0; k < D; ++k) x = fma(nb, x - flip(x, k), x);
  return x;
}

// transpose: this lane's node contribution from the Gauss-point tests S, Phi
template <typename T, int D>
__device__ __forceinline__ T test_t(T S, T (&Phi)[3], T nb, const T (&sh)[3]) {
  T A = S;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    const T pA = flip(A, k);
    const T pH = flip(Phi[k], k);
    T pP[3];
#pragma unroll
    for (int j = 0; j < k; ++j) pP[j] = flip(Phi[j], k);
    A = fma(nb, A - pA, fma(sh[k], Phi[k] + pH, A));
#pragma unroll
    for (int j = 0; j < k; ++j) Phi[j] = fma(nb, Phi[j] - pP[j], Phi[j]);
  }
  return A;
}

// 2^e exactly, from the exponent bits (|e| well inside the exponent range)
__device__ __forceinline__ float pow2i(int e, float) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2i(int e, double) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// physical parameters in the kernel's arithmetic type
template <typename T>
struct LaneParams {
  T kappa;   // beta0 / dt
  T tau_t;   // 4 / dt^2
  T cid;     // C_I d
  T e2;      // 2 Lambda^2
};

// nodal values of NF interleaved fields at node id (hanging: the parents' mean)
template <typename T, int NF>
__device__ __forceinline__ void load_node(const ElemArgs<T>& A, int32_t id, bool valid, const T* __restrict__ src,
                                          int stride, T (&dst)[NF]) {
#pragma unroll
  for (int f = 0; f < NF; ++f) dst[f] = T(0);
  if (!valid) return;
  if (id >= 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) dst[f] = __ldg(src + (int64_t)stride * id + f);
  } else {
    const int32_t h = -id - 1;
    const int np = A.hang_np[h];
    const T wgt = np == 2 ? T(0.5) : T(0.25);
    for (int p = 0; p < np; ++p) {
      const int32_t pid = A.hang_par[4 * h + p];
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[f] += wgt * __ldg(src + (int64_t)stride * pid + f);
    }
  }
}

// the FP32 state of node id from its 32-byte record (two 16-byte loads; hanging: the
// parents' mean)
template <typename T>
__device__ __forceinline__ void load_record(const ElemArgs<T>& A, int32_t id, bool valid, float (&un)[3],
                                            float (&hn)[2], float (&vn)[3]) {
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
  if (valid) {
    if (id >= 0) {
      r0 = __ldg(A.rec + 2 * (int64_t)id);
      r1 = __ldg(A.rec + 2 * (int64_t)id + 1);
    } else {
      const int32_t h = -id - 1;
      const int np = A.hang_np[h];
      const float wgt = np == 2 ? 0.5f : 0.25f;
      for (int p = 0; p < np; ++p) {
        const int64_t pid = A.hang_par[4 * h + p];
        const float4 a = __ldg(A.rec + 2 * pid), b = __ldg(A.rec + 2 * pid + 1);
        r0.x += wgt * a.x; r0.y += wgt * a.y; r0.z += wgt * a.z; r0.w += wgt * a.w;
        r1.x += wgt * b.x; r1.y += wgt * b.y; r1.z += wgt * b.z; r1.w += wgt * b.w;
      }
    }
  }
  un[0] = r0.x; un[1] = r0.y; un[2] = r0.z;
  hn[0] = r0.w; hn[1] = r1.x;
  vn[0] = r1.y; vn[1] = r1.z; vn[2] = r1.w;
}

// the padded FP32 direction at node id (hanging: the parents' mean)
template <typename T>
__device__ __forceinline__ void load_dir4(const ElemArgs<T>& A, int32_t id, bool valid, float (&dn)[3]) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    if (id >= 0) {
      v = __ldg(A.V4 + id);
    } else {
      const int32_t h = -id - 1;
      const int np = A.hang_np[h];
      const float wgt = np == 2 ? 0.5f : 0.25f;
      for (int p = 0; p < np; ++p) {
        const float4 a = __ldg(A.V4 + A.hang_par[4 * h + p]);
        v.x += wgt * a.x; v.y += wgt * a.y; v.z += wgt * a.z;
      }
    }
  }
  dn[0] = v.x; dn[1] = v.y; dn[2] = v.z;
}

// one vector atomic per target node (hanging: weighted to its parents)
template <typename T>
__device__ __forceinline__ void scatter4(const ElemArgs<T>& A, int32_t id, const float (&r)[3]) {
  if (id >= 0) {
    atomicAdd(A.out4 + id, make_float4(r[0], r[1], r[2], 0.f));
  } else {
    const int32_t h = -id - 1;
    const int np = A.hang_np[h];
    const float wgt = np == 2 ? 0.5f : 0.25f;
    for (int p = 0; p < np; ++p)
      atomicAdd(A.out4 + A.hang_par[4 * h + p], make_float4(wgt * r[0], wgt * r[1], wgt * r[2], 0.f));
  }
}

template <typename T, int D, bool JV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) k_element_lanes(ElemArgs<T> A, LaneParams<T> K) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // warps whose first element is past the end leave together (shuffles need the warp)
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;
  const int64_t e = t / NC;
  const int c = (int)(t & (NC - 1));
  const bool valid = e < A.n_elem;
  const int32_t id = valid ? __ldg(A.conn + e * NC + c) : 0;
  const int lev = valid ? A.level[e] : 0;

  const T inv_h = pow2i(lev, T(0));
  const T w = pow2i(-D * (lev + 1), T(0));  // (h/2)^D
  const T nb = T(-0.5 * (1.0 - kG));
  T sh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[k] = ((c >> k) & 1) ? inv_h : -inv_h;
  const T G2 = pow2i(2 * lev + 2, T(0));  // (2/h)^2
  const T kappa = K.kappa;
  const T tau0 = fma(K.cid * G2, G2, K.tau_t);
  const T e2 = K.e2;

  T un[3], vn[3], hn[2];
  if constexpr (sizeof(T) == 4) {
    if (A.rec) {
      load_record(A, id, valid, un, hn, vn);
    } else {
      load_node<T, 3>(A, id, valid, A.U, 3, un);
      load_node<T, 3>(A, id, valid, A.adv, 3, vn);
      load_node<T, 2>(A, id, valid, A.hs, 2, hn);
    }
  } else {
    load_node<T, 3>(A, id, valid, A.U, 3, un);
    load_node<T, 3>(A, id, valid, A.adv, 3, vn);
    load_node<T, 2>(A, id, valid, A.hs, 2, hn);
  }

  // state at this lane's Gauss point
  T cv[2], gc[2][3], gp[3], v[3] = {T(0), T(0), T(0)}, hq[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    interp_vg<T, D>(un[s], nb, sh, cv[s], gc[s]);
    hq[s] = interp_v<T, D>(hn[s], nb);
  }
  interp_g<T, D>(un[2], nb, sh, gp);
  T vv = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = interp_v<T, D>(vn[k], nb);
    vv = fma(v[k], v[k], vv);
  }
  T tau;
  if constexpr (sizeof(T) == 4) tau = rsqrtf(tau0 + G2 * vv);
  else tau = T(1) / sqrt(tau0 + G2 * vv);
  T R[2], P[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T z = s == 0 ? T(1) : T(-1);
    T pg = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      P[s][k] = v[k] - z * gp[k];
      pg = fma(P[s][k], gc[s][k], pg);
    }
    R[s] = fma(kappa, cv[s], hq[s] + pg);
  }

  T S[3], Phi[3][3];
  if constexpr (!JV) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T z = s == 0 ? T(1) : T(-1);
      T vg = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) vg = fma(v[k], gc[s][k], vg);
      S[s] = fma(kappa, cv[s], hq[s] + vg);
      const T tR = tau * R[s];
      const T zc = z * cv[s];
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[s][k] = fma(tR, P[s][k], fma(zc, gp[k], gc[s][k]));
    }
    S[2] = fma(tau, R[0] - R[1], cv[1] - cv[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Phi[2][k] = e2 * gp[k];
  } else {
    T dn[3];
    if constexpr (sizeof(T) == 4) {
      if (A.V4) load_dir4(A, id, valid, dn);
      else load_node<T, 3>(A, id, valid, A.V, 3, dn);
    } else {
      load_node<T, 3>(A, id, valid, A.V, 3, dn);
    }
    T dcv[2], dgc[2][3], dgp[3], dR[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) interp_vg<T, D>(dn[s], nb, sh, dcv[s], dgc[s]);
    interp_g<T, D>(dn[2], nb, sh, dgp);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T z = s == 0 ? T(1) : T(-1);
      T vg = T(0), pg = T(0), gcd = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vg = fma(v[k], dgc[s][k], vg);
        pg = fma(P[s][k], dgc[s][k], pg);
        gcd = fma(gc[s][k], dgp[k], gcd);
      }
      dR[s] = fma(kappa, dcv[s], pg - z * gcd);
      S[s] = fma(kappa, dcv[s], vg);
      const T tdR = tau * dR[s];
      const T zdc = z * dcv[s];
      const T zc_tR = z * (cv[s] - tau * R[s]);
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[s][k] = fma(tdR, P[s][k], fma(zc_tR, dgp[k], fma(zdc, gp[k], dgc[s][k])));
    }
    S[2] = fma(tau, dR[0] - dR[1], dcv[1] - dcv[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Phi[2][k] = e2 * dgp[k];
  }

  T r[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) r[f] = w * test_t<T, D>(S[f], Phi[f], nb, sh);
  if (!valid) return;
  if constexpr (sizeof(T) == 4) {
    if (A.out4) {
      scatter4(A, id, r);
      return;
    }
  }
  if (id >= 0) {
#pragma unroll
    for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)id + f, r[f]);
  } else {
    const int32_t hh = -id - 1;
    const int np = A.hang_np[hh];
    const T wgt = np == 2 ? T(0.5) : T(0.25);
    for (int p = 0; p < np; ++p) {
      const int32_t pid = A.hang_par[4 * hh + p];
#pragma unroll
      for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)pid + f, wgt * r[f]);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_element_lanes(int dim, bool jv, const ElemArgs<T>& A, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  const int t = 256;
  const int64_t threads = A.n_elem << dim;
  const unsigned blocks = (unsigned)((threads + t - 1) / t);
  const LaneParams<T> K{T(A.P.kappa), T(A.P.tau_t), T(A.P.C_I * dim), T(A.P.eps2x2)};
  if (dim == 2) {
    if (jv) k_element_lanes<T, 2, true><<<blocks, t, 0, s>>>(A, K);
    else k_element_lanes<T, 2, false><<<blocks, t, 0, s>>>(A, K);
  } else {
    if (jv) k_element_lanes<T, 3, true><<<blocks, t, 0, s>>>(A, K);
    else k_element_lanes<T, 3, false><<<blocks, t, 0, s>>>(A, K);
  }
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_element_lanes<double>(int, bool, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_element_lanes<float>(int, bool, const ElemArgs<float>&, cudaStream_t);
