// element_kernels.cuh -- Q1 element arithmetic on octree leaves for the VMS PNP residual
// (Def. 3 of arXiv 2301.05985) and its Jacobian action.
//
// Sum factorisation used here.  Nodal values u_c of a Q1 function on the reference cube
// [-1,1]^d (corner c: bit k set <=> +1 along axis k) map by a Walsh-Hadamard butterfly
// to monomial coefficients a_m (u = 2^-d sum_m a_m xi^m, m a subset of the axes).  At the
// 2^d Gauss points xi = g sigma (g = 1/sqrt 3, sigma in {-1,+1}^d) with b_m = 2^-d g^|m| a_m
// and t_m = sigma^m b_m:
//     u(q)           = sum_m t_m
//     du/dx_k(q)     = (2 / (h g)) sigma_k sum_{m contains k} t_m.
// The test side is the transpose: element vector
//     r_c = w 2^-d sum_m s^m(c) g^|m| A_m,
//     A_m = sum_q sigma^m(q) [ S_q + (2/(h g)) sum_{k in m} sigma_k(q) Phi_{q,k} ],
// where S_q / Phi_q multiply q / grad q in the weak form and w = (h/2)^d.
#pragma once

#include "pnp_internal.h"

namespace pnpk {

constexpr double kGauss = 0.57735026918962576450914878050196;  // 1/sqrt(3)

__host__ __device__ constexpr int popc_c(int x) { return x ? (x & 1) + popc_c(x >> 1) : 0; }
__host__ __device__ constexpr double gpow(int p) {
  return p == 0 ? 1.0 : (p == 1 ? kGauss : (p == 2 ? 1.0 / 3.0 : kGauss / 3.0));
}
// sign of sigma^m at Gauss point q
__host__ __device__ constexpr bool neg_sig(int m, int q) { return (popc_c(m & ~q) & 1) != 0; }

template <typename T, int D>
__device__ __forceinline__ void fwd_butterfly(T (&u)[1 << D]) {
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int c = 0; c < (1 << D); ++c)
      if (!((c >> k) & 1)) {
        const T lo = u[c], hi = u[c | (1 << k)];
        u[c] = lo + hi;
        u[c | (1 << k)] = hi - lo;
      }
}

template <typename T, int D>
__device__ __forceinline__ void bwd_butterfly(T (&x)[1 << D]) {
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int m = 0; m < (1 << D); ++m)
      if (!((m >> k) & 1)) {
        const T lo = x[m], hi = x[m | (1 << k)];
        x[m] = lo - hi;
        x[m | (1 << k)] = lo + hi;
      }
}

// nodal -> scaled monomial coefficients b_m
template <typename T, int D>
__device__ __forceinline__ void to_modal(T (&u)[1 << D]) {
  fwd_butterfly<T, D>(u);
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) u[m] *= T(gpow(popc_c(m)) / double(1 << D));
}

template <typename T, int D, int Q>
__device__ __forceinline__ T qp_value(const T (&b)[1 << D]) {
  T v = T(0);
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) v = neg_sig(m, Q) ? v - b[m] : v + b[m];
  return v;
}

// value and physical gradient at Gauss point Q; Gs = 2/(h g)
template <typename T, int D, int Q>
__device__ __forceinline__ void qp_value_grad(const T (&b)[1 << D], T Gs, T& v, T (&g)[3]) {
  v = qp_value<T, D, Q>(b);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    T s = T(0);
#pragma unroll
    for (int m = 0; m < (1 << D); ++m)
      if ((m >> k) & 1) s = neg_sig(m, Q) ? s - b[m] : s + b[m];
    g[k] = ((Q >> k) & 1) ? Gs * s : -Gs * s;
  }
#pragma unroll
  for (int k = D; k < 3; ++k) g[k] = T(0);
}

template <typename T, int D, int Q>
__device__ __forceinline__ void qp_grad(const T (&b)[1 << D], T Gs, T (&g)[3]) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    T s = T(0);
#pragma unroll
    for (int m = 0; m < (1 << D); ++m)
      if ((m >> k) & 1) s = neg_sig(m, Q) ? s - b[m] : s + b[m];
    g[k] = ((Q >> k) & 1) ? Gs * s : -Gs * s;
  }
#pragma unroll
  for (int k = D; k < 3; ++k) g[k] = T(0);
}

// A_m += sigma^m (S + sum_{k in m} Gs sigma_k Phi_k)
template <typename T, int D, int Q>
__device__ __forceinline__ void qp_test_acc(T (&A)[1 << D], T S, const T (&Phi)[3], T Gs) {
  T p[3];
#pragma unroll
  for (int k = 0; k < D; ++k) p[k] = ((Q >> k) & 1) ? Gs * Phi[k] : -Gs * Phi[k];
  T term[1 << D];
  term[0] = S;
#pragma unroll
  for (int m = 1; m < (1 << D); ++m) {
    // add the highest axis of m to the term of m without it
    const int k = (m & 4) ? 2 : ((m & 2) ? 1 : 0);
    term[m] = term[m & ~(1 << k)] + p[k];
  }
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) A[m] = neg_sig(m, Q) ? A[m] - term[m] : A[m] + term[m];
}

// A_m -> element vector r_c (in place), including w 2^-d g^|m|
template <typename T, int D>
__device__ __forceinline__ void from_modal(T (&A)[1 << D], T w) {
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) A[m] *= w * T(gpow(popc_c(m)) / double(1 << D));
  bwd_butterfly<T, D>(A);
}

// ---- runtime Gauss-point variants (one loop body for all points: small code) ----
// s[m] = sigma^m(q), sg[k] = sigma_k(q) for the Gauss point with bit pattern q.
template <typename T, int D>
struct QpSign {
  T s[1 << D];
  T sg[3];
};

template <typename T, int D>
__device__ __forceinline__ void qp_sign(int q, QpSign<T, D>& S) {
#pragma unroll
  for (int k = 0; k < D; ++k) S.sg[k] = ((q >> k) & 1) ? T(1) : T(-1);
#pragma unroll
  for (int k = D; k < 3; ++k) S.sg[k] = T(0);
  S.s[0] = T(1);
#pragma unroll
  for (int m = 1; m < (1 << D); ++m) {
    const int k = (m & 4) ? 2 : ((m & 2) ? 1 : 0);
    S.s[m] = S.s[m & ~(1 << k)] * S.sg[k];
  }
}

template <typename T, int D>
__device__ __forceinline__ T qpr_value(const T (&b)[1 << D], const QpSign<T, D>& S) {
  T v = T(0);
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) v = fma(S.s[m], b[m], v);
  return v;
}

// gradient: d/dx_k = Gs * sum_{m contains k} sigma^{m without k} b_m
template <typename T, int D>
__device__ __forceinline__ void qpr_grad(const T (&b)[1 << D], const QpSign<T, D>& S, T Gs, T (&g)[3]) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    T a = T(0);
#pragma unroll
    for (int m = 0; m < (1 << D); ++m)
      if ((m >> k) & 1) a = fma(S.s[m ^ (1 << k)], b[m], a);
    g[k] = Gs * a;
  }
#pragma unroll
  for (int k = D; k < 3; ++k) g[k] = T(0);
}

// A_m += sigma^m (S + sum_{k in m} Gs sigma_k Phi_k)
template <typename T, int D>
__device__ __forceinline__ void qpr_test_acc(T (&A)[1 << D], T Sv, const T (&Phi)[3], T Gs, const QpSign<T, D>& S) {
  T p[3];
#pragma unroll
  for (int k = 0; k < D; ++k) p[k] = (Gs * S.sg[k]) * Phi[k];
  T term[1 << D];
  term[0] = Sv;
#pragma unroll
  for (int m = 1; m < (1 << D); ++m) {
    const int k = (m & 4) ? 2 : ((m & 2) ? 1 : 0);
    term[m] = term[m & ~(1 << k)] + p[k];
  }
#pragma unroll
  for (int m = 0; m < (1 << D); ++m) A[m] = fma(S.s[m], term[m], A[m]);
}

}  // namespace pnpk
