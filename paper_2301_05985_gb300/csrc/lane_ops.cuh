// lane_ops.cuh -- lane-group Q1 arithmetic shared by the element kernels: 2^d lanes of a
// warp hold the corners of one element and the Gauss points next to them.  Interpolation
// is a tensor product of 1D operators on the two nodes of an axis: at the Gauss point
// next to node b (xi = -g for b = 0, +g for b = 1, g = 1/sqrt 3)
//     value:       a u_b + b' u_{1-b} = u_b - b' (u_b - u_{1-b}),   a = (1 + g)/2, b' = (1 - g)/2
//     derivative:  (u_1 - u_0) / h           (constant along the axis)
// applied axis by axis with the partner value fetched by a lane shuffle (lane ^ 2^k).
// The test side (element vector r_c = w sum_q [N_c(q) S_q + grad N_c(q) . Phi_q], w =
// (h/2)^d) is the transpose: the value operator is symmetric and the derivative's
// transpose sends s_b (x_0 + x_1) / h to node b (s_0 = -1, s_1 = +1).
#pragma once

#include "df32.cuh"

namespace {

constexpr double kG = 0.57735026918962576450914878050196;  // 1/sqrt(3)
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T flip(T x, int k) {
  return __shfl_xor_sync(kFull, x, 1 << k);
}
__device__ __forceinline__ df flip(df x, int k) {
  return df(__shfl_xor_sync(kFull, x.hi, 1 << k), __shfl_xor_sync(kFull, x.lo, 1 << k));
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
__device__ __forceinline__ df pow2i(int e, df) { return df(pow2i(e, 0.0f), 0.0f); }

// value and gradient of corner i's shape function at this lane's Gauss point (corner c)
template <typename T, int D>
__device__ __forceinline__ void shape_at(int i, int c, T inv_h, T& N, T (&dN)[3]) {
  const T fs = T(0.5 * (1.0 + kG)), fo = T(0.5 * (1.0 - kG));
  T f[3];
#pragma unroll
  for (int k = 0; k < D; ++k) f[k] = (((i ^ c) >> k) & 1) ? fo : fs;
  N = T(1);
#pragma unroll
  for (int k = 0; k < D; ++k) N *= f[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T a = T(0);
    if (k < D) {
      a = ((i >> k) & 1) ? inv_h : -inv_h;
#pragma unroll
      for (int l = 0; l < D; ++l)
        if (l != k) a *= f[l];
    }
    dN[k] = a;
  }
}

// loaded value in the arithmetic type, and back to the storage type
template <typename C, typename T>
__device__ __forceinline__ C to_compute(T x) { return C(x); }
template <>
__device__ __forceinline__ df to_compute<df, double>(double x) { return df_split(x); }
template <typename T>
__device__ __forceinline__ T to_storage(T x) { return x; }
template <typename T>
__device__ __forceinline__ T to_storage(df x) { return df_to_double(x); }

}  // namespace
