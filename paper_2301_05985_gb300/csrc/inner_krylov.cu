// inner_krylov.cu -- FP32 kernels of the inner GMRES(d) that preconditions the flexible
// outer GMRES in mixed precision.  The inner solve is a fixed number of Arnoldi steps on
// J M^-1 (M: the 3x3 block diagonal) whose small Hessenberg bookkeeping also stays on the
// device, so it needs no host round trip; the outer Krylov method keeps FP64 dots,
// orthogonalisation and basis (Sec. 4.1's Newton-Krylov, with the bulk work in FP32).
#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace {

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ float warp_sum4f(const float (&s)[4], int lane) {
  const bool hi4 = lane & 16, hi3 = lane & 8;
  const float a0 = (hi4 ? s[2] : s[0]) + __shfl_xor_sync(0xffffffffu, hi4 ? s[0] : s[2], 16);
  const float a1 = (hi4 ? s[3] : s[1]) + __shfl_xor_sync(0xffffffffu, hi4 ? s[1] : s[3], 16);
  float b = (hi3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, hi3 ? a0 : a1, 8);
  b += __shfl_xor_sync(0xffffffffu, b, 4);
  b += __shfl_xor_sync(0xffffffffu, b, 2);
  b += __shfl_xor_sync(0xffffffffu, b, 1);
  return b;
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// The inner basis has rows padded to a multiple of four floats (zeros beyond the
// vector's length), so both Gram-Schmidt kernels move float4: four entries per load.

// d_i = U_i . w (i < k) for FP32 vectors of n4 float4.  Persistent grid (kInnerBlocks, 8
// per SM): each block strides over chunks of 256 x kRows float4; for every group of four
// basis vectors a thread accumulates its rows of all chunks (w re-read from L2 per
// group), then one warp reduce-scatter and a fixed-order block sum give the block's
// partials part[block][k].
constexpr int kRows = 2;
__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, s))));
}
__global__ void __launch_bounds__(256, 8) k_multi_dot_f32(int64_t n4, int k, const float4* __restrict__ Ub,
                                                          int64_t ld4, const float4* __restrict__ w,
                                                          double* __restrict__ part) {
  __shared__ float sh[4][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = 256 * kRows;
  for (int j0 = 0; j0 < k; j0 += 4) {
    const int cnt = min(4, k - j0);
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < n4; c0 += (int64_t)gridDim.x * chunk) {
      float4 wv[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int64_t t = c0 + threadIdx.x + r * 256;
        wv[r] = t < n4 ? w[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < cnt) {
          const float4* ui = Ub + (int64_t)(j0 + q) * ld4;
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            const int64_t t = c0 + threadIdx.x + r * 256;
            if (t < n4) s[q] = dot4(__ldg(ui + t), wv[r], s[q]);
          }
        }
      }
    }
    const float tot = warp_sum4f(s, lane);
    const int q = (lane >> 3) & 3;
    if ((lane & 7) == 0) sh[q][wid] = tot;
    __syncthreads();
    if (threadIdx.x < cnt) {
      double t = 0.0;
#pragma unroll
      for (int v = 0; v < 8; ++v) t += (double)sh[threadIdx.x][v];
      part[(int64_t)blockIdx.x * k + j0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// w -= sum_i (d_i dinv_i) U_i (i < k) in FP32 on n4 float4, then per-block partials of
// w . w.  Persistent grid of 6 blocks per SM.
constexpr int kUpdBlocks = 6 * 152;
__global__ void __launch_bounds__(256, 6) k_multi_axpy_norm_f32(int64_t n4, int k, const float4* __restrict__ Ub,
                                                             int64_t ld4, const double* __restrict__ d,
                                                             const double* __restrict__ dinv, float4* __restrict__ w,
                                                             double* __restrict__ part) {
  extern __shared__ float cf[];
  __shared__ double sh[256];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = (float)(d[i] * dinv[i]);
  __syncthreads();
  float ss = 0.0f;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    float4 a = w[t];
    for (int i = 0; i < k; ++i) {
      const float4 u = Ub[(int64_t)i * ld4 + t];
      const float c = -cf[i];
      a.x = fmaf(c, u.x, a.x);
      a.y = fmaf(c, u.y, a.y);
      a.z = fmaf(c, u.z, a.z);
      a.w = fmaf(c, u.w, a.w);
    }
    if (k > 0) w[t] = a;
    ss = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, ss))));
  }
  const double tot = block_sum_d((double)ss, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// y_i = Dinv_i (inv_s[0] u_i) per node, FP32 3x3 blocks
__global__ void k_block_apply32(int64_t N, const float* __restrict__ Dinv, const float* __restrict__ u,
                                const float* __restrict__ inv_s, float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float sc = inv_s ? inv_s[0] : 1.0f;
  const float* B = Dinv + 9 * i;
  const float a = sc * u[3 * i], b = sc * u[3 * i + 1], c = sc * u[3 * i + 2];
  y[3 * i] = fmaf(B[0], a, fmaf(B[1], b, B[2] * c));
  y[3 * i + 1] = fmaf(B[3], a, fmaf(B[4], b, B[5] * c));
  y[3 * i + 2] = fmaf(B[6], a, fmaf(B[7], b, B[8] * c));
}

__global__ void k_block_apply32_pad(int64_t N, const float* __restrict__ Dinv, const float* __restrict__ u,
                                    const float* __restrict__ inv_s, float4* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float sc = inv_s ? inv_s[0] : 1.0f;
  const float* B = Dinv + 9 * i;
  const float a = sc * u[3 * i], b = sc * u[3 * i + 1], c = sc * u[3 * i + 2];
  y[i] = make_float4(fmaf(B[0], a, fmaf(B[1], b, B[2] * c)), fmaf(B[3], a, fmaf(B[4], b, B[5] * c)),
                     fmaf(B[6], a, fmaf(B[7], b, B[8] * c)), 0.0f);
}

__global__ void k_pad4(int64_t N, const float* __restrict__ x, float4* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) y[i] = make_float4(x[3 * i], x[3 * i + 1], x[3 * i + 2], 0.0f);
}

// out <- acc with the Dirichlet rows of J V (= V) for threads i < N; threads N + h write
// the constraint row of hanging node h: out_h = V_h - sum_p w_p V_p (V padded)
__global__ void k_pack_jv4(int64_t N, int64_t H, const uint8_t* __restrict__ faces, BcTable bc,
                           const int32_t* __restrict__ hnode, const int32_t* __restrict__ hpar,
                           const uint8_t* __restrict__ hnp, const float4* __restrict__ V4,
                           const float4* __restrict__ acc, float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) {
    const uint8_t fm = faces[i];
    if (fm & 0x80) return;
    const float4 a = acc[i];
    float r[3] = {a.x, a.y, a.z};
    if (fm & 0x3F) {
      const float4 v = V4[i];
      const float vv[3] = {v.x, v.y, v.z};
#pragma unroll
      for (int f = 0; f < 3; ++f)
        if (fm & bc.dir_faces[f] & 0x3F) r[f] = vv[f];
    }
    out[3 * i] = r[0];
    out[3 * i + 1] = r[1];
    out[3 * i + 2] = r[2];
    return;
  }
  const int64_t h = i - N;
  if (h >= H) return;
  const int np = hnp[h];
  const float wgt = np == 2 ? 0.5f : 0.25f;
  const int64_t id = hnode[h];
  float4 sv = V4[id];
  for (int p = 0; p < np; ++p) {
    const float4 a = V4[hpar[4 * h + p]];
    sv.x -= wgt * a.x; sv.y -= wgt * a.y; sv.z -= wgt * a.z;
  }
  out[3 * id] = sv.x;
  out[3 * id + 1] = sv.y;
  out[3 * id + 2] = sv.z;
}

// Arnoldi bookkeeping of the inner process.  Basis vectors u_i are kept unnormalised
// with norms s_i (q_i = u_i / s_i); the Hessenberg columns are reduced by Givens rotations
// as they arrive, so the least-squares solve at the end is a back-substitution.
// Scalar layout: R [(d+1) x d] row-major, cs[d], sn[d], g[d+1], kv[1] (the number of
// columns before the first breakdown, as a double).
struct InnerScalars {
  double *R, *cs, *sn, *g, *kv;
};
__device__ __forceinline__ InnerScalars inner_scalars(double* base, int d) {
  InnerScalars S;
  S.R = base;
  S.cs = S.R + (size_t)(d + 1) * d;
  S.sn = S.cs + d;
  S.g = S.sn + d;
  S.kv = S.g + (d + 1);
  return S;
}

// sum of the norm partials of k_multi_axpy_norm_f32 in a fixed order (one block of 64)
// sum of the norm partials by one block of kBookThreads threads: every thread issues its
// loads at once (at most four), then a fixed-order tree
constexpr int kBookThreads = 256;
__device__ __forceinline__ double sum_parts(const double* __restrict__ part, int nparts, double* sh) {
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  int b = threadIdx.x;
  for (; b + 3 * kBookThreads < nparts; b += 4 * kBookThreads) {
    t0 += part[b];
    t1 += part[b + kBookThreads];
    t2 += part[b + 2 * kBookThreads];
    t3 += part[b + 3 * kBookThreads];
  }
  for (; b < nparts; b += kBookThreads) t0 += part[b];
  sh[threadIdx.x] = (t0 + t1) + (t2 + t3);
  __syncthreads();
  for (int o = kBookThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

__global__ void __launch_bounds__(kBookThreads) k_inner_start(int d, const double* __restrict__ part, int nparts,
                                                              double* sv, double* dinv, float* inv_s, double* sc) {
  __shared__ double sh[kBookThreads];
  const InnerScalars S = inner_scalars(sc, d);
  for (int i = threadIdx.x; i <= d; i += blockDim.x) S.g[i] = 0.0;
  const double nrm2 = sum_parts(part, nparts, sh);
  if (threadIdx.x == 0) {
    const double s = sqrt(nrm2);
    sv[0] = s;
    dinv[0] = s > 0 ? 1.0 / (s * s) : 0.0;
    inv_s[0] = s > 0 ? (float)(1.0 / s) : 0.0f;
    S.g[0] = s;
    S.kv[0] = 0.0;
  }
}

// column j: h_i = d_i / s_i (i <= j), h_{j+1} = ||u_{j+1}||; apply the earlier rotations,
// make rotation j, update g.  One block of kBookThreads threads (the first kMaxInner hold
// the column).
constexpr int kMaxInner = 64;
static_assert(kBookThreads >= kMaxInner, "one thread per column entry");
__global__ void __launch_bounds__(kBookThreads) k_inner_col(int j, int d, const double* __restrict__ dd,
                                                            const double* __restrict__ part, int nparts, double* sv,
                                                            double* dinv, float* inv_s, double* sc) {
  __shared__ double h[kMaxInner + 1];
  __shared__ double sh[kBookThreads];
  __shared__ double cs[kMaxInner], sn[kMaxInner];
  const InnerScalars S = inner_scalars(sc, d);
  const int i = threadIdx.x;
  if (i <= j) h[i] = sv[i] > 0 ? dd[i] / sv[i] : 0.0;
  if (i < j) {
    cs[i] = S.cs[i];
    sn[i] = S.sn[i];
  }
  const double nrm2 = sum_parts(part, nparts, sh);
  if (i == 0) {
    const double s = sqrt(nrm2);
    h[j + 1] = s;
    sv[j + 1] = s;
    dinv[j + 1] = s > 0 ? 1.0 / (s * s) : 0.0;
    inv_s[j + 1] = s > 0 ? (float)(1.0 / s) : 0.0f;
  }
  __syncthreads();
  if (i != 0) return;
  for (int l = 0; l < j; ++l) {
    const double t = cs[l] * h[l] + sn[l] * h[l + 1];
    h[l + 1] = -sn[l] * h[l] + cs[l] * h[l + 1];
    h[l] = t;
  }
  const double rr = hypot(h[j], h[j + 1]);
  if (rr > 0) {
    S.cs[j] = h[j] / rr;
    S.sn[j] = h[j + 1] / rr;
    h[j] = rr;
    S.g[j + 1] = -S.sn[j] * S.g[j];
    S.g[j] = S.cs[j] * S.g[j];
    if (S.kv[0] == (double)j) S.kv[0] = j + 1;
  } else {
    S.cs[j] = 1.0;
    S.sn[j] = 0.0;
  }
  for (int l = 0; l <= j; ++l) S.R[l * d + j] = h[l];
}

// y = R^-1 g over the columns before the first breakdown; coef_i = y_i / s_i, so that
// sum_i y_i q_i = sum_i coef_i u_i.  The block stages R, g and s in shared memory, then
// one thread back-substitutes.
__global__ void __launch_bounds__(kMaxInner) k_inner_lsq(int d, const double* __restrict__ sv, double* sc,
                                                         double* __restrict__ coef) {
  __shared__ double R[kMaxInner * kMaxInner], g[kMaxInner], y[kMaxInner];
  const InnerScalars S = inner_scalars(sc, d);
  const int k = (int)S.kv[0];
  for (int t = threadIdx.x; t < k * d; t += blockDim.x) R[t] = S.R[t];
  for (int t = threadIdx.x; t < k; t += blockDim.x) g[t] = S.g[t];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < k; ++l) t -= R[i * d + l] * y[l];
      y[i] = t / R[i * d + i];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < d; t += blockDim.x) coef[t] = t < k ? y[t] / sv[t] : 0.0;
}

// out = sum_i coef_i U_i (FP32 vectors, coefficients on the device)
__global__ void k_combine_f32(int64_t n, int k, const float* __restrict__ Ub, int64_t ld,
                              const double* __restrict__ coef, float* __restrict__ out) {
  extern __shared__ float cf[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = (float)coef[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    float v0 = 0.0f, v1 = 0.0f;
    int i = 0;
    for (; i + 2 <= k; i += 2) {
      v0 = fmaf(cf[i], Ub[(int64_t)i * ld + t], v0);
      v1 = fmaf(cf[i + 1], Ub[(int64_t)(i + 1) * ld + t], v1);
    }
    if (i < k) v0 = fmaf(cf[i], Ub[(int64_t)i * ld + t], v0);
    out[t] = v0 + v1;
  }
}

// x += sum_i coef_i Z_i: FP32 vectors combined in FP32, added to an FP64 vector
__global__ void k_combine_f32_add_f64(int64_t n, int k, const float* __restrict__ Zb, int64_t ld,
                                      const double* __restrict__ coef, double* __restrict__ x) {
  extern __shared__ float cf[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = (float)coef[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    float v0 = 0.0f, v1 = 0.0f;
    int i = 0;
    for (; i + 2 <= k; i += 2) {
      v0 = fmaf(cf[i], Zb[(int64_t)i * ld + t], v0);
      v1 = fmaf(cf[i + 1], Zb[(int64_t)(i + 1) * ld + t], v1);
    }
    if (i < k) v0 = fmaf(cf[i], Zb[(int64_t)i * ld + t], v0);
    x[t] += (double)(v0 + v1);
  }
}

// y = scale * (double) x
__global__ void k_to_f64_scaled(int64_t n, const float* __restrict__ x, double scale, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = scale * (double)x[i];
}

}  // namespace

int inner_dot_blocks(int64_t) { return kInnerBlocks; }
int inner_max_depth() { return kMaxInner; }

cudaError_t launch_multi_dot_f32(int64_t n, int k, const float* Ub, int64_t ld, const float* w, double* part, double* d,
                                 cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if ((n | ld) & 3) return cudaErrorInvalidValue;  // rows padded to float4
  const int nb = inner_dot_blocks(n);
  k_multi_dot_f32<<<nb, 256, 0, s>>>(n / 4, k, (const float4*)Ub, ld / 4, (const float4*)w, part);
  note_launch();
  launch_reduce_parts(nb, k, part, d, s);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy_norm_f32(int64_t n, int k, const float* Ub, int64_t ld, const double* d,
                                       const double* dinv, float* w, double* part, cudaStream_t s) {
  if ((n | ld) & 3) return cudaErrorInvalidValue;  // rows padded to float4
  k_multi_axpy_norm_f32<<<kUpdBlocks, 256, (k > 0 ? k : 1) * sizeof(float), s>>>(n / 4, k, (const float4*)Ub, ld / 4,
                                                                                 d, dinv, (float4*)w, part);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_block_apply32(int64_t N, const float* Dinv32, const float* u, const float* inv_s, float* y,
                                 cudaStream_t s) {
  if (N) {
    k_block_apply32<<<nblk(N, 256), 256, 0, s>>>(N, Dinv32, u, inv_s, y);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_block_apply32_pad(int64_t N, const float* Dinv32, const float* u, const float* inv_s, float4* y4,
                                     cudaStream_t s) {
  if (N) {
    k_block_apply32_pad<<<nblk(N, 256), 256, 0, s>>>(N, Dinv32, u, inv_s, y4);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_pad4(int64_t N, const float* x, float4* y4, cudaStream_t s) {
  if (N) {
    k_pad4<<<nblk(N, 256), 256, 0, s>>>(N, x, y4);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_jv4(const RowArgs& R, const float4* V4, const float4* acc4, float* out, cudaStream_t s) {
  if (R.n_nodes + R.n_hanging) {
    k_pack_jv4<<<nblk(R.n_nodes + R.n_hanging, 256), 256, 0, s>>>(R.n_nodes, R.n_hanging, R.faces, R.bc, R.hnode,
                                                                  R.hpar, R.hnp, V4, acc4, out);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_inner_start(int d, const double* part, double* sv, double* dinv, float* inv_s, double* sc,
                               cudaStream_t s) {
  k_inner_start<<<1, kBookThreads, 0, s>>>(d, part, kUpdBlocks, sv, dinv, inv_s, sc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_inner_col(int j, int d, const double* dd, const double* part, double* sv, double* dinv, float* inv_s,
                             double* sc, cudaStream_t s) {
  k_inner_col<<<1, kBookThreads, 0, s>>>(j, d, dd, part, kUpdBlocks, sv, dinv, inv_s, sc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_inner_lsq(int d, const double* sv, double* sc, double* coef, cudaStream_t s) {
  k_inner_lsq<<<1, kMaxInner, 0, s>>>(d, sv, sc, coef);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_combine_f32(int64_t n, int k, const float* Ub, int64_t ld, const double* coef, float* out,
                               cudaStream_t s) {
  k_combine_f32<<<kRedBlocks, 256, (k > 0 ? k : 1) * sizeof(float), s>>>(n, k, Ub, ld, coef, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_combine_f32_add_f64(int64_t n, int k, const float* Zb, int64_t ld, const double* coef, double* x,
                                       cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_combine_f32_add_f64<<<kRedBlocks, 256, k * sizeof(float), s>>>(n, k, Zb, ld, coef, x);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_to_f64_scaled(int64_t n, const float* x, double scale, double* y, cudaStream_t s) {
  k_to_f64_scaled<<<kRedBlocks, 256, 0, s>>>(n, x, scale, y);
  note_launch();
  return cudaGetLastError();
}
