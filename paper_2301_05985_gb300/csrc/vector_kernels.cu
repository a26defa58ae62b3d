// vector_kernels.cu -- streaming kernels of the Newton-Krylov loop (history, conversions,
// deterministic FP64 reductions, Gram-Schmidt multi-dot / multi-axpy, 3x3 block Jacobi).
// All of these are HBM-bound: one coalesced pass over their operands.
#include <algorithm>
#include <atomic>

#include "kernels.h"

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }
extern "C" int64_t pnp_kernel_launches(void) { return g_launches.load(); }
static std::atomic<int64_t> g_captures{0};
void note_capture() { g_captures.fetch_add(1, std::memory_order_relaxed); }
extern "C" int64_t pnp_graph_captures(void) { return g_captures.load(); }

namespace {

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }
inline int gs_blocks(int64_t n, int t) {
  const int64_t b = (n + t - 1) / t;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

__global__ void k_history(int64_t N, const double* __restrict__ Uk, const double* __restrict__ Ukm1, double b1,
                          double b2, double inv_dt, double* __restrict__ hs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  hs[2 * i + 0] = (b1 * Uk[3 * i + 0] + b2 * Ukm1[3 * i + 0]) * inv_dt;
  hs[2 * i + 1] = (b1 * Uk[3 * i + 1] + b2 * Ukm1[3 * i + 1]) * inv_dt;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_to_f64(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
// b = 0 does not read y (it may hold any bit pattern, NaN included: 0 * NaN is NaN)
__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}
__global__ void k_axpbyz(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                         double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
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

__global__ void __launch_bounds__(kRedThreads) k_dot_part(int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// one block per output: out[j] = sum_b part[b*k + j]  (optionally sqrt)
__global__ void __launch_bounds__(kRedThreads) k_reduce_parts(int nparts, int k, const double* __restrict__ part,
                                                              double* __restrict__ out, int take_sqrt) {
  __shared__ double sh[kRedThreads];
  const int j = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(int64_t)b * k + j];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[j] = take_sqrt ? sqrt(s) : s;
}

// Sum over the warp of four per-lane values at once (reduce-scatter: 6 adds per lane
// instead of 4 x 5); lanes 8q .. 8q+7 end with the total of s[q].  Fixed order.
__device__ __forceinline__ double warp_sum4(const double (&s)[4], int lane) {
  const bool hi4 = lane & 16, hi3 = lane & 8;
  const double a0 = (hi4 ? s[2] : s[0]) + __shfl_xor_sync(0xffffffffu, hi4 ? s[0] : s[2], 16);
  const double a1 = (hi4 ? s[3] : s[1]) + __shfl_xor_sync(0xffffffffu, hi4 ? s[1] : s[3], 16);
  double b = (hi3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, hi3 ? a0 : a1, 8);
  b += __shfl_xor_sync(0xffffffffu, b, 4);
  b += __shfl_xor_sync(0xffffffffu, b, 2);
  b += __shfl_xor_sync(0xffffffffu, b, 1);
  return b;
}

// d_i = V_i . w (i < k; and w . w as entry k when kk > k).  Each block owns a contiguous
// chunk of kMdRows x 256 rows: w's rows stay in registers while the block sweeps the basis
// four vectors at a time (4 x kMdRows independent loads per thread, one reduce-scatter
// over the warp, fixed order).  The FP64 pipe bounds the kernel on GB300, so the rows per
// thread are many enough that the reduction adds stay small next to the FMAs.  Per-block
// partials part[block][kk].
constexpr int kMdRows = 16;
__global__ void __launch_bounds__(256, 4) k_multi_dot2(int64_t n, int k, int kk, const double* __restrict__ Vb,
                                                    int64_t ld, const double* __restrict__ w,
                                                    double* __restrict__ part) {
  __shared__ double sh[64][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * (256 * kMdRows) + threadIdx.x;
  double wv[kMdRows];
#pragma unroll
  for (int r = 0; r < kMdRows; ++r) {
    const int64_t t = base + r * 256;
    wv[r] = t < n ? w[t] : 0.0;
  }
  for (int i0 = 0; i0 < kk; i0 += 64) {
    const int cnt = min(64, kk - i0);
    // four basis vectors per pass: 4 x kMdRows independent loads, four interleaved shuffle trees
    for (int j0 = 0; j0 < cnt; j0 += 4) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + j0 + q;
        if (j0 + q < cnt) {
          const double* vi = i < k ? Vb + (int64_t)i * ld : w;
#pragma unroll
          for (int r = 0; r < kMdRows; ++r) {
            const int64_t t = base + r * 256;
            if (t < n) s[q] = fma(__ldg(vi + t), wv[r], s[q]);
          }
        }
      }
      const double tot = warp_sum4(s, lane);
      const int q = (lane >> 3) & 3;
      if ((lane & 7) == 0 && j0 + q < cnt) sh[j0 + q][wid] = tot;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) s += sh[j][q];
      part[(int64_t)blockIdx.x * kk + i0 + j] = s;
    }
    __syncthreads();
  }
}

// w -= sum_i (d_i * dinv_i) V_i  and per-block partial sums of the updated w . w
__global__ void __launch_bounds__(kRedThreads) k_multi_axpy_norm(int64_t n, int k, const double* __restrict__ Vb,
                                                                 int64_t ld, const double* __restrict__ d,
                                                                 const double* __restrict__ dinv,
                                                                 double* __restrict__ w, double* __restrict__ part) {
  extern __shared__ double cf[];
  __shared__ double sh[kRedThreads];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = d[i] * dinv[i];
  __syncthreads();
  double ss = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    // two independent chains (the loads are independent anyway); one add to join them
    double v0 = w[t], v1 = 0.0;
    int i = 0;
    for (; i + 2 <= k; i += 2) {
      v0 -= cf[i] * Vb[(int64_t)i * ld + t];
      v1 -= cf[i + 1] * Vb[(int64_t)(i + 1) * ld + t];
    }
    if (i < k) v0 -= cf[i] * Vb[(int64_t)i * ld + t];
    const double v = v0 + v1;
    w[t] = v;
    ss += v * v;
  }
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = ss;
}

__global__ void __launch_bounds__(256) k_multi_axpy(int64_t n, int k, const double* __restrict__ Vb, int64_t ld,
                                                    const double* __restrict__ h, double* __restrict__ w,
                                                    double* __restrict__ hacc) {
  extern __shared__ double hs[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  if (hacc && blockIdx.x == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) hacc[i] += hs[i];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double v = w[t];
    for (int i = 0; i < k; ++i) v -= hs[i] * Vb[(int64_t)i * ld + t];
    w[t] = v;
  }
}

__global__ void k_block_apply(int64_t N, const double* __restrict__ Dinv, const double* __restrict__ v, double scale,
                              double* __restrict__ z, float* __restrict__ z32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* B = Dinv + 9 * i;
  const double a = scale * v[3 * i], b = scale * v[3 * i + 1], c = scale * v[3 * i + 2];
  const double r0 = B[0] * a + B[1] * b + B[2] * c;
  const double r1 = B[3] * a + B[4] * b + B[5] * c;
  const double r2 = B[6] * a + B[7] * b + B[8] * c;
  if (z) {
    z[3 * i] = r0;
    z[3 * i + 1] = r1;
    z[3 * i + 2] = r2;
  }
  if (z32) {
    z32[3 * i] = (float)r0;
    z32[3 * i + 1] = (float)r1;
    z32[3 * i + 2] = (float)r2;
  }
}

template <typename T>
__global__ void k_block_invert(int64_t N, const T* D, double* Dinv, int* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double a[3][6];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      a[r][c] = (double)D[9 * i + 3 * r + c];
      a[r][3 + c] = (r == c) ? 1.0 : 0.0;
    }
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0 || !isfinite(a[piv][col])) {
      atomicOr(flag, 1);
      return;
    }
    if (piv != col)
      for (int c = 0; c < 6; ++c) {
        const double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    const double inv = 1.0 / a[col][col];
    for (int c = 0; c < 6; ++c) a[col][c] *= inv;
    for (int r = 0; r < 3; ++r)
      if (r != col) {
        const double f = a[r][col];
        for (int c = 0; c < 6; ++c) a[r][c] -= f * a[col][c];
      }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Dinv[9 * i + 3 * r + c] = a[r][3 + c];
}

__global__ void k_set_dirichlet(int64_t N, const uint8_t* __restrict__ faces, BcTable bc, double* __restrict__ U) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint8_t fm = faces[i];
  if (fm & 0x80) return;
  for (int f = 0; f < 3; ++f) {
    const unsigned msk = fm & bc.dir_faces[f] & 0x3F;
    if (msk) U[3 * i + f] = bc.val[31 - __clz(msk)][f];
  }
}

__global__ void k_interp_hanging(int64_t H, const int32_t* __restrict__ hnode, const int32_t* __restrict__ hpar,
                                 const uint8_t* __restrict__ hnp, double* __restrict__ U) {
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= H) return;
  const int np = hnp[h];
  const double wgt = np == 2 ? 0.5 : 0.25;
  for (int f = 0; f < 3; ++f) {
    double s = 0;
    for (int p = 0; p < np; ++p) s += wgt * U[3 * (int64_t)hpar[4 * h + p] + f];
    U[3 * (int64_t)hnode[h] + f] = s;
  }
}

__global__ void k_vel_pack(int64_t N, int dim, const double* __restrict__ src, double* __restrict__ dst3) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int k = 0; k < 3; ++k) dst3[3 * i + k] = k < dim ? src[dim * i + k] : 0.0;
}
__global__ void k_vel_unpack(int64_t N, int dim, const double* __restrict__ src3, double* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int k = 0; k < dim; ++k) dst[dim * i + k] = src3[3 * i + k];
}

}  // namespace

cudaError_t launch_history(int64_t N, const double* Uk, const double* Ukm1, double b1, double b2, double dt,
                           double* hs, cudaStream_t s) {
  if (N) { k_history<<<nblk(N, 256), 256, 0, s>>>(N, Uk, Ukm1, b1, b2, 1.0 / dt, hs); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  if (n) { k_to_f32<<<gs_blocks(n, 256), 256, 0, s>>>(n, x, y); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_to_f64(int64_t n, const float* x, double* y, cudaStream_t s) {
  if (n) { k_to_f64<<<gs_blocks(n, 256), 256, 0, s>>>(n, x, y); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s) {
  if (n) { k_axpby<<<gs_blocks(n, 256), 256, 0, s>>>(n, a, x, b, y); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_axpbyz(int64_t n, double a, const double* x, double b, const double* y, double* z, cudaStream_t s) {
  if (n) { k_axpbyz<<<gs_blocks(n, 256), 256, 0, s>>>(n, a, x, b, y, z); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* part, double* result, cudaStream_t s) {
  k_dot_part<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, y, part); note_launch();
  k_reduce_parts<<<1, kRedThreads, 0, s>>>(kRedBlocks, 1, part, result, 0); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_norm2(int64_t n, const double* x, double* part, double* result, cudaStream_t s) {
  k_dot_part<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, x, part); note_launch();
  k_reduce_parts<<<1, kRedThreads, 0, s>>>(kRedBlocks, 1, part, result, 1); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_multi_axpy(int64_t n, int k, const double* Vb, int64_t ld, const double* h, double* w,
                              double* hacc, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_multi_axpy<<<gs_blocks(n, 256), 256, k * sizeof(double), s>>>(n, k, Vb, ld, h, w, hacc); note_launch();
  return cudaGetLastError();
}
__global__ void k_node_records(int64_t N, const double* __restrict__ U, const double* __restrict__ hs,
                               const double* __restrict__ adv, float4* __restrict__ rec) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  rec[2 * i] = make_float4((float)U[3 * i], (float)U[3 * i + 1], (float)U[3 * i + 2], (float)hs[2 * i]);
  rec[2 * i + 1] = make_float4((float)hs[2 * i + 1], (float)adv[3 * i], (float)adv[3 * i + 1], (float)adv[3 * i + 2]);
}

cudaError_t launch_node_records(int64_t N, const double* U, const double* hs, const double* adv, float4* rec,
                                cudaStream_t s) {
  if (N) {
    k_node_records<<<nblk(N, 256), 256, 0, s>>>(N, U, hs, adv, rec);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_parts(int nparts, int k, const double* part, double* out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_reduce_parts<<<k, kRedThreads, 0, s>>>(nparts, k, part, out, 0);
  note_launch();
  return cudaGetLastError();
}

int multi_dot_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + 256 * kMdRows - 1) / (256 * kMdRows)); }

cudaError_t launch_multi_dot_ext(int64_t n, int k, bool with_self, const double* Vb, int64_t ld, const double* w,
                                 double* part, double* d, cudaStream_t s) {
  const int kk = k + (with_self ? 1 : 0);
  if (kk <= 0) return cudaSuccess;
  const int nb = multi_dot_blocks(n);
  k_multi_dot2<<<nb, 256, 0, s>>>(n, k, kk, Vb, ld, w, part); note_launch();
  k_reduce_parts<<<kk, kRedThreads, 0, s>>>(nb, kk, part, d, 0); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_multi_axpy_norm(int64_t n, int k, const double* Vb, int64_t ld, const double* d, const double* dinv,
                                   double* w, double* part, double* nrm2, cudaStream_t s) {
  k_multi_axpy_norm<<<kRedBlocks, kRedThreads, (k > 0 ? k : 1) * sizeof(double), s>>>(n, k, Vb, ld, d, dinv, w, part);
  note_launch();
  k_reduce_parts<<<1, kRedThreads, 0, s>>>(kRedBlocks, 1, part, nrm2, 0); note_launch();
  return cudaGetLastError();
}
cudaError_t launch_block_apply(int64_t N, const double* Dinv, const double* v, double scale, double* z, float* z32,
                               cudaStream_t s) {
  if (N) { k_block_apply<<<nblk(N, 256), 256, 0, s>>>(N, Dinv, v, scale, z, z32); note_launch(); }
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_block_invert(int64_t N, const T* D, double* Dinv, int* flag, cudaStream_t s) {
  if (N) { k_block_invert<T><<<nblk(N, 128), 128, 0, s>>>(N, D, Dinv, flag); note_launch(); }
  return cudaGetLastError();
}
template cudaError_t launch_block_invert<double>(int64_t, const double*, double*, int*, cudaStream_t);
template cudaError_t launch_block_invert<float>(int64_t, const float*, double*, int*, cudaStream_t);
cudaError_t launch_make_consistent(const RowArgs& R, double* U, cudaStream_t s) {
  if (R.n_nodes) { k_set_dirichlet<<<nblk(R.n_nodes, 256), 256, 0, s>>>(R.n_nodes, R.faces, R.bc, U); note_launch(); }
  if (R.n_hanging) { k_interp_hanging<<<nblk(R.n_hanging, 256), 256, 0, s>>>(R.n_hanging, R.hnode, R.hpar, R.hnp, U); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_vel_pack(int64_t N, int dim, const double* src, double* dst3, cudaStream_t s) {
  if (N) { k_vel_pack<<<nblk(N, 256), 256, 0, s>>>(N, dim, src, dst3); note_launch(); }
  return cudaGetLastError();
}
cudaError_t launch_vel_unpack(int64_t N, int dim, const double* src3, double* dst, cudaStream_t s) {
  if (N) { k_vel_unpack<<<nblk(N, 256), 256, 0, s>>>(N, dim, src3, dst); note_launch(); }
  return cudaGetLastError();
}
