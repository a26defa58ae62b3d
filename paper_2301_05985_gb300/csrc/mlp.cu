// mlp.cu -- learned Newton start: stencil features, a BF16 tensor-core MLP (forward and
// backward through mma.sync m16n8k16, FP32 accumulation), Adam, training on solver
// trajectories, and the judged start of a time step.
//
// The paper has no learned component; this follows the library's own design: a per-node
// network maps the 3x3x3 stencil of (c+, c-, phi, u_z) at t^k and t^{k-1} to the
// correction U^{k+1} - (2 U^k - U^{k-1}); plain Newton judges it against extrapolation.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "mlp_tc.h"

#define CK(call)                                 \
  do {                                           \
    int _rc = ctx_check(c, (call), #call);       \
    if (_rc) return _rc;                         \
  } while (0)
#define RC(call)              \
  do {                        \
    int _rc = (call);         \
    if (_rc) return _rc;      \
  } while (0)

namespace {

constexpr int K0 = 216, K0P = 224, HID = 128, NO = 3, NOP = 8, NPT = 27;
constexpr int64_t oW1 = 0, ob1 = oW1 + (int64_t)K0 * HID, oW2 = ob1 + HID, ob2 = oW2 + (int64_t)HID * HID,
                  oW3 = ob2 + HID, ob3 = oW3 + (int64_t)HID * HID, oW4 = ob3 + HID, ob4 = oW4 + (int64_t)HID * NO,
                  oEnd = ob4 + NO;
static_assert(oEnd == PNP_MLP_PARAMS, "packed parameter count");
constexpr int64_t kMaxRows = 65536;

using bf16 = __nv_bfloat16;

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ features
// Stencil CSR: for free node r and point p, entries [ptr[r*27+p], ptr[r*27+p+1]) of
// (node, weight) whose weighted sum is the Q1 field at the point.
struct FeatArgs {
  int64_t rows;
  int64_t N;                  // nodes per state
  const int32_t* row_slot;    // [rows] free-node slot of each row, or null (row = slot)
  const int64_t* row_state;   // [rows] state index s of U^k in `base`, or null (use Uk/Ukm1)
  const double* base;         // [S][N][3] states (training)
  const double* ubase;        // [S][N] u_z (training) or null
  const double* Uk;           // [N][3] (inference)
  const double* Ukm1;
  const double* uzk;          // [N] or null
  const double* uzkm1;
  const int32_t* ptr;
  const int32_t* idx;
  const double* wt;
  double mu[4], isd[4];       // standardisation of inputs
  float mu_f[4], isd_f[4];    // the same in FP32
  double* raw;                // [rows][216] FP64 (raw mode) or null
  bf16* X;                    // [rows][224] standardised BF16 (or null)
};

// RAW: FP64 features (the parity path); otherwise FP32 accumulation and standardisation,
// rounded to BF16 (GB300 runs FP64 at 1/64 of the FP32 rate, and BF16 keeps 8 bits)
template <bool RAW>
__global__ void k_features(FeatArgs a) {
  using A = typename std::conditional<RAW, double, float>::type;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.rows * NPT) return;
  const int64_t r = t / NPT;
  const int p = (int)(t % NPT);
  const int64_t slot = a.row_slot ? a.row_slot[r] : r;
  const double *U0, *U1, *z0, *z1;
  if (a.row_state) {
    const int64_t s = a.row_state[r];
    U0 = a.base + s * a.N * 3;
    U1 = a.base + (s - 1) * a.N * 3;
    z0 = a.ubase ? a.ubase + s * a.N : nullptr;
    z1 = a.ubase ? a.ubase + (s - 1) * a.N : nullptr;
  } else {
    U0 = a.Uk;
    U1 = a.Ukm1;
    z0 = a.uzk;
    z1 = a.uzkm1;
  }
  A v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int32_t b = a.ptr[slot * NPT + p], e = a.ptr[slot * NPT + p + 1];
  for (int32_t q = b; q < e; ++q) {
    const int64_t id = a.idx[q];
    const A w = (A)a.wt[q];
    for (int f = 0; f < 3; ++f) {
      v[f] += w * (A)U0[3 * id + f];
      v[4 + f] += w * (A)U1[3 * id + f];
    }
    if (z0) v[3] += w * (A)z0[id];
    if (z1) v[7] += w * (A)z1[id];
  }
  for (int g = 0; g < 8; ++g) {
    const int col = g * NPT + p;
    if (RAW) {
      a.raw[r * K0 + col] = (double)v[g];
      if (a.X) a.X[r * K0P + col] = __float2bfloat16((float)((v[g] - a.mu[g & 3]) * a.isd[g & 3]));
    } else if (a.X) {
      a.X[r * K0P + col] = __float2bfloat16((v[g] - a.mu_f[g & 3]) * a.isd_f[g & 3]);
    }
  }
  if (a.X && p < K0P - K0) a.X[r * K0P + K0 + p] = __float2bfloat16(0.f);
}

// standardised training targets: (U^{t+1} - 2 U^t + U^{t-1} - mu) / sd
__global__ void k_targets(int64_t rows, int64_t N, const int32_t* __restrict__ row_slot,
                          const int64_t* __restrict__ row_state, const int32_t* __restrict__ free_nodes,
                          const double* __restrict__ base, double m0, double m1, double m2, double s0, double s1,
                          double s2, float* __restrict__ Y) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t id = free_nodes[row_slot[r]];
  const int64_t s = row_state[r];
  const double* U0 = base + s * N * 3;
  const double mu[3] = {m0, m1, m2}, isd[3] = {1.0 / s0, 1.0 / s1, 1.0 / s2};
  for (int f = 0; f < 3; ++f) {
    const double d = (U0 + N * 3)[3 * id + f] - 2.0 * U0[3 * id + f] + (U0 - N * 3)[3 * id + f];
    Y[r * NOP + f] = (float)((d - mu[f]) * isd[f]);
  }
  for (int f = 3; f < NOP; ++f) Y[r * NOP + f] = 0.f;
}

__global__ void k_f32_to_bf16_rows(int64_t rows, int cols, int ldin, int ldout, const float* __restrict__ in,
                                   bf16* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * ldout) return;
  const int64_t r = t / ldout;
  const int cidx = (int)(t % ldout);
  out[t] = __float2bfloat16(cidx < cols ? in[r * ldin + cidx] : 0.f);
}

__global__ void k_f32_rows(int64_t rows, int cols, int ldin, int ldout, const float* __restrict__ in,
                           float* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * ldout) return;
  const int64_t r = t / ldout;
  const int cidx = (int)(t % ldout);
  out[t] = cidx < cols ? in[r * ldin + cidx] : 0.f;
}

// ------------------------------------------------------------------ GEMM (mma.sync bf16)
enum { EPI_F32 = 0, EPI_FWD_GELU = 1, EPI_BWD_GELU = 2 };

struct GemmArgs {
  int M, N, K;
  const bf16* A;
  int64_t sam, sak;  // A(m,k) = A[m*sam + k*sak]
  const bf16* B;
  int64_t sbk, sbn;  // B(k,n) = B[k*sbk + n*sbn]
  const float* bias; // [N] or null
  float* Cf;
  int64_t ldc;
  bf16* Cb;
  int64_t ldcb;
  const float* Zs;   // saved pre-activation (backward)
  int64_t ldz;
};

constexpr int BM = 64, BN = 64, BK = 32, SPAD = 8;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t ld_b32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A B with a 64x64 block tile, 4 warps of 32x32, BF16 operands staged through shared
// memory (strided global reads, so any operand may be transposed), FP32 accumulation.
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM][BK + SPAD];
  __shared__ __align__(16) bf16 Bs[BN][BK + SPAD];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int i = threadIdx.x; i < BM * BK; i += blockDim.x) {
      int mm, kk;
      if (g.sak == 1) { mm = i / BK; kk = i % BK; } else { kk = i / BM; mm = i % BM; }
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = (m < g.M && k < g.K) ? g.A[(int64_t)m * g.sam + (int64_t)k * g.sak] : zero;
    }
    for (int i = threadIdx.x; i < BN * BK; i += blockDim.x) {
      int nn, kk;
      if (g.sbn == 1) { kk = i / BN; nn = i % BN; } else { nn = i / BK; kk = i % BK; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[nn][kk] = (n < g.N && k < g.K) ? g.B[(int64_t)k * g.sbk + (int64_t)n * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        a[i][0] = ld_b32(&As[r][ks + tig * 2]);
        a[i][1] = ld_b32(&As[r + 8][ks + tig * 2]);
        a[i][2] = ld_b32(&As[r][ks + tig * 2 + 8]);
        a[i][3] = ld_b32(&As[r + 8][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = wn + j * 8 + gid;
        b[j][0] = ld_b32(&Bs[cc][ks + tig * 2]);
        b[j][1] = ld_b32(&Bs[cc][ks + tig * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gid + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = acc[i][j][q];
        if (EPI == EPI_F32) {
          g.Cf[(int64_t)m * g.ldc + n] = v + (g.bias ? g.bias[n] : 0.f);
        } else if (EPI == EPI_FWD_GELU) {
          const float z = v + g.bias[n];
          if (g.Cf) g.Cf[(int64_t)m * g.ldc + n] = z;
          g.Cb[(int64_t)m * g.ldcb + n] = __float2bfloat16(gelu_f(z));
        } else {
          const float dz = v * gelu_prime_f(g.Zs[(int64_t)m * g.ldz + n]);
          g.Cf[(int64_t)m * g.ldc + n] = dz;
          g.Cb[(int64_t)m * g.ldcb + n] = __float2bfloat16(dz);
        }
      }
}

template <int EPI>
cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  k_gemm<EPI><<<grid, 128, 0, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

// loss = mean (out - y)^2 over rows x 3; dOut = 2 (out - y) / (3 rows)
__global__ void k_loss_grad(int64_t rows, const float* __restrict__ out, const float* __restrict__ Y,
                            bf16* __restrict__ dOb, float* __restrict__ dOf, double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0;
  const double scale = 2.0 / (3.0 * (double)rows);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * NOP;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(t % NOP);
    float d = 0.f;
    if (col < NO) {
      const double e = (double)out[t] - (double)Y[t];
      s += e * e;
      d = (float)(scale * e);
    }
    dOb[t] = __float2bfloat16(d);
    dOf[t] = d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// db[n] = sum_r dZ[r][n]  (one block per column, fixed order)
__global__ void k_colsum(int64_t rows, int ld, const float* __restrict__ dZ, float* __restrict__ db) {
  __shared__ float sh[256];
  const int n = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += dZ[r * ld + n];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[n] = sh[0];
}

__global__ void k_adam(int64_t n, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// packed FP32 parameters -> padded BF16 weights and FP32 biases
__global__ void k_refresh(const float* __restrict__ P, bf16* W1, bf16* W2, bf16* W3, bf16* W4, float* b1, float* b2,
                          float* b3, float* b4) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < (int64_t)K0P * HID) {
    const int64_t k = t / HID, n = t % HID;
    W1[t] = __float2bfloat16(k < K0 ? P[oW1 + k * HID + n] : 0.f);
  }
  if (t < (int64_t)HID * HID) {
    W2[t] = __float2bfloat16(P[oW2 + t]);
    W3[t] = __float2bfloat16(P[oW3 + t]);
  }
  if (t < (int64_t)HID * NOP) {
    const int64_t k = t / NOP, n = t % NOP;
    W4[t] = __float2bfloat16(n < NO ? P[oW4 + k * NO + n] : 0.f);
  }
  if (t < HID) {
    b1[t] = P[ob1 + t];
    b2[t] = P[ob2 + t];
    b3[t] = P[ob3 + t];
  }
  if (t < NOP) b4[t] = t < NO ? P[ob4 + t] : 0.f;
}

// U[node] = Uex[node] + sd * out + mu  for the rows' nodes
__global__ void k_apply_correction(int64_t rows, const int32_t* __restrict__ nodes, const float* __restrict__ out,
                                   double m0, double m1, double m2, double s0, double s1, double s2,
                                   const double* __restrict__ Uex, double* __restrict__ U) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t id = nodes[r];
  const double mu[3] = {m0, m1, m2}, sd[3] = {s0, s1, s2};
  for (int f = 0; f < 3; ++f) U[3 * id + f] = Uex[3 * id + f] + sd[f] * (double)out[r * NOP + f] + mu[f];
}

// per-block partial sums (sum, sum of squares) of 4 input fields over states x nodes and
// of 3 target fields over valid (state, node) pairs
__global__ void k_stats(int64_t n_items, int64_t N, const double* __restrict__ base, const double* __restrict__ ub,
                        const uint8_t* __restrict__ valid_state, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc[14];
  for (int q = 0; q < 14; ++q) acc[q] = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_items; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / N, id = t % N;
    const double* U0 = base + s * N * 3;
    for (int f = 0; f < 3; ++f) {
      const double x = U0[3 * id + f];
      acc[2 * f] += x;
      acc[2 * f + 1] += x * x;
    }
    const double u = ub ? ub[s * N + id] : 0.0;
    acc[6] += u;
    acc[7] += u * u;
    if (valid_state[s]) {
      for (int f = 0; f < 3; ++f) {
        const double d = (U0 + N * 3)[3 * id + f] - 2.0 * U0[3 * id + f] + (U0 - N * 3)[3 * id + f];
        acc[8 + 2 * f] += d;
        acc[9 + 2 * f] += d * d;
      }
    }
  }
  for (int q = 0; q < 14; ++q) {
    sh[threadIdx.x] = acc[q];
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * 14 + q] = sh[0];
    __syncthreads();
  }
}

}  // namespace

// ------------------------------------------------------------------ network state
struct Mlp {
  bool trained = false;
  float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr;
  float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr, *b4 = nullptr;
  double in_mu[4] = {0, 0, 0, 0}, in_sd[4] = {1, 1, 1, 1}, out_mu[3] = {0, 0, 0}, out_sd[3] = {1, 1, 1};
  int64_t adam_t = 0;
  // stencil tables
  int64_t n_free = 0;
  int32_t *free_nodes = nullptr, *st_ptr = nullptr, *st_idx = nullptr;
  double* st_w = nullptr;
  // workspace (kMaxRows rows)
  bf16 *X = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr, *dZa = nullptr, *dZb = nullptr, *dOb = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *out = nullptr, *Y = nullptr, *dZf = nullptr, *dOf = nullptr;
  double* part = nullptr;
  int32_t* d_rows = nullptr;
  int64_t* d_state = nullptr;
  // training data
  double* states = nullptr;
  double* uz = nullptr;
  int64_t S = 0, S_cap = 0;
  std::vector<std::pair<int64_t, int64_t>> trajs;  // (first state, T)
  bool have_uz = false;
  // judge bookkeeping: consecutive steps the extrapolated start won, steps left to skip
  int losses = 0, skip = 0;
};

namespace {

void mlp_free(Mlp* m) {
  void* ptrs[] = {m->P,  m->G,  m->Am, m->Av, m->W1, m->W2, m->W3, m->W4, m->b1,     m->b2,      m->b3,
                  m->b4, m->X,  m->A1, m->A2, m->A3, m->dZa, m->dZb, m->dOb, m->Z1,   m->Z2,      m->Z3,
                  m->out, m->Y, m->dZf, m->dOf, m->part, m->d_rows, m->d_state, m->free_nodes, m->st_ptr,
                  m->st_idx, m->st_w, m->states, m->uz};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

// Build the stencil CSR of every non-hanging node (host point location in the Morton-
// ordered leaves, then Q1 weights of the containing leaf with hanging corners resolved).
int build_stencils(pnp_ctx* c, Mlp* m) {
  const pnp_mesh& hm = c->host_mesh;
  const int dim = hm.dim;
  if (dim != 3) PNP_FAIL(PNP_ERR_STATE, "learned start: 3D meshes only");
  const int nc = 8;
  const int64_t size = int64_t(1) << hm.L;
  const int64_t E = hm.n_elem, N = hm.n_nodes;
  std::vector<uint64_t> ekey(E);
  for (int64_t e = 0; e < E; ++e) {
    int64_t a[3] = {hm.el_anchor[e * 3], hm.el_anchor[e * 3 + 1], hm.el_anchor[e * 3 + 2]};
    ekey[e] = pnp_morton(3, a);
  }
  // finest incident element of every node
  std::vector<int64_t> hmin(N, size);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t s = size >> hm.el_level[e];
    for (int cc = 0; cc < nc; ++cc) {
      int32_t id = hm.el_conn[e * nc + cc];
      if (id < 0) id = hm.hang_node[-id - 1];
      hmin[id] = std::min(hmin[id], s);
    }
  }
  std::vector<int32_t> freev;
  for (int64_t i = 0; i < N; ++i)
    if (hm.node_hang[i] < 0) freev.push_back((int32_t)i);
  const int64_t nf = (int64_t)freev.size();
  std::vector<int32_t> ptr(nf * NPT + 1);
  std::vector<int32_t> idx;
  std::vector<double> wt;
  idx.reserve(nf * NPT * 2);
  wt.reserve(nf * NPT * 2);
  ptr[0] = 0;
  for (int64_t r = 0; r < nf; ++r) {
    const int64_t i = freev[r];
    for (int p = 0; p < NPT; ++p) {
      const int off[3] = {p % 3 - 1, (p / 3) % 3 - 1, p / 9 - 1};
      int64_t q[3], ql[3];
      for (int k = 0; k < 3; ++k) {
        q[k] = std::min(std::max((int64_t)hm.node_ijk[i * 3 + k] + off[k] * hmin[i], (int64_t)0), size);
        ql[k] = std::min(q[k], size - 1);
      }
      const uint64_t key = pnp_morton(3, ql);
      int64_t e = (int64_t)(std::upper_bound(ekey.begin(), ekey.end(), key) - ekey.begin()) - 1;
      const int64_t s = size >> hm.el_level[e];
      double t[3];
      for (int k = 0; k < 3; ++k) {
        const int64_t d = q[k] - hm.el_anchor[e * 3 + k];
        if (d < 0 || d > s) PNP_FAIL(PNP_ERR_STATE, "stencil point location failed");
        t[k] = (double)d / (double)s;
      }
      std::vector<std::pair<int32_t, double>> ent;
      for (int cc = 0; cc < nc; ++cc) {
        double w = 1.0;
        for (int k = 0; k < 3; ++k) w *= ((cc >> k) & 1) ? t[k] : 1.0 - t[k];
        if (w == 0.0) continue;
        const int32_t id = hm.el_conn[e * nc + cc];
        if (id >= 0) {
          ent.push_back({id, w});
        } else {
          const int32_t h = -id - 1;
          const int np = hm.hang_np[h];
          for (int pp = 0; pp < np; ++pp) ent.push_back({hm.hang_par[4 * h + pp], w / np});
        }
      }
      std::sort(ent.begin(), ent.end());
      for (size_t k = 0; k < ent.size(); ++k) {
        if (!idx.empty() && (int64_t)idx.size() > ptr[r * NPT + p] && idx.back() == ent[k].first) {
          wt.back() += ent[k].second;
        } else {
          idx.push_back(ent[k].first);
          wt.push_back(ent[k].second);
        }
      }
      ptr[r * NPT + p + 1] = (int32_t)idx.size();
    }
  }
  m->n_free = nf;
  cudaStream_t s = c->stream;
  CK(cudaMalloc((void**)&m->free_nodes, sizeof(int32_t) * std::max<int64_t>(nf, 1)));
  CK(cudaMalloc((void**)&m->st_ptr, sizeof(int32_t) * ptr.size()));
  CK(cudaMalloc((void**)&m->st_idx, sizeof(int32_t) * std::max<size_t>(idx.size(), 1)));
  CK(cudaMalloc((void**)&m->st_w, sizeof(double) * std::max<size_t>(wt.size(), 1)));
  CK(cudaMemcpyAsync(m->free_nodes, freev.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m->st_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m->st_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(m->st_w, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return PNP_OK;
}

int mlp_refresh(pnp_ctx* c, Mlp* m) {
  k_refresh<<<nblk((int64_t)K0P * HID, 256), 256, 0, c->stream>>>(m->P, m->W1, m->W2, m->W3, m->W4, m->b1, m->b2,
                                                                   m->b3, m->b4);
  note_launch();
  return ctx_check(c, cudaGetLastError(), "mlp refresh");
}

FeatArgs feat_args(const Mlp* m, int64_t N) {
  FeatArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = N;
  a.ptr = m->st_ptr;
  a.idx = m->st_idx;
  a.wt = m->st_w;
  for (int f = 0; f < 4; ++f) {
    a.mu[f] = m->in_mu[f];
    a.isd[f] = 1.0 / m->in_sd[f];
    a.mu_f[f] = (float)a.mu[f];
    a.isd_f[f] = (float)a.isd[f];
  }
  return a;
}

GemmArgs gargs(int M, int N, int K, const bf16* A, int64_t sam, int64_t sak, const bf16* B, int64_t sbk, int64_t sbn) {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  return g;
}

// forward of `rows` standardised rows in m->X; output in m->out [rows][8]
int mlp_forward_rows(pnp_ctx* c, Mlp* m, int64_t rows) {
  cudaStream_t s = c->stream;
  const int R = (int)rows;
  GemmArgs g = gargs(R, HID, K0P, m->X, K0P, 1, m->W1, HID, 1);
  g.bias = m->b1; g.Cf = m->Z1; g.ldc = HID; g.Cb = m->A1; g.ldcb = HID;
  CK(gemm<EPI_FWD_GELU>(g, s));
  g = gargs(R, HID, HID, m->A1, HID, 1, m->W2, HID, 1);
  g.bias = m->b2; g.Cf = m->Z2; g.ldc = HID; g.Cb = m->A2; g.ldcb = HID;
  CK(gemm<EPI_FWD_GELU>(g, s));
  g = gargs(R, HID, HID, m->A2, HID, 1, m->W3, HID, 1);
  g.bias = m->b3; g.Cf = m->Z3; g.ldc = HID; g.Cb = m->A3; g.ldcb = HID;
  CK(gemm<EPI_FWD_GELU>(g, s));
  g = gargs(R, NO, HID, m->A3, HID, 1, m->W4, NOP, 1);
  g.bias = m->b4; g.Cf = m->out; g.ldc = NOP;
  CK(gemm<EPI_F32>(g, s));
  return PNP_OK;
}

// inference of `rows` standardised rows in m->X on the tensor cores (tcgen05, all layers
// in one kernel, no saved activations); output in m->out [rows][8]
int mlp_infer_rows(pnp_ctx* c, Mlp* m, int64_t rows) {
  MlpTcArgs a;
  a.rows = rows;
  a.X = m->X;
  a.W1 = m->W1;
  a.W2 = m->W2;
  a.W3 = m->W3;
  a.W4 = m->W4;
  a.b1 = m->b1;
  a.b2 = m->b2;
  a.b3 = m->b3;
  a.b4 = m->b4;
  a.out = m->out;
  a.err = c->dflag + 2;
  CK(launch_mlp_infer_tc(a, c->stream));
  return PNP_OK;
}

// PNP_ERR_DEVICE_FLAG once a wait of the tensor-core inference has given up (latched)
int mlp_check_infer(pnp_ctx* c) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->dflag + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) PNP_FAIL(PNP_ERR_DEVICE_FLAG, "network inference: the tensor core did not signal completion");
  return PNP_OK;
}

// loss and packed gradient for `rows` rows (X, Y in the workspace); loss on the host
int mlp_backward_rows(pnp_ctx* c, Mlp* m, int64_t rows, double* loss) {
  cudaStream_t s = c->stream;
  const int R = (int)rows;
  const int nb = 256;
  k_loss_grad<<<nb, 256, 0, s>>>(rows, m->out, m->Y, m->dOb, m->dOf, m->part);
  note_launch();
  // layer 4
  GemmArgs g = gargs(HID, NO, R, m->A3, 1, HID, m->dOb, NOP, 1);
  g.Cf = m->G + oW4; g.ldc = NO;
  CK(gemm<EPI_F32>(g, s));
  k_colsum<<<NO, 256, 0, s>>>(rows, NOP, m->dOf, m->G + ob4);
  note_launch();
  g = gargs(R, HID, NO, m->dOb, NOP, 1, m->W4, 1, NOP);
  g.Zs = m->Z3; g.ldz = HID; g.Cf = m->dZf; g.ldc = HID; g.Cb = m->dZa; g.ldcb = HID;
  CK(gemm<EPI_BWD_GELU>(g, s));
  // layer 3
  g = gargs(HID, HID, R, m->A2, 1, HID, m->dZa, HID, 1);
  g.Cf = m->G + oW3; g.ldc = HID;
  CK(gemm<EPI_F32>(g, s));
  k_colsum<<<HID, 256, 0, s>>>(rows, HID, m->dZf, m->G + ob3);
  note_launch();
  g = gargs(R, HID, HID, m->dZa, HID, 1, m->W3, 1, HID);
  g.Zs = m->Z2; g.ldz = HID; g.Cf = m->dZf; g.ldc = HID; g.Cb = m->dZb; g.ldcb = HID;
  CK(gemm<EPI_BWD_GELU>(g, s));
  // layer 2
  g = gargs(HID, HID, R, m->A1, 1, HID, m->dZb, HID, 1);
  g.Cf = m->G + oW2; g.ldc = HID;
  CK(gemm<EPI_F32>(g, s));
  k_colsum<<<HID, 256, 0, s>>>(rows, HID, m->dZf, m->G + ob2);
  note_launch();
  g = gargs(R, HID, HID, m->dZb, HID, 1, m->W2, 1, HID);
  g.Zs = m->Z1; g.ldz = HID; g.Cf = m->dZf; g.ldc = HID; g.Cb = m->dZa; g.ldcb = HID;
  CK(gemm<EPI_BWD_GELU>(g, s));
  // layer 1
  g = gargs(K0, HID, R, m->X, 1, K0P, m->dZa, HID, 1);
  g.Cf = m->G + oW1; g.ldc = HID;
  CK(gemm<EPI_F32>(g, s));
  k_colsum<<<HID, 256, 0, s>>>(rows, HID, m->dZf, m->G + ob1);
  note_launch();
  CK(cudaGetLastError());
  if (loss) {
    std::vector<double> hp(nb);
    CK(cudaMemcpyAsync(hp.data(), m->part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double t = 0;
    for (double v : hp) t += v;
    *loss = t / (3.0 * (double)rows);
  }
  return PNP_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
void pnp_mlp_release(pnp_ctx* c) {
  if (c && c->mlp) {
    mlp_free(c->mlp);
    c->mlp = nullptr;
  }
}

// One Adam update of the FP32 master parameters with gradient G (device FP32 [P]), the
// moments and step count carried in the network's state, then the BF16 weight refresh.
static int mlp_adam(pnp_ctx* c, Mlp* m, const float* G, const pnp_train_cfg* cfg) {
  m->adam_t++;
  const float c1 = (float)(1.0 - std::pow(cfg->beta1, (double)m->adam_t));
  const float c2 = (float)(1.0 - std::pow(cfg->beta2, (double)m->adam_t));
  k_adam<<<nblk(PNP_MLP_PARAMS, 256), 256, 0, c->stream>>>(PNP_MLP_PARAMS, m->P, G, m->Am, m->Av, (float)cfg->lr,
                                                          (float)cfg->beta1, (float)cfg->beta2,
                                                          (float)cfg->adam_eps, c1, c2);
  note_launch();
  return mlp_refresh(c, m);
}

#define MLP_GUARD(c)                                                                   \
  do {                                                                                 \
    if (!(c)) PNP_FAIL(PNP_ERR_ARG, "null context");                                   \
    if ((c)->latched != cudaSuccess) PNP_FAIL(PNP_ERR_CUDA, "context latched");        \
    if (!(c)->mlp) PNP_FAIL(PNP_ERR_STATE, "learned start: call pnp_mlp_init first");  \
  } while (0)

extern "C" {

int pnp_mlp_init(pnp_ctx* c, uint64_t seed) {
  if (!c) PNP_FAIL(PNP_ERR_ARG, "null context");
  if (c->latched != cudaSuccess) PNP_FAIL(PNP_ERR_CUDA, "context latched");
  if (c->dim != 3) PNP_FAIL(PNP_ERR_STATE, "learned start: 3D meshes only");
  if (c->host_mesh.periodic) PNP_FAIL(PNP_ERR_ARG, "learned start: periodic meshes are not supported");
  pnp_mlp_release(c);
  Mlp* m = new Mlp();
  c->mlp = m;
  auto fail = [&](int rc) {
    pnp_mlp_release(c);
    return rc;
  };
  const int64_t P = PNP_MLP_PARAMS;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&m->P, 4 * P);
  A((void**)&m->G, 4 * P);
  A((void**)&m->Am, 4 * P);
  A((void**)&m->Av, 4 * P);
  A((void**)&m->W1, 2 * K0P * HID);
  A((void**)&m->W2, 2 * HID * HID);
  A((void**)&m->W3, 2 * HID * HID);
  A((void**)&m->W4, 2 * HID * NOP);
  A((void**)&m->b1, 4 * HID);
  A((void**)&m->b2, 4 * HID);
  A((void**)&m->b3, 4 * HID);
  A((void**)&m->b4, 4 * NOP);
  const size_t R = kMaxRows;
  A((void**)&m->X, 2 * R * K0P);
  A((void**)&m->A1, 2 * R * HID);
  A((void**)&m->A2, 2 * R * HID);
  A((void**)&m->A3, 2 * R * HID);
  A((void**)&m->dZa, 2 * R * HID);
  A((void**)&m->dZb, 2 * R * HID);
  A((void**)&m->dOb, 2 * R * NOP);
  A((void**)&m->Z1, 4 * R * HID);
  A((void**)&m->Z2, 4 * R * HID);
  A((void**)&m->Z3, 4 * R * HID);
  A((void**)&m->out, 4 * R * NOP);
  A((void**)&m->Y, 4 * R * NOP);
  A((void**)&m->dZf, 4 * R * HID);
  A((void**)&m->dOf, 4 * R * NOP);
  A((void**)&m->part, 8 * 256 * 16);
  A((void**)&m->d_rows, 4 * R);
  A((void**)&m->d_state, 8 * R);
  if (e != cudaSuccess) {
    pnp_set_error("pnp_mlp_init: allocation failed: %s", cudaGetErrorString(e));
    return fail(e == cudaErrorMemoryAllocation ? PNP_ERR_NOMEM : PNP_ERR_CUDA);
  }
  // He-normal initialisation (std sqrt(2/fan_in)), zero biases
  std::vector<float> h(P, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  const int64_t wo[4] = {oW1, oW2, oW3, oW4}, fi[4] = {K0, HID, HID, HID}, fo[4] = {HID, HID, HID, NO};
  for (int l = 0; l < 4; ++l)
    for (int64_t i = 0; i < fi[l] * fo[l]; ++i) h[wo[l] + i] = (float)(nd(rng) * std::sqrt(2.0 / fi[l]));
  if (int rc = ctx_check(c, cudaMemcpyAsync(m->P, h.data(), 4 * P, cudaMemcpyHostToDevice, c->stream), "init"))
    return fail(rc);
  cudaMemsetAsync(m->Am, 0, 4 * P, c->stream);
  cudaMemsetAsync(m->Av, 0, 4 * P, c->stream);
  cudaMemsetAsync(m->out, 0, 4 * R * NOP, c->stream);
  if (int rc = mlp_refresh(c, m)) return fail(rc);
  if (int rc = build_stencils(c, m)) return fail(rc);
  return PNP_OK;
}

int pnp_mlp_set_weights(pnp_ctx* c, const float* params, int64_t n) {
  MLP_GUARD(c);
  if (!params || n != PNP_MLP_PARAMS) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_set_weights: need %d floats", PNP_MLP_PARAMS);
  CK(cudaMemcpyAsync(c->mlp->P, params, 4 * n, cudaMemcpyHostToDevice, c->stream));
  RC(mlp_refresh(c, c->mlp));
  CK(cudaStreamSynchronize(c->stream));
  c->mlp->trained = true;
  c->mlp->losses = c->mlp->skip = 0;
  return PNP_OK;
}

int pnp_mlp_get_weights(pnp_ctx* c, float* params, int64_t n) {
  MLP_GUARD(c);
  if (!params || n != PNP_MLP_PARAMS) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_get_weights: need %d floats", PNP_MLP_PARAMS);
  CK(cudaMemcpyAsync(params, c->mlp->P, 4 * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_mlp_set_normalization(pnp_ctx* c, const double* in_mean, const double* in_std, const double* out_mean,
                              const double* out_std) {
  MLP_GUARD(c);
  if (!in_mean || !in_std || !out_mean || !out_std) PNP_FAIL(PNP_ERR_ARG, "null normalisation array");
  for (int f = 0; f < 4; ++f) {
    if (!(in_std[f] > 0)) PNP_FAIL(PNP_ERR_ARG, "input std must be > 0");
    c->mlp->in_mu[f] = in_mean[f];
    c->mlp->in_sd[f] = in_std[f];
  }
  for (int f = 0; f < 3; ++f) {
    if (!(out_std[f] > 0)) PNP_FAIL(PNP_ERR_ARG, "output std must be > 0");
    c->mlp->out_mu[f] = out_mean[f];
    c->mlp->out_sd[f] = out_std[f];
  }
  return PNP_OK;
}

int pnp_mlp_get_normalization(pnp_ctx* c, double* in_mean, double* in_std, double* out_mean, double* out_std) {
  MLP_GUARD(c);
  for (int f = 0; f < 4; ++f) {
    if (in_mean) in_mean[f] = c->mlp->in_mu[f];
    if (in_std) in_std[f] = c->mlp->in_sd[f];
  }
  for (int f = 0; f < 3; ++f) {
    if (out_mean) out_mean[f] = c->mlp->out_mu[f];
    if (out_std) out_std[f] = c->mlp->out_sd[f];
  }
  return PNP_OK;
}

int pnp_mlp_add_trajectory(pnp_ctx* c, const double* states, int64_t T, const double* uz) {
  MLP_GUARD(c);
  if (!states || T < 3) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_add_trajectory: need T >= 3 states");
  Mlp* m = c->mlp;
  const int64_t N = c->n_nodes;
  if (m->S + T > m->S_cap) {
    const int64_t cap = std::max<int64_t>(2 * m->S_cap, m->S + T);
    double *ns = nullptr, *nu = nullptr;
    CK(cudaMalloc((void**)&ns, sizeof(double) * 3 * N * cap));
    CK(cudaMalloc((void**)&nu, sizeof(double) * N * cap));
    if (m->S) {
      CK(cudaMemcpyAsync(ns, m->states, sizeof(double) * 3 * N * m->S, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(nu, m->uz, sizeof(double) * N * m->S, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    if (m->states) cudaFree(m->states);
    if (m->uz) cudaFree(m->uz);
    m->states = ns;
    m->uz = nu;
    m->S_cap = cap;
  }
  CK(cudaMemcpyAsync(m->states + 3 * N * m->S, states, sizeof(double) * 3 * N * T, cudaMemcpyDeviceToDevice,
                     c->stream));
  if (uz) {
    CK(cudaMemcpyAsync(m->uz + N * m->S, uz, sizeof(double) * N * T, cudaMemcpyDeviceToDevice, c->stream));
    m->have_uz = true;
  } else {
    CK(cudaMemsetAsync(m->uz + N * m->S, 0, sizeof(double) * N * T, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  m->trajs.push_back({m->S, T});
  m->S += T;
  return PNP_OK;
}

int pnp_mlp_clear_data(pnp_ctx* c) {
  MLP_GUARD(c);
  c->mlp->trajs.clear();
  c->mlp->S = 0;
  return PNP_OK;
}

int pnp_mlp_features(pnp_ctx* c, const double* Uk, const double* Ukm1, const double* uz_k, const double* uz_km1,
                     double* X, int32_t* nodes) {
  MLP_GUARD(c);
  if (!Uk || !Ukm1 || !X) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_features: null pointer");
  Mlp* m = c->mlp;
  FeatArgs a = feat_args(m, c->n_nodes);
  a.rows = m->n_free;
  a.Uk = Uk;
  a.Ukm1 = Ukm1;
  a.uzk = uz_k;
  a.uzkm1 = uz_km1;
  a.raw = X;
  if (a.rows) {
    if (a.raw) k_features<true><<<nblk(a.rows * NPT, 256), 256, 0, c->stream>>>(a);
    else k_features<false><<<nblk(a.rows * NPT, 256), 256, 0, c->stream>>>(a);
    note_launch();
  }
  CK(cudaGetLastError());
  if (nodes) CK(cudaMemcpyAsync(nodes, m->free_nodes, 4 * m->n_free, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PNP_OK;
}

int pnp_mlp_forward(pnp_ctx* c, const float* X, int64_t B, float* Y) {
  MLP_GUARD(c);
  if (!X || !Y || B < 0) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_forward: bad arguments");
  Mlp* m = c->mlp;
  for (int64_t r0 = 0; r0 < B; r0 += kMaxRows) {
    const int64_t rows = std::min<int64_t>(kMaxRows, B - r0);
    k_f32_to_bf16_rows<<<nblk(rows * K0P, 256), 256, 0, c->stream>>>(rows, K0, K0, K0P, X + r0 * K0, m->X);
    note_launch();
    RC(mlp_infer_rows(c, m, rows));
    k_f32_rows<<<nblk(rows * NO, 256), 256, 0, c->stream>>>(rows, NO, NOP, NO, m->out, Y + r0 * NO);
    note_launch();
  }
  CK(cudaGetLastError());
  return mlp_check_infer(c);
}

int pnp_mlp_loss_grad(pnp_ctx* c, const float* X, const float* Yt, int64_t B, float* grad, double* loss) {
  MLP_GUARD(c);
  if (!X || !Yt || !grad || B <= 0 || B > kMaxRows) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_loss_grad: bad arguments");
  Mlp* m = c->mlp;
  k_f32_to_bf16_rows<<<nblk(B * K0P, 256), 256, 0, c->stream>>>(B, K0, K0, K0P, X, m->X);
  note_launch();
  k_f32_rows<<<nblk(B * NOP, 256), 256, 0, c->stream>>>(B, NO, NO, NOP, Yt, m->Y);
  note_launch();
  RC(mlp_forward_rows(c, m, B));
  double l = 0;
  RC(mlp_backward_rows(c, m, B, &l));
  CK(cudaMemcpyAsync(grad, m->G, 4 * (size_t)PNP_MLP_PARAMS, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (loss) *loss = l;
  return PNP_OK;
}

int pnp_mlp_train(pnp_ctx* c, const pnp_train_cfg* cfg, pnp_train_stats* st) {
  MLP_GUARD(c);
  if (!cfg || cfg->steps < 0 || cfg->batch <= 0 || cfg->batch > kMaxRows || !(cfg->lr > 0))
    PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_train: bad configuration");
  Mlp* m = c->mlp;
  if (m->trajs.empty()) PNP_FAIL(PNP_ERR_STATE, "pnp_mlp_train: no trajectories");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->stream;
  const int64_t N = c->n_nodes;
  // valid U^t: 1 <= t <= T-2 within a trajectory
  std::vector<uint8_t> valid(m->S, 0);
  std::vector<int64_t> vstates;
  for (auto& tr : m->trajs)
    for (int64_t t = 1; t + 1 < tr.second; ++t) {
      valid[tr.first + t] = 1;
      vstates.push_back(tr.first + t);
    }
  if (vstates.empty()) PNP_FAIL(PNP_ERR_STATE, "pnp_mlp_train: trajectories too short");
  // standardisation from the data (states interior to trajectories only for targets)
  {
    uint8_t* dvalid = nullptr;
    CK(cudaMalloc((void**)&dvalid, m->S));
    CK(cudaMemcpyAsync(dvalid, valid.data(), m->S, cudaMemcpyHostToDevice, s));
    // items exclude the first and last state so that the second difference stays in bounds
    const int64_t items = (m->S - 2) * N;
    k_stats<<<256, 256, 0, s>>>(items, N, m->states + 3 * N, m->uz + N, dvalid + 1, m->part);
    note_launch();
    std::vector<double> hp(256 * 14);
    CK(cudaMemcpyAsync(hp.data(), m->part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cudaFree(dvalid);
    double acc[14] = {0};
    for (int b = 0; b < 256; ++b)
      for (int q = 0; q < 14; ++q) acc[q] += hp[b * 14 + q];
    const double n_in = (double)items;
    const double n_out = (double)vstates.size() * (double)N;
    for (int f = 0; f < 4; ++f) {
      const double mu = acc[2 * f] / n_in, var = acc[2 * f + 1] / n_in - mu * mu;
      m->in_mu[f] = mu;
      m->in_sd[f] = var > 1e-24 ? std::sqrt(var) : 1.0;
    }
    for (int f = 0; f < 3; ++f) {
      const double mu = acc[8 + 2 * f] / n_out, var = acc[9 + 2 * f] / n_out - mu * mu;
      m->out_mu[f] = mu;
      m->out_sd[f] = var > 1e-30 ? std::sqrt(var) : 1.0;
    }
  }
  std::mt19937_64 rng(cfg->seed);
  std::uniform_int_distribution<int64_t> pick_state(0, (int64_t)vstates.size() - 1);
  std::uniform_int_distribution<int64_t> pick_node(0, m->n_free - 1);
  const int64_t B = cfg->batch;
  std::vector<int64_t> hs(B);
  std::vector<int32_t> hr(B);
  int64_t* pin_s = nullptr;
  int32_t* pin_r = nullptr;
  CK(cudaMallocHost((void**)&pin_s, 8 * B));
  CK(cudaMallocHost((void**)&pin_r, 4 * B));
  double l_first = 0, l_last = 0;
  int rc = PNP_OK;
  for (int it = 0; it < cfg->steps; ++it) {
    CK(cudaStreamSynchronize(s));  // pinned index buffers are free
    for (int64_t b = 0; b < B; ++b) {
      pin_s[b] = vstates[pick_state(rng)];
      pin_r[b] = (int32_t)pick_node(rng);
    }
    CK(cudaMemcpyAsync(m->d_state, pin_s, 8 * B, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->d_rows, pin_r, 4 * B, cudaMemcpyHostToDevice, s));
    FeatArgs a = feat_args(m, N);
    a.rows = B;
    a.row_slot = m->d_rows;
    a.row_state = m->d_state;
    a.base = m->states;
    a.ubase = m->uz;
    a.X = m->X;
    k_features<false><<<nblk(B * NPT, 256), 256, 0, s>>>(a);
    note_launch();
    k_targets<<<nblk(B, 256), 256, 0, s>>>(B, N, m->d_rows, m->d_state, m->free_nodes, m->states, m->out_mu[0],
                                            m->out_mu[1], m->out_mu[2], m->out_sd[0], m->out_sd[1], m->out_sd[2],
                                            m->Y);
    note_launch();
    if ((rc = mlp_forward_rows(c, m, B))) break;
    double l = 0;
    const bool want = it == 0 || it + 1 == cfg->steps;
    if ((rc = mlp_backward_rows(c, m, B, want ? &l : nullptr))) break;
    if (it == 0) l_first = l;
    if (it + 1 == cfg->steps) l_last = l;
    if ((rc = mlp_adam(c, m, m->G, cfg))) break;
  }
  cudaStreamSynchronize(s);
  cudaFreeHost(pin_s);
  cudaFreeHost(pin_r);
  if (rc) return rc;
  CK(cudaGetLastError());
  m->trained = true;
  m->losses = m->skip = 0;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->loss_first = l_first;
    st->loss_last = l_last;
    st->steps = cfg->steps;
    st->samples = (int64_t)vstates.size() * m->n_free;
    st->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return PNP_OK;
}

int pnp_mlp_adam_step(pnp_ctx* c, const float* grad, const pnp_train_cfg* cfg) {
  MLP_GUARD(c);
  if (!grad || !cfg || !(cfg->lr > 0) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) ||
      !(cfg->adam_eps >= 0))
    PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_adam_step: bad arguments");
  RC(mlp_adam(c, c->mlp, grad, cfg));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->mlp->trained = true;
  return PNP_OK;
}

int pnp_mlp_get_adam_state(pnp_ctx* c, float* m1, float* m2, int64_t* t) {
  MLP_GUARD(c);
  if (m1) CK(cudaMemcpyAsync(m1, c->mlp->Am, 4 * (size_t)PNP_MLP_PARAMS, cudaMemcpyDeviceToHost, c->stream));
  if (m2) CK(cudaMemcpyAsync(m2, c->mlp->Av, 4 * (size_t)PNP_MLP_PARAMS, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (t) *t = c->mlp->adam_t;
  return PNP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free forward
// The network forward of pnp_mlp_forward without a context and without allocating: the
// BF16 weights, the activations and the output rows live in one file-scope device array
// of fixed size (kNoAllocRows rows), shared by every call of this entry point.
namespace {
constexpr int64_t kNoAllocRows = 4096;
struct NoAllocScratch {
  bf16 W1[K0P * HID];
  bf16 W2[HID * HID];
  bf16 W3[HID * HID];
  bf16 W4[HID * NOP];
  float b1[HID], b2[HID], b3[HID], b4[NOP];
  bf16 X[kNoAllocRows * K0P];
  bf16 A1[kNoAllocRows * HID];
  bf16 A2[kNoAllocRows * HID];
  bf16 A3[kNoAllocRows * HID];
  float out[kNoAllocRows * NOP];
};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[128] = {};  // device address of g_noalloc_scratch per device ordinal

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) PNP_FAIL(PNP_ERR_CUDA, "pnp_mlp_forward_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_forward_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      PNP_FAIL(PNP_ERR_CUDA, "pnp_mlp_forward_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<NoAllocScratch*>(g_noalloc_addr[dev]);
  return PNP_OK;
}
}  // namespace

extern "C" int pnp_mlp_forward_noalloc(const float* params, const float* X, int64_t B, float* Y, void* stream) {
  if (!params || B < 0 || (B > 0 && (!X || !Y))) PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_forward_noalloc: null pointer");
  if (B > kNoAllocRows)
    PNP_FAIL(PNP_ERR_ARG, "pnp_mlp_forward_noalloc: %lld rows exceed the fixed scratch of %lld rows; split the call",
             (long long)B, (long long)kNoAllocRows);
  NoAllocScratch* S = nullptr;
  if (int rc = noalloc_scratch(&S)) return rc;
  if (B == 0) return PNP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_refresh<<<nblk((int64_t)K0P * HID, 256), 256, 0, s>>>(params, S->W1, S->W2, S->W3, S->W4, S->b1, S->b2, S->b3,
                                                          S->b4);
  note_launch();
  k_f32_to_bf16_rows<<<nblk(B * K0P, 256), 256, 0, s>>>(B, K0, K0, K0P, X, S->X);
  note_launch();
  const int R = (int)B;
  cudaError_t e = cudaSuccess;
  GemmArgs g = gargs(R, HID, K0P, S->X, K0P, 1, S->W1, HID, 1);
  g.bias = S->b1; g.Cb = S->A1; g.ldcb = HID;
  if (e == cudaSuccess) e = gemm<EPI_FWD_GELU>(g, s);
  g = gargs(R, HID, HID, S->A1, HID, 1, S->W2, HID, 1);
  g.bias = S->b2; g.Cb = S->A2; g.ldcb = HID;
  if (e == cudaSuccess) e = gemm<EPI_FWD_GELU>(g, s);
  g = gargs(R, HID, HID, S->A2, HID, 1, S->W3, HID, 1);
  g.bias = S->b3; g.Cb = S->A3; g.ldcb = HID;
  if (e == cudaSuccess) e = gemm<EPI_FWD_GELU>(g, s);
  g = gargs(R, NO, HID, S->A3, HID, 1, S->W4, NOP, 1);
  g.bias = S->b4; g.Cf = S->out; g.ldc = NOP;
  if (e == cudaSuccess) e = gemm<EPI_F32>(g, s);
  if (e == cudaSuccess) {
    k_f32_rows<<<nblk(B * NO, 256), 256, 0, s>>>(B, NO, NOP, NO, S->out, Y);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) PNP_FAIL(PNP_ERR_CUDA, "pnp_mlp_forward_noalloc: %s", cudaGetErrorString(e));
  return PNP_OK;
}

// Judged learned start of a time step: U <- the best (smallest ||F||) of the network's
// start, the extrapolated start 2 U^k - U^{k-1} and the residual-minimising blend of the
// two; st->start_used says whether a network-based start won.
int pnp_learned_start(pnp_ctx* c, pnp_solve_stats* st) {
  if (!c->mlp || !c->mlp->trained) PNP_FAIL(PNP_ERR_STATE, "learned start: no trained network in this context");
  if (c->step == 0) PNP_FAIL(PNP_ERR_STATE, "learned start: needs two previous time levels");
  Mlp* m = c->mlp;
  // after kJudgeLosses steps in a row won by the extrapolated start, the network (and the
  // judge's residuals) are skipped for kJudgeSkip steps: the extrapolated start is used
  constexpr int kJudgeLosses = 3, kJudgeSkip = 4;
  if (m->skip > 0) {
    --m->skip;
    st->start_used = PNP_START_EXTRAPOLATE;
    st->res_start_learned = -1.0;  // not evaluated
    return PNP_OK;
  }
  cudaStream_t s = c->stream;
  const int64_t N = c->n_nodes, n = c->n3();
  // extrapolated start in Ut (consistent)
  CK(launch_axpbyz(n, 2.0, c->Uk, -1.0, c->Ukm1, c->Ut, s));
  CK(launch_make_consistent(c->rows(), c->Ut, s));
  // network start in U
  CK(cudaMemcpyAsync(c->U, c->Ut, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  // last-axis velocity component of v^k and v^{k-1} (strided view through scratch)
  double* uzk = c->w;
  double* uzkm1 = c->w + N;
  {
    const int d = c->dim - 1;
    CK(cudaMemcpy2DAsync(uzk, sizeof(double), c->vel + d, 3 * sizeof(double), sizeof(double), N,
                         cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy2DAsync(uzkm1, sizeof(double), c->vel_prev + d, 3 * sizeof(double), sizeof(double), N,
                         cudaMemcpyDeviceToDevice, s));
  }
  // features, network and correction; algorithmic bytes per free node: U^k, U^{k-1}
  // and u_z read once (64 B), the extrapolated start read and the start written (48 B);
  // flops: the four layers
  {
    ProfScope ps(c, PNP_PROF_MLP, (64.0 + 48.0) * m->n_free,
                 2.0 * m->n_free * (double)(K0 * HID + 2 * HID * HID + HID * NO));
    for (int64_t r0 = 0; r0 < m->n_free; r0 += kMaxRows) {
      const int64_t rows = std::min<int64_t>(kMaxRows, m->n_free - r0);
      FeatArgs a = feat_args(m, N);
      a.rows = rows;
      a.row_slot = nullptr;
      a.ptr = m->st_ptr + r0 * NPT;  // rows are consecutive free-node slots
      a.Uk = c->Uk;
      a.Ukm1 = c->Ukm1;
      a.uzk = uzk;
      a.uzkm1 = uzkm1;
      a.X = m->X;
      k_features<false><<<nblk(rows * NPT, 256), 256, 0, s>>>(a);
      note_launch();
      RC(mlp_infer_rows(c, m, rows));
      k_apply_correction<<<nblk(rows, 256), 256, 0, s>>>(rows, m->free_nodes + r0, m->out, m->out_mu[0], m->out_mu[1],
                                                         m->out_mu[2], m->out_sd[0], m->out_sd[1], m->out_sd[2], c->Ut,
                                                         c->U);
      note_launch();
    }
  }
  CK(cudaGetLastError());
  RC(mlp_check_infer(c));
  CK(launch_make_consistent(c->rows(), c->U, s));
  // judge with the residual
  RC(ctx_prepare_history(c));
  double fl, fe;
  RC(ctx_residual(c, c->U, c->F));
  RC(ctx_norm(c, c->F, &fl));
  RC(ctx_residual(c, c->Ut, c->Ft));
  RC(ctx_norm(c, c->Ft, &fe));
  // residual-minimising blend U_b = U_e + a (U_l - U_e): over this short segment F is
  // close to linear, so ||F_e + a (F_l - F_e)|| is least near a* = <F_e, D> / ||D||^2
  // with D = F_e - F_l; a* is checked with one more residual
  double fb = INFINITY;
  if (std::isfinite(fl)) {
    double* D = c->w;
    CK(launch_axpbyz(n, 1.0, c->Ft, -1.0, c->F, D, s));
    double dn, ed;
    RC(ctx_norm(c, D, &dn));
    RC(ctx_dot(c, c->Ft, D, &ed));
    const double a = dn > 0 ? std::min(std::max(ed / (dn * dn), 0.0), 2.0) : 0.0;
    if (a > 0.02 && std::fabs(a - 1.0) > 0.02) {
      CK(launch_axpbyz(n, 1.0 - a, c->Ut, a, c->U, c->dU, s));
      RC(ctx_residual(c, c->dU, c->F));
      RC(ctx_norm(c, c->F, &fb));
    }
  }
  st->res_start_extrapolated = fe;
  if (std::isfinite(fb) && fb < fe && fb < fl) {
    st->start_used = PNP_START_LEARNED;
    st->res_start_learned = fb;
    CK(cudaMemcpyAsync(c->U, c->dU, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else if (std::isfinite(fl) && fl < fe) {
    st->start_used = PNP_START_LEARNED;
    st->res_start_learned = fl;
  } else {
    st->start_used = PNP_START_EXTRAPOLATE;
    st->res_start_learned = std::isfinite(fb) ? std::min(fl, fb) : fl;
    CK(cudaMemcpyAsync(c->U, c->Ut, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (st->start_used == PNP_START_LEARNED) {
    m->losses = 0;
  } else if (++m->losses >= kJudgeLosses) {
    m->losses = 0;
    m->skip = kJudgeSkip;
  }
  CK(cudaStreamSynchronize(s));
  return PNP_OK;
}
