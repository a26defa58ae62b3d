// mlp_tc.cu -- inference of the learned-start network on the fifth-generation tensor
// cores: all four layers of a 128-row tile in one CTA, BF16 operands in shared memory,
// FP32 accumulators in tensor memory (TMEM), bias + GELU epilogues read back with
// tcgen05.ld and written as the next layer's operand, never leaving the SM.
//
// Per CTA (one per SM, persistent over tiles): the four weight matrices stay resident in
// shared memory (K-major, no swizzle: 8x8 core matrices of 128 contiguous bytes); per
// tile the input rows are loaded once, and per layer one thread issues K/16 MMAs of
// 128 x N x 16 (tcgen05.mma kind::f16, BF16 x BF16 -> FP32) and commits them to an
// mbarrier that the epilogue warps wait on (bounded).  Sixteen warps: warp w reads TMEM
// lanes 32 (w mod 4) .. + 31 (the rows it may access) and a quarter of the columns.
#include <cuda_bf16.h>

#include <cstdint>

#include "mlp_tc.h"

#include <mutex>
#include "kernels.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kRows = 128;   // tile rows = MMA M = TMEM lanes
constexpr int kK1 = 224;     // padded input width
constexpr int kHid = 128;
constexpr int kN4 = 16;      // output layer padded to the smallest N of an M = 128 MMA
constexpr int kNo = 3;       // outputs written
constexpr int kLdOut = 8;    // row stride of the output
constexpr int kThreads = 512;
constexpr int kTmemCols = 128;
constexpr int kWaitPolls = 1 << 22;

// shared-memory carve-up (bytes from a 1024-byte aligned base)
constexpr uint32_t kCore = 128;                       // one 8 x 8 BF16 core matrix
constexpr uint32_t kSboK1 = (kK1 / 8) * kCore;        // 8-row group stride, K = 224
constexpr uint32_t kSboHid = (kHid / 8) * kCore;      // 8-row group stride, K = 128
constexpr uint32_t oW1 = 0;                           // [128 n][224 k]
constexpr uint32_t oW2 = oW1 + kHid * kK1 * 2;        // [128][128]
constexpr uint32_t oW3 = oW2 + kHid * kHid * 2;
constexpr uint32_t oW4 = oW3 + kHid * kHid * 2;       // [16][128]
constexpr uint32_t oA = oW4 + kN4 * kHid * 2;         // [128 rows][224] (layer 1), [128][128] (layer 3)
constexpr uint32_t oH = oA + kRows * kK1 * 2;         // [128][128] (layers 2 and 4)
constexpr uint32_t oBar = oH + kRows * kHid * 2;
constexpr uint32_t oTmem = oBar + 8;
constexpr uint32_t kSmemUsed = oTmem + 8;
static_assert(oA % 1024 == 0 && oH % 1024 == 0, "operand tiles aligned");

// byte offset of element (r, k) in a K-major no-swizzle operand whose 8-row groups are
// sbo bytes apart (core matrices along K 128 bytes apart)
__device__ __forceinline__ uint32_t core_off(int r, int k, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 3) * kCore + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// weight W [K][N] row-major (global, BF16) -> K-major operand rows n < N_pad of K
// columns; rows n >= n_src are zero
__device__ void stage_weight(uint8_t* dst, const bf16* __restrict__ W, int K, int n_src, int ldw, int n_pad,
                             uint32_t sbo) {
  const int chunks = n_pad * (K / 8);
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    const int n = i % n_pad, kc = i / n_pad;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (n < n_src) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bf16 lo = W[(int64_t)(kc * 8 + 2 * j) * ldw + n];
        const bf16 hi = W[(int64_t)(kc * 8 + 2 * j + 1) * ldw + n];
        w[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      }
    }
    *reinterpret_cast<uint4*>(dst + core_off(n, kc * 8, sbo)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// bias + GELU of 32 accumulator columns of this thread's row, written as BF16 into the
// next layer's operand (K = 128)
__device__ __forceinline__ void epilogue_gelu(uint32_t tmem_row, int col0, int row, const float* __restrict__ bias,
                                              uint8_t* dst) {
#pragma unroll 1
  for (int c = col0; c < col0 + 32; c += 16) {
    float v[16];
    tmem_ld16(tmem_row + (uint32_t)c, v);
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a = gelu(v[2 * i] + __ldg(bias + c + 2 * i));
      const float b = gelu(v[2 * i + 1] + __ldg(bias + c + 2 * i + 1));
      p[i] = pack_bf16(a, b);
    }
    *reinterpret_cast<uint4*>(dst + core_off(row, c, kSboHid)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4*>(dst + core_off(row, c + 8, kSboHid)) = make_uint4(p[4], p[5], p[6], p[7]);
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_infer_tc(MlpTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar = smem_u32(sm + oBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + oTmem);

  // resident weights
  stage_weight(sm + oW1, a.W1, kK1, kHid, kHid, kHid, kSboK1);
  stage_weight(sm + oW2, a.W2, kHid, kHid, kHid, kHid, kSboHid);
  stage_weight(sm + oW3, a.W3, kHid, kHid, kHid, kHid, kSboHid);
  stage_weight(sm + oW4, a.W4, kHid, kLdOut, kLdOut, kN4, kSboHid);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  // this warp's TMEM lanes (rows) and accumulator column quarter
  const int quarter = warp & 3, part = warp >> 2;
  const int row = quarter * 32 + lane;
  const uint32_t tmem_row = tmem + ((uint32_t)(quarter * 32) << 16);
  const uint32_t sA = smem_u32(sm + oA), sH = smem_u32(sm + oH);
  const uint32_t sW[4] = {smem_u32(sm + oW1), smem_u32(sm + oW2), smem_u32(sm + oW3), smem_u32(sm + oW4)};

  const int64_t n_tiles = (a.rows + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = tile * kRows;
    // input rows -> layer-1 operand; 8 consecutive threads fill one core matrix
    for (int i = tid; i < kRows * (kK1 / 8); i += kThreads) {
      const int r = (i & 7) + 8 * (i / (8 * (kK1 / 8)));
      const int kc = (i >> 3) % (kK1 / 8);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + r < a.rows) v = __ldg(reinterpret_cast<const uint4*>(a.X + (r0 + r) * kK1) + kc);
      *reinterpret_cast<uint4*>(sm + oA + core_off(r, kc * 8, kSboK1)) = v;
    }
    for (int layer = 0; layer < 4; ++layer) {
      fence_async_smem();  // operand writes -> visible to the tensor core
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        const int K = layer == 0 ? kK1 : kHid, N = layer == 3 ? kN4 : kHid;
        const uint32_t src = (layer == 0 || layer == 2) ? sA : sH;
        const uint32_t sbo_a = layer == 0 ? kSboK1 : kSboHid;
        const uint32_t sbo_b = layer == 0 ? kSboK1 : kSboHid;
        const uint32_t idesc = instr_desc(kRows, N);
        for (int k = 0; k < K / 16; ++k)
          mma_bf16(tmem, mat_desc(src + 256u * k, kCore, sbo_a), mat_desc(sW[layer] + 256u * k, kCore, sbo_b), idesc,
                   k > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      const bool ok = mbar_wait(bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      fence_after();
      if (layer < 3) {
        const float* bias = layer == 0 ? a.b1 : layer == 1 ? a.b2 : a.b3;
        uint8_t* dst = sm + ((layer == 1) ? oA : oH);
        epilogue_gelu(tmem_row, part * 32, row, bias, dst);
      } else if (part == 0) {
        float v[4];
        tmem_ld4(tmem_row, v);
        if (r0 + row < a.rows) {
          float* o = a.out + (r0 + row) * kLdOut;
#pragma unroll
          for (int f = 0; f < kNo; ++f) o[f] = v[f] + __ldg(a.b4 + f);
        }
      }
    }
    if (failed) break;
  }
  if (failed) {
    // the tensor core did not signal completion: flag it, give the outstanding MMAs a
    // last bounded wait, then free the tensor memory
    if (tid == 0) {
      atomicOr(a.err, 1);
      mbar_wait(bar, phase ^ 1u);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t mlp_tc_smem_bytes() { return kSmemUsed + 1024; }

cudaError_t launch_mlp_infer_tc(const MlpTcArgs& a, cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  // the SM count and the shared-memory attribute, once per device (the attribute is a
  // per-device setting); only a successful set-up is cached
  static std::mutex mu;
  static int n_sm_of[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  int n_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!n_sm_of[dev]) {
      int n = 0;
      e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_tc_smem_bytes());
      if (e != cudaSuccess) return e;
      n_sm_of[dev] = n;
    }
    n_sm = n_sm_of[dev];
  }
  const int64_t tiles = (a.rows + kRows - 1) / kRows;
  const unsigned blocks = (unsigned)(tiles < n_sm ? tiles : n_sm);
  k_mlp_infer_tc<<<blocks, kThreads, mlp_tc_smem_bytes(), s>>>(a);
  note_launch();
  return cudaGetLastError();
}
