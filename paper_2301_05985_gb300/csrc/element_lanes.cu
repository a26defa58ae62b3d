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
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "df32.cuh"
#include "kernels.h"
#include "lane_ops.cuh"

namespace {

// blocks per SM the lane kernel's register cap is set for
template <typename T, typename C>
constexpr int lane_min_blocks() {
  return sizeof(T) == 4 ? 5 : (std::is_same<C, df>::value ? 4 : 3);
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

// the same in arithmetic type C from storage type T
template <typename T, typename C, int NF>
__device__ __forceinline__ void load_node_c(const ElemArgs<T>& A, int32_t id, bool valid, const T* __restrict__ src,
                                            int stride, C (&dst)[NF]) {
#pragma unroll
  for (int f = 0; f < NF; ++f) dst[f] = C(0);
  if (!valid) return;
  if (id >= 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) dst[f] = to_compute<C>(__ldg(src + (int64_t)stride * id + f));
  } else {
    const int32_t h = -id - 1;
    const int np = A.hang_np[h];
    const C wgt = np == 2 ? C(0.5) : C(0.25);
    for (int p = 0; p < np; ++p) {
      const int32_t pid = A.hang_par[4 * h + p];
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[f] += wgt * to_compute<C>(__ldg(src + (int64_t)stride * pid + f));
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

// U-dependent quantities at this lane's Gauss point: values and gradients of c+-, grad
// phi, the advection v, the history h, tau_c, R_s and P_s = v - z_s grad phi
template <typename T, int D>
__device__ __forceinline__ void lane_state(const T (&un)[3], const T (&vn)[3], const T (&hn)[2], T nb,
                                           const T (&sh)[3], T kappa, T tau0, T G2, T (&cv)[2], T (&gc)[2][3],
                                           T (&gp)[3], T (&v)[3], T (&hq)[2], T& tau, T (&R)[2], T (&P)[2][3]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    interp_vg<T, D>(un[s], nb, sh, cv[s], gc[s]);
    hq[s] = interp_v<T, D>(hn[s], nb);
  }
  interp_g<T, D>(un[2], nb, sh, gp);
  T vv = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = interp_v<T, D>(vn[k], nb);
    vv = fma(v[k], v[k], vv);
  }
  tau = inv_sqrt(tau0 + G2 * vv);
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

// T: storage type of the vectors; C: arithmetic type (T, or double-float for FP64 data)
template <typename T, typename C, int D, bool JV>
__global__ void __launch_bounds__(256, lane_min_blocks<T, C>()) k_element_lanes(ElemArgs<T> A, LaneParams<C> K) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // warps whose first element is past the end leave together (shuffles need the warp)
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;
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
  const C G2 = pow2i(2 * lev + 2, C(0));  // (2/h)^2
  const C kappa = K.kappa;
  const C tau0 = fma(K.cid * G2, G2, K.tau_t);
  const C e2 = K.e2;

  C un[3], vn[3], hn[2];
  if constexpr (sizeof(T) == 4) {
    if (A.rec) {
      load_record(A, id, valid, un, hn, vn);
    } else {
      load_node_c<T, C, 3>(A, id, valid, A.U, 3, un);
      load_node_c<T, C, 3>(A, id, valid, A.adv, 3, vn);
      load_node_c<T, C, 2>(A, id, valid, A.hs, 2, hn);
    }
  } else {
    load_node_c<T, C, 3>(A, id, valid, A.U, 3, un);
    load_node_c<T, C, 3>(A, id, valid, A.adv, 3, vn);
    load_node_c<T, C, 2>(A, id, valid, A.hs, 2, hn);
  }

  // state at this lane's Gauss point
  C cv[2], gc[2][3], gp[3], v[3], hq[2], tau, R[2], P[2][3];
  lane_state<C, D>(un, vn, hn, nb, sh, kappa, tau0, G2, cv, gc, gp, v, hq, tau, R, P);

  C S[3], Phi[3][3];
  if constexpr (!JV) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C z = s == 0 ? C(1) : C(-1);
      C vg = C(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) vg = fma(v[k], gc[s][k], vg);
      S[s] = fma(kappa, cv[s], hq[s] + vg);
      const C tR = tau * R[s];
      const C zc = z * cv[s];
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[s][k] = fma(tR, P[s][k], fma(zc, gp[k], gc[s][k]));
    }
    S[2] = fma(tau, R[0] - R[1], cv[1] - cv[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Phi[2][k] = e2 * gp[k];
  } else {
    C dn[3];
    if constexpr (sizeof(T) == 4) {
      if (A.V4) load_dir4(A, id, valid, dn);
      else load_node_c<T, C, 3>(A, id, valid, A.V, 3, dn);
    } else {
      load_node_c<T, C, 3>(A, id, valid, A.V, 3, dn);
    }
    C dcv[2], dgc[2][3], dgp[3], dR[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) interp_vg<C, D>(dn[s], nb, sh, dcv[s], dgc[s]);
    interp_g<C, D>(dn[2], nb, sh, dgp);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const C z = s == 0 ? C(1) : C(-1);
      C vg = C(0), pg = C(0), gcd = C(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        vg = fma(v[k], dgc[s][k], vg);
        pg = fma(P[s][k], dgc[s][k], pg);
        gcd = fma(gc[s][k], dgp[k], gcd);
      }
      dR[s] = fma(kappa, dcv[s], pg - z * gcd);
      S[s] = fma(kappa, dcv[s], vg);
      const C tdR = tau * dR[s];
      const C zdc = z * dcv[s];
      const C zc_tR = z * (cv[s] - tau * R[s]);
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[s][k] = fma(tdR, P[s][k], fma(zc_tR, dgp[k], fma(zdc, gp[k], dgc[s][k])));
    }
    S[2] = fma(tau, dR[0] - dR[1], dcv[1] - dcv[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Phi[2][k] = e2 * dgp[k];
  }

  C r[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) r[f] = w * test_t<C, D>(S[f], Phi[f], nb, sh);
  if (!valid) return;
  if constexpr (sizeof(T) == 4) {
    if (A.out4) {
      scatter4(A, id, r);
      return;
    }
  }
  T ro[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) ro[f] = to_storage<T>(r[f]);
  if (id >= 0) {
#pragma unroll
    for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)id + f, ro[f]);
  } else {
    const int32_t hh = -id - 1;
    const int np = A.hang_np[hh];
    const T wgt = np == 2 ? T(0.5) : T(0.25);
    for (int p = 0; p < np; ++p) {
      const int32_t pid = A.hang_par[4 * hh + p];
#pragma unroll
      for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)pid + f, wgt * ro[f]);
    }
  }
}

// ---- FP32 J V from a stored linearisation ---------------------------------------
// Inside one Krylov solve the state (U, h, v) is fixed, so the Gauss-point quantities J V
// needs from it are computed once per solve and stored per lane, NR float4 in lane-major
// order (qp[j * L + t], L = 2^d E).  With advection (NR = 4): (v0 v1 v2 gp0)
// (gp1 gp2 gc+0 gc+1) (gc+2 gc-0 gc-1 gc-2) (tau, z+(c+ - tau R+), z-(c- - tau R-), level).
// Without (the advection field is zero, NR = 3): (gp0 gp1 gp2 gc+0) (gc+1 gc+2 gc-0 gc-1)
// (gc-2, z+(c+ - tau R+), z-(c- - tau R-), level), and tau = (4/dt^2 + C_I d (2/h)^4)^(-1/2)
// is recomputed from the level (the same FP32 value: |v|^2 = 0).  The level is stored as
// integer bits.  Each J V then reads 16 NR bytes per lane, coalesced, instead of gathering
// and interpolating the state.
constexpr int kLaneThreads = 256;

template <int D, int NR>
__global__ void __launch_bounds__(kLaneThreads, 5) k_lane_state(ElemArgs<float> A, LaneParams<float> K, float4* qp) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;
  const int64_t e = t / NC;
  const int c = (int)(t & (NC - 1));
  const bool valid = e < A.n_elem;
  const int32_t id = valid ? __ldg(A.conn + e * NC + c) : 0;
  const int lev = valid ? A.level[e] : 0;
  const float inv_h = pow2i(lev, 0.0f);
  const float nb = float(-0.5 * (1.0 - kG));
  float sh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[k] = ((c >> k) & 1) ? inv_h : -inv_h;
  const float G2 = pow2i(2 * lev + 2, 0.0f);
  const float tau0 = fmaf(K.cid * G2, G2, K.tau_t);
  float un[3], vn[3], hn[2];
  load_record(A, id, valid, un, hn, vn);
  float cv[2], gc[2][3], gp[3], v[3], hq[2], tau, R[2], P[2][3];
  lane_state<float, D>(un, vn, hn, nb, sh, K.kappa, tau0, G2, cv, gc, gp, v, hq, tau, R, P);
  if (!valid) return;
  const int64_t L = A.n_elem * NC;
  const float zc0 = cv[0] - tau * R[0], zc1 = -(cv[1] - tau * R[1]);
  if constexpr (NR == 4) {
    qp[t] = make_float4(v[0], v[1], v[2], gp[0]);
    qp[L + t] = make_float4(gp[1], gp[2], gc[0][0], gc[0][1]);
    qp[2 * L + t] = make_float4(gc[0][2], gc[1][0], gc[1][1], gc[1][2]);
    qp[3 * L + t] = make_float4(tau, zc0, zc1, __int_as_float(lev));
  } else {
    qp[t] = make_float4(gp[0], gp[1], gp[2], gc[0][0]);
    qp[L + t] = make_float4(gc[0][1], gc[0][2], gc[1][0], gc[1][1]);
    qp[2 * L + t] = make_float4(gc[1][2], zc0, zc1, __int_as_float(lev));
  }
}

// The J V kernel streams the stored state through shared memory: a persistent grid
// walks tiles of kLaneThreads lanes, and per tile one thread issues bulk copies (TMA,
// cp.async.bulk) of the four state rows and the tile's connectivity into a stage of
// shared memory, completing on the stage's mbarrier.  kStages tiles are in flight per
// block, so the state's HBM stream does not wait on the per-lane arithmetic and
// atomics of the tile before.  Two stages with five blocks per SM measured fastest: three
// (four blocks per SM) and four (three) were 6% and 16% slower per launch.
constexpr int kStages = 2;
constexpr size_t jv_stage_bytes(int S, int NR) {
  return (size_t)S * ((size_t)NR * kLaneThreads * 16 + kLaneThreads * 4 + 8);
}
// try_wait polls before a wait on a stage gives up (about a second by default; a launch
// argument), and the longer limit of the drain that follows a give-up: the block waits
// for the copies it issued before it exits
constexpr int kWaitPolls = 1 << 22;
constexpr int kDrainPolls = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase of the given parity to complete; false when it did not
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int polls = kWaitPolls) {
  const uint32_t a = smem_u32(bar);
  for (int i = 0; i < polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <int D, int NS, int NR>
__global__ void __launch_bounds__(kLaneThreads, 5) k_jv_from_state(ElemArgs<float> A, LaneParams<float> K,
                                                                 const float4* __restrict__ qp, int* err,
                                                                 int polls) {
  constexpr int NC = 1 << D;
  extern __shared__ __align__(128) uint8_t jv_smem[];
  // NS stages of {NR state rows, connectivity} and NS mbarriers (jv_stage_bytes(NS, NR))
  auto sq = reinterpret_cast<float4(*)[NR][kLaneThreads]>(jv_smem);
  auto sconn = reinterpret_cast<int32_t(*)[kLaneThreads]>(jv_smem + NS * NR * kLaneThreads * sizeof(float4));
  uint64_t* bar = reinterpret_cast<uint64_t*>(jv_smem + NS * (NR * kLaneThreads * sizeof(float4) + kLaneThreads * 4));
  const int tid = threadIdx.x;
  const int64_t L = A.n_elem * NC;
  const int64_t n_tiles = (L + kLaneThreads - 1) / kLaneThreads;
  const int64_t G = gridDim.x;
  // thread 0: copy tile `tl` into stage `st` (sizes are multiples of 16 bytes: L and the
  // tile start are multiples of 2^d lanes, 4 B of connectivity per lane)
  auto issue = [&](int64_t tl, int st) {
    const int64_t t0 = tl * kLaneThreads;
    const uint32_t n = (uint32_t)(L - t0 < kLaneThreads ? L - t0 : kLaneThreads);
    mbar_expect_tx(&bar[st], (uint32_t)NR * 16u * n + 4u * n);
#pragma unroll
    for (int j = 0; j < NR; ++j) bulk_g2s(&sq[st][j][0], qp + j * L + t0, 16u * n, &bar[st]);
    bulk_g2s(&sconn[st][0], A.conn + t0, 4u * n, &bar[st]);
  };
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < NS; ++st) mbar_init(&bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t pending = 0;  // thread 0: stages with a copy in flight
  if (tid == 0) {
#pragma unroll
    for (int st = 0; st < NS; ++st)
      if (blockIdx.x + st * G < n_tiles) {
        issue(blockIdx.x + st * G, st);
        pending |= 1u << st;
      }
  }

  const float nb = float(-0.5 * (1.0 - kG));
  const float kappa = K.kappa, e2 = K.e2;
  for (int k = 0;; ++k) {
    const int64_t tl = blockIdx.x + (int64_t)k * G;
    if (tl >= n_tiles) break;
    const int st = k % NS;
    const uint32_t parity = (uint32_t)(k / NS) & 1u;
    const bool ok = mbar_wait(&bar[st], parity, polls);
    if (__syncthreads_or(!ok)) {
      // a copy did not complete: flag it, let the copies still in flight land, return
      if (tid == 0) {
        atomicOr(err, 1);
        for (int j = 0; j < NS; ++j) {
          const int kk = k + ((j - st + NS) % NS);
          if (pending >> j & 1u) mbar_wait(&bar[j], (uint32_t)(kk / NS) & 1u, kDrainPolls);
        }
      }
      return;
    }
    const int64_t t = tl * kLaneThreads + tid;
    const bool valid = t < L;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0, q3 = q0;
    int32_t id = 0;
    if (valid) {
      q0 = sq[st][0][tid];
      q1 = sq[st][1][tid];
      q2 = sq[st][2][tid];
      if constexpr (NR == 4) q3 = sq[st][NR - 1][tid];
      id = sconn[st][tid];
    }
    __syncthreads();  // stage st is read: refill it with the tile NS ahead
    if (tid == 0) {
      pending &= ~(1u << st);
      if (tl + NS * G < n_tiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(tl + NS * G, st);
        pending |= 1u << st;
      }
    }

    const int c = (int)(t & (NC - 1));
    float v[3], gp[3], gc[2][3], tau, zc_tR[2];
    int lev;
    if constexpr (NR == 4) {
      lev = __float_as_int(q3.w);  // 0 for lanes past the end
      v[0] = q0.x; v[1] = q0.y; v[2] = q0.z;
      gp[0] = q0.w; gp[1] = q1.x; gp[2] = q1.y;
      gc[0][0] = q1.z; gc[0][1] = q1.w; gc[0][2] = q2.x;
      gc[1][0] = q2.y; gc[1][1] = q2.z; gc[1][2] = q2.w;
      tau = q3.x;
      zc_tR[0] = q3.y; zc_tR[1] = q3.z;
    } else {
      lev = __float_as_int(q2.w);
      v[0] = v[1] = v[2] = 0.0f;
      gp[0] = q0.x; gp[1] = q0.y; gp[2] = q0.z;
      gc[0][0] = q0.w; gc[0][1] = q1.x; gc[0][2] = q1.y;
      gc[1][0] = q1.z; gc[1][1] = q1.w; gc[1][2] = q2.x;
      zc_tR[0] = q2.y; zc_tR[1] = q2.z;
      const float G2 = pow2i(2 * lev + 2, 0.0f);
      tau = rsqrtf(fmaf(K.cid * G2, G2, K.tau_t));
    }
    const float inv_h = pow2i(lev, 0.0f);
    const float w = pow2i(-D * (lev + 1), 0.0f);
    float sh[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) sh[kk] = ((c >> kk) & 1) ? inv_h : -inv_h;
    float dn[3];
    if (A.V4) load_dir4(A, id, valid, dn);
    else load_node<float, 3>(A, id, valid, A.V, 3, dn);
    float dcv[2], dgc[2][3], dgp[3], dR[2], S[3], Phi[3][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) interp_vg<float, D>(dn[s], nb, sh, dcv[s], dgc[s]);
    interp_g<float, D>(dn[2], nb, sh, dgp);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float z = s == 0 ? 1.0f : -1.0f;
      float P[3], vg = 0.0f, pg = 0.0f, gcd = 0.0f;
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        P[kk] = v[kk] - z * gp[kk];
        vg = fmaf(v[kk], dgc[s][kk], vg);
        pg = fmaf(P[kk], dgc[s][kk], pg);
        gcd = fmaf(gc[s][kk], dgp[kk], gcd);
      }
      dR[s] = fmaf(kappa, dcv[s], pg - z * gcd);
      S[s] = fmaf(kappa, dcv[s], vg);
      const float tdR = tau * dR[s];
      const float zdc = z * dcv[s];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk)
        Phi[s][kk] = fmaf(tdR, P[kk], fmaf(zc_tR[s], dgp[kk], fmaf(zdc, gp[kk], dgc[s][kk])));
    }
    S[2] = fmaf(tau, dR[0] - dR[1], dcv[1] - dcv[0]);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) Phi[2][kk] = e2 * dgp[kk];
    float r[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) r[f] = w * test_t<float, D>(S[f], Phi[f], nb, sh);
    if (!valid) continue;
    if (A.out4) {
      scatter4(A, id, r);
      continue;
    }
    if (id >= 0) {
#pragma unroll
      for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)id + f, r[f]);
    } else {
      const int32_t hh = -id - 1;
      const int np = A.hang_np[hh];
      const float wgt = np == 2 ? 0.5f : 0.25f;
      for (int p = 0; p < np; ++p) {
        const int32_t pid = A.hang_par[4 * hh + p];
#pragma unroll
        for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)pid + f, wgt * r[f]);
      }
    }
  }
}


// ---- block diagonal of the Jacobian (block-Jacobi preconditioner) ----------------
// D_n = sum over elements, Gauss points and local pairs (i, j) whose constraint targets
// both reach node n of t_i(n) t_j(n) B_ij, B_ij the 3x3 block (test N_i, trial N_j) of
// the linearised element operator and t the constraint weight (1 for a regular node, 1/2
// or 1/4 for a hanging node's parents).  Regular corners only pair with themselves; the
// pairs i != j arise only through hanging corners.  Lane c of an element group holds
// Gauss point c.  A block has seven nonzero entries, stored in this order:
// (+,+) (+,phi) (-,-) (-,phi) (phi,+) (phi,-) (phi,phi).
constexpr int kBlk = 7;
__device__ __forceinline__ int blk_slot(int k) {  // position in the row-major 3x3 block
  return k == 0 ? 0 : k == 1 ? 2 : k == 2 ? 4 : k == 3 ? 5 : k == 4 ? 6 : k == 5 ? 7 : 8;
}

// the seven entries of B_ij at this Gauss point (without the quadrature weight):
// derivatives of the species rows S_s, Phi_s and the Poisson row with respect to the
// trial field N_j, tested with N_i (Def. 3 linearised, as in the J V)
template <typename T>
__device__ __forceinline__ void pair_block(T Ni, const T (&dNi)[3], T Nj, const T (&dNj)[3], T kappa, T e2, T tau,
                                           const T (&cv)[2], const T (&gc)[2][3], const T (&gp)[3], const T (&v)[3],
                                           const T (&R)[2], const T (&P)[2][3], T (&B)[kBlk]) {
  T gij = T(0), gip = T(0), vgj = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gij = fma(dNi[k], dNj[k], gij);
    gip = fma(dNi[k], gp[k], gip);
    vgj = fma(v[k], dNj[k], vgj);
  }
  T pp = T(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T z = s == 0 ? T(1) : T(-1);
    T pgj = T(0), giP = T(0), gcj = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      pgj = fma(P[s][k], dNj[k], pgj);
      giP = fma(dNi[k], P[s][k], giP);
      gcj = fma(gc[s][k], dNj[k], gcj);
    }
    const T dRdc = fma(kappa, Nj, pgj);  // d R_s / d c_s
    const T dRdp = -z * gcj;             // d R_s / d phi
    B[2 * s] = Ni * fma(kappa, Nj, vgj) + gij + z * Nj * gip + tau * dRdc * giP;
    B[2 * s + 1] = z * cv[s] * gij + tau * dRdp * giP - tau * R[s] * z * gij;
    B[4 + s] = z * Ni * (tau * dRdc - Nj);
    pp = fma(z * tau, dRdp, pp);
  }
  B[6] = fma(e2, gij, Ni * pp);
}

// constraint targets of a corner: itself, or a hanging node's parents with their weights
template <typename T>
__device__ __forceinline__ int corner_targets(const int32_t* __restrict__ hpar, const uint8_t* __restrict__ hnp,
                                              int32_t id, int32_t (&tg)[4], T& wt) {
  if (id >= 0) {
    tg[0] = id;
    tg[1] = tg[2] = tg[3] = -1;
    wt = T(1);
    return 1;
  }
  const int32_t h = -id - 1;
  const int np = hnp[h];
#pragma unroll
  for (int p = 0; p < 4; ++p) tg[p] = p < np ? hpar[4 * h + p] : -1;
  wt = np == 2 ? T(0.5) : T(0.25);
  return np;
}

template <typename T, int D>
__global__ void __launch_bounds__(256) k_block_diag_lanes(ElemArgs<T> A, LaneParams<T> K, T* __restrict__ Dout) {
  constexpr int NC = 1 << D;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~int64_t(31)) / NC >= A.n_elem) return;
  const int64_t e = t / NC;
  const int c = (int)(t & (NC - 1));
  const int lane = threadIdx.x & 31, gb = lane & ~(NC - 1);
  const bool valid = e < A.n_elem;
  const int32_t id = valid ? __ldg(A.conn + e * NC + c) : 0;
  const int lev = valid ? A.level[e] : 0;
  const T inv_h = pow2i(lev, T(0));
  const T w = pow2i(-D * (lev + 1), T(0));
  const T nb = T(-0.5 * (1.0 - kG));
  T sh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[k] = ((c >> k) & 1) ? inv_h : -inv_h;
  const T G2 = pow2i(2 * lev + 2, T(0));
  const T tau0 = fma(K.cid * G2, G2, K.tau_t);
  T un[3], vn[3], hn[2];
  bool have = false;
  if constexpr (sizeof(T) == 4) {
    if (A.rec) {
      load_record(A, id, valid, un, hn, vn);
      have = true;
    }
  }
  if (!have) {
    load_node<T, 3>(A, id, valid, A.U, 3, un);
    load_node<T, 3>(A, id, valid, A.adv, 3, vn);
    load_node<T, 2>(A, id, valid, A.hs, 2, hn);
  }
  T cv[2], gc[2][3], gp[3], v[3], hq[2], tau, R[2], P[2][3];
  lane_state<T, D>(un, vn, hn, nb, sh, K.kappa, tau0, G2, cv, gc, gp, v, hq, tau, R, P);

  // diagonal pairs: B_ii at this Gauss point for every corner i, then a reduce-scatter
  // over the group leaves lane c with sum_q B_cc
  T a[NC][kBlk];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    T Ni, dNi[3];
    shape_at<T, D>(i, c, inv_h, Ni, dNi);
    pair_block<T>(Ni, dNi, Ni, dNi, K.kappa, K.e2, tau, cv, gc, gp, v, R, P, a[i]);
  }
  T b[(NC + 1) / 2][kBlk];
  {
    const bool hi = c & 1;
#pragma unroll
    for (int m = 0; m < NC / 2; ++m)
#pragma unroll
      for (int x = 0; x < kBlk; ++x) {
        const T keep = hi ? a[2 * m + 1][x] : a[2 * m][x];
        const T send = hi ? a[2 * m][x] : a[2 * m + 1][x];
        b[m][x] = keep + flip(send, 0);
      }
  }
  T r[kBlk];
  if constexpr (D == 2) {
    const bool hi = (c >> 1) & 1;
#pragma unroll
    for (int x = 0; x < kBlk; ++x) {
      const T keep = hi ? b[1][x] : b[0][x];
      const T send = hi ? b[0][x] : b[1][x];
      r[x] = keep + flip(send, 1);
    }
  } else {
    T b2[2][kBlk];
    const bool hi1 = (c >> 1) & 1, hi2 = (c >> 2) & 1;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int x = 0; x < kBlk; ++x) {
        const T keep = hi1 ? b[2 * m + 1][x] : b[2 * m][x];
        const T send = hi1 ? b[2 * m][x] : b[2 * m + 1][x];
        b2[m][x] = keep + flip(send, 1);
      }
#pragma unroll
    for (int x = 0; x < kBlk; ++x) {
      const T keep = hi2 ? b2[1][x] : b2[0][x];
      const T send = hi2 ? b2[0][x] : b2[1][x];
      r[x] = keep + flip(send, 2);
    }
  }
  int32_t tg[4] = {-1, -1, -1, -1};
  T wt = T(0);
  const int nt = valid ? corner_targets<T>(A.hang_par, A.hang_np, id, tg, wt) : 0;
  for (int p = 0; p < nt; ++p) {
    const T ww = w * wt * wt;
#pragma unroll
    for (int x = 0; x < kBlk; ++x) atomicAdd(Dout + 9 * (int64_t)tg[p] + blk_slot(x), ww * r[x]);
  }

  // pairs i != j through hanging corners: lane gb + i owns the pair's scatter
  if (!__any_sync(kFull, valid && id < 0)) return;
#pragma unroll 1
  for (int i = 0; i < NC; ++i) {
#pragma unroll 1
    for (int j = 0; j < NC; ++j) {
      if (i == j) continue;
      const int32_t id_i = __shfl_sync(kFull, id, gb + i), id_j = __shfl_sync(kFull, id, gb + j);
      // targets of j at lane gb + i (the owner), compared with its own
      int32_t tj[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) tj[p] = __shfl_sync(kFull, tg[p], gb + j);
      const T wj = __shfl_sync(kFull, wt, gb + j);
      bool share = false;
      if (c == i && valid && (id_i < 0 || id_j < 0))
        for (int p = 0; p < nt; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) share |= tg[p] == tj[q];
      const bool need = __shfl_sync(kFull, share, gb + i);
      if (!__any_sync(kFull, need)) continue;
      T Ni, dNi[3], Nj, dNj[3], B[kBlk];
      shape_at<T, D>(i, c, inv_h, Ni, dNi);
      shape_at<T, D>(j, c, inv_h, Nj, dNj);
      pair_block<T>(Ni, dNi, Nj, dNj, K.kappa, K.e2, tau, cv, gc, gp, v, R, P, B);
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int x = 0; x < kBlk; ++x) B[x] += flip(B[x], k);
      if (c == i && share)
        for (int p = 0; p < nt; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (tg[p] == tj[q]) {
              const T ww = w * wt * wj;
#pragma unroll
              for (int x = 0; x < kBlk; ++x) atomicAdd(Dout + 9 * (int64_t)tg[p] + blk_slot(x), ww * B[x]);
            }
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
    if (jv) k_element_lanes<T, T, 2, true><<<blocks, t, 0, s>>>(A, K);
    else k_element_lanes<T, T, 2, false><<<blocks, t, 0, s>>>(A, K);
  } else {
    if (jv) k_element_lanes<T, T, 3, true><<<blocks, t, 0, s>>>(A, K);
    else k_element_lanes<T, T, 3, false><<<blocks, t, 0, s>>>(A, K);
  }
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_element_lanes<double>(int, bool, const ElemArgs<double>&, cudaStream_t);
template cudaError_t launch_element_lanes<float>(int, bool, const ElemArgs<float>&, cudaStream_t);

// FP64 residual with double-float arithmetic (FP32 pipe), FP64 data in and out
cudaError_t launch_residual_df(int dim, const ElemArgs<double>& A, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  const int t = 256;
  const unsigned blocks = (unsigned)(((A.n_elem << dim) + t - 1) / t);
  const LaneParams<df> K{df(A.P.kappa), df(A.P.tau_t), df(A.P.C_I * dim), df(A.P.eps2x2)};
  if (dim == 2) k_element_lanes<double, df, 2, false><<<blocks, t, 0, s>>>(A, K);
  else k_element_lanes<double, df, 3, false><<<blocks, t, 0, s>>>(A, K);
  note_launch();
  return cudaGetLastError();
}

// the stored linearisation of the FP32 J V (qp: 4 * 2^dim * n_elem float4; A.rec set)
cudaError_t launch_lane_state(int dim, const ElemArgs<float>& A, float4* qp, int rows, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  if (rows != 3 && rows != 4) return cudaErrorInvalidValue;
  const LaneParams<float> K{float(A.P.kappa), float(A.P.tau_t), float(A.P.C_I * dim), float(A.P.eps2x2)};
  const unsigned blocks = (unsigned)(((A.n_elem << dim) + kLaneThreads - 1) / kLaneThreads);
  if (dim == 2) {
    if (rows == 4) k_lane_state<2, 4><<<blocks, kLaneThreads, 0, s>>>(A, K, qp);
    else k_lane_state<2, 3><<<blocks, kLaneThreads, 0, s>>>(A, K, qp);
  } else {
    if (rows == 4) k_lane_state<3, 4><<<blocks, kLaneThreads, 0, s>>>(A, K, qp);
    else k_lane_state<3, 3><<<blocks, kLaneThreads, 0, s>>>(A, K, qp);
  }
  note_launch();
  return cudaGetLastError();
}

template <int S, int NR>
static cudaError_t launch_jv_stages(int dim, const ElemArgs<float>& A, const LaneParams<float>& K, const float4* qp,
                                    int* err, int polls, cudaStream_t s) {
  // persistent grid: the resident blocks of every SM, no more than there are tiles
  static int per_sm[2] = {0, 0}, n_sm = 0;
  const size_t smem = jv_stage_bytes(S, NR);
  if (n_sm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_jv_from_state<2, S, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_jv_from_state<3, S, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_jv_from_state<2, S, NR>, kLaneThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_jv_from_state<3, S, NR>, kLaneThreads, smem);
    if (e != cudaSuccess) {
      n_sm = 0;
      return e;
    }
  }
  const int64_t tiles = ((A.n_elem << dim) + kLaneThreads - 1) / kLaneThreads;
  const unsigned blocks = (unsigned)std::min<int64_t>(tiles, (int64_t)n_sm * std::max(1, per_sm[dim - 2]));
  if (dim == 2) k_jv_from_state<2, S, NR><<<blocks, kLaneThreads, smem, s>>>(A, K, qp, err, polls);
  else k_jv_from_state<3, S, NR><<<blocks, kLaneThreads, smem, s>>>(A, K, qp, err, polls);
  return cudaSuccess;
}

cudaError_t launch_jv_from_state(int dim, const ElemArgs<float>& A, const float4* qp, int rows, int* err,
                                 int polls, cudaStream_t s) {
  if (polls < 0) polls = kWaitPolls;
  if (A.n_elem == 0) return cudaSuccess;
  if (rows != 3 && rows != 4) return cudaErrorInvalidValue;
  const LaneParams<float> K{float(A.P.kappa), float(A.P.tau_t), float(A.P.C_I * dim), float(A.P.eps2x2)};
  const cudaError_t e = rows == 4 ? launch_jv_stages<kStages, 4>(dim, A, K, qp, err, polls, s)
                                  : launch_jv_stages<kStages, 3>(dim, A, K, qp, err, polls, s);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// per lane of the stored-linearisation J V: direction values and gradients, the J V
// physics (incl. P_s), three transposes; the state part is read, not computed
double jv_from_state_flops(int D) {
  const double tri = D * (D - 1) / 2.0;
  const double vg = 3 * tri + 4 * D, g = vg - 2, tt = 6 * D + 3 * tri + 1;
  return (double)(1 << D) * (2 * vg + g + 101 + 12 + 3 * tt);
}

template <typename T>
cudaError_t launch_block_diag_lanes(int dim, const ElemArgs<T>& A, T* Dout, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  const int t = 256;
  const unsigned blocks = (unsigned)(((A.n_elem << dim) + t - 1) / t);
  const LaneParams<T> K{T(A.P.kappa), T(A.P.tau_t), T(A.P.C_I * dim), T(A.P.eps2x2)};
  if (dim == 2) k_block_diag_lanes<T, 2><<<blocks, t, 0, s>>>(A, K, Dout);
  else k_block_diag_lanes<T, 3><<<blocks, t, 0, s>>>(A, K, Dout);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_block_diag_lanes<double>(int, const ElemArgs<double>&, double*, cudaStream_t);
template cudaError_t launch_block_diag_lanes<float>(int, const ElemArgs<float>&, float*, cudaStream_t);

// per element of the block-diagonal kernel, hanging pairs not counted: per lane the
// state at its Gauss point (as in the residual), per corner the shape function (8) and
// the seven block entries (114), the reduce-scatter (7 adds per stage and entry over
// 2^d - 1 entries in all) and the scaling
double block_diag_flops(int D) {
  const double NC = 1 << D;
  const double tri = D * (D - 1) / 2.0;
  const double vg = 3 * tri + 4 * D, g = vg - 2, v = 3 * D;
  const double state = 2 * vg + 2 * v + g + D * v + 2 * D + 3 + 30;
  return NC * (state + NC * (8 + 114) + 7 * (NC - 1) + 7);
}
