// jv_pair.cu -- FP32 Jacobian action of the VMS PNP residual on hexahedra with two lanes
// per element.
//
// Physics per Gauss point as in Def. 3 of arXiv 2301.05985 with the fine scales
// c^f = -tau_c R_c (Sec. 3.1), linearised (the same statement as element_lanes.cu):
//     dR_s   = kappa dc_s + P_s . grad dc_s - z_s grad c_s . grad dphi,   P_s = v - z_s grad phi
//     S_s    = kappa dc_s + v . grad dc_s
//     Phi_s  = grad dc_s + z_s dc_s grad phi + z_s (c_s - tau R_s) grad dphi + tau dR_s P_s
//     S_phi  = tau (dR_+ - dR_-) + dc_- - dc_+,     Phi_phi = 2 Lambda^2 grad dphi
// and the element vector r_c = (h/2)^3 sum_q [N_c(q) S_q + grad N_c(q) . Phi_q].
//
// Layout of the work: lane z (0 or 1) of an element's pair holds the four corners with
// z-bit z and the four Gauss points next to them.  The trilinear interpolation is a tensor
// product of 1D two-node operators; its z factor needs the partner's corner values (one
// shuffle per scalar and corner), its x and y factors run in registers.  The transposed
// test side accumulates, per corner column (x, y), the parts of the test functions that
// do not depend on z, and applies the z factor at the end, sending the partner its
// corners' share (one shuffle per field and corner).  Against one lane per corner this
// trades 24 of the 57 shuffles per corner for register arithmetic, and recomputes the
// state's Gauss-point quantities from the 32-byte FP32 node records instead of streaming
// a stored linearisation: the kernel reads 48 B per node and element corner from L2/HBM
// (record and padded direction) and adds one vector atomic per corner.
#include <cstdint>

#include "kernels.h"

namespace {

constexpr float kGf = 0.57735026918962576450914878050196f;  // 1/sqrt(3)
constexpr float kNear = 0.5f * (1.0f + kGf);                 // 1D shape value at the near Gauss point
constexpr float kFar = 0.5f * (1.0f - kGf);                  // ... at the far one
constexpr float kNb = -kFar;  // value at the near point: u_near + kNb (u_near - u_far)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kPairThreads = 256;

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ float partner(float x) { return __shfl_xor_sync(kFull, x, 1); }

// node records {c+, c-, phi, h+, h-, v0, v1, v2} and directions of a lane's four corners.
// The loads of all four corners are issued before any is used (a hanging corner first
// loads node 0 in its place), so twelve 16-byte loads are in flight per lane; corners that
// hang on coarser neighbours are then replaced by the mean of their parents.
template <bool PAD>
__device__ __forceinline__ float4 load_dir(const ElemArgs<float>& A, int64_t nid) {
  if constexpr (PAD) {
    return __ldg(A.V4 + nid);
  } else {
    return make_float4(__ldg(A.V + 3 * nid), __ldg(A.V + 3 * nid + 1), __ldg(A.V + 3 * nid + 2), 0.f);
  }
}
template <bool PAD>
__device__ __forceinline__ void load_corners(const ElemArgs<float>& A, const int32_t (&id)[4], bool valid,
                                             float4 (&r0)[4], float4 (&r1)[4], float4 (&dv)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t nid = (valid && id[j] >= 0) ? id[j] : 0;
    r0[j] = __ldg(A.rec + 2 * nid);
    r1[j] = __ldg(A.rec + 2 * nid + 1);
    dv[j] = load_dir<PAD>(A, nid);
  }
  if (!valid) {
#pragma unroll
    for (int j = 0; j < 4; ++j) r0[j] = r1[j] = dv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (id[j] >= 0) continue;
    const int32_t h = -id[j] - 1;
    const int np = A.hang_np[h];
    const float wgt = np == 2 ? 0.5f : 0.25f;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, ad = a0;
    for (int p = 0; p < np; ++p) {
      const int64_t pid = A.hang_par[4 * h + p];
      const float4 x = __ldg(A.rec + 2 * pid), y = __ldg(A.rec + 2 * pid + 1), d = load_dir<PAD>(A, pid);
      a0.x += wgt * x.x; a0.y += wgt * x.y; a0.z += wgt * x.z; a0.w += wgt * x.w;
      a1.x += wgt * y.x; a1.y += wgt * y.y; a1.z += wgt * y.z; a1.w += wgt * y.w;
      ad.x += wgt * d.x; ad.y += wgt * d.y; ad.z += wgt * d.z;
    }
    r0[j] = a0;
    r1[j] = a1;
    dv[j] = ad;
  }
}

// z factor of a field with gradient: value at this lane's Gauss-point level and z-derivative
__device__ __forceinline__ void zstage_vg(float u, float szh, float& v, float& dz) {
  const float diff = u - partner(u);
  v = fmaf(kNb, diff, u);
  dz = szh * diff;
}
__device__ __forceinline__ float zstage_v(float u) { return fmaf(kNb, u - partner(u), u); }

// y factor at row qy of a 2x2 (x, y) array: value and y-derivative per x
struct YCol {
  float v[2], dy[2], dz[2];
};
__device__ __forceinline__ void ystage(const float (&u)[4], const float (&dz)[4], int qy, float inv_h, YCol& o) {
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const float un = u[x + 2 * qy], uf = u[x + 2 * (1 - qy)];
    o.v[x] = fmaf(kNb, un - uf, un);
    o.dy[x] = (u[x + 2] - u[x]) * inv_h;
    const float zn = dz[x + 2 * qy], zf = dz[x + 2 * (1 - qy)];
    o.dz[x] = fmaf(kNb, zn - zf, zn);
  }
}
// x factor at column qx: value and gradient at the Gauss point
__device__ __forceinline__ void xstage(const YCol& c, int qx, float inv_h, float& val, float (&g)[3]) {
  const float vn = c.v[qx], vf = c.v[1 - qx];
  val = fmaf(kNb, vn - vf, vn);
  g[0] = (c.v[1] - c.v[0]) * inv_h;
  g[1] = fmaf(kNb, c.dy[qx] - c.dy[1 - qx], c.dy[qx]);
  g[2] = fmaf(kNb, c.dz[qx] - c.dz[1 - qx], c.dz[qx]);
}
__device__ __forceinline__ float xy_value(const float (&u)[4], int qx, int qy) {
  float a[2];
#pragma unroll
  for (int x = 0; x < 2; ++x) a[x] = fmaf(kNb, u[x + 2 * qy] - u[x + 2 * (1 - qy)], u[x + 2 * qy]);
  return fmaf(kNb, a[qx] - a[1 - qx], a[qx]);
}

// the (x, y) part of the test functions of the four corner columns at Gauss point (qx, qy):
// A[x + 2y] += Nx Ny S + dNx Ny Phi_x + Nx dNy Phi_y,  B[x + 2y] += Nx Ny Phi_z
__device__ __forceinline__ void test_acc(float S, const float (&Phi)[3], int qx, int qy, float inv_h, float (&A)[4],
                                         float (&B)[4]) {
  float tx[2], ty[2], tz[2];
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const float nx = x == qx ? kNear : kFar;
    const float dx = x ? inv_h : -inv_h;
    tx[x] = fmaf(nx, S, dx * Phi[0]);
    ty[x] = nx * Phi[1];
    tz[x] = nx * Phi[2];
  }
#pragma unroll
  for (int y = 0; y < 2; ++y) {
    const float ny = y == qy ? kNear : kFar;
    const float dy = y ? inv_h : -inv_h;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      A[x + 2 * y] = fmaf(ny, tx[x], fmaf(dy, ty[x], A[x + 2 * y]));
      B[x + 2 * y] = fmaf(ny, tz[x], B[x + 2 * y]);
    }
  }
}

#ifndef PNP_JV_PAIR_MINB
#define PNP_JV_PAIR_MINB 2  // blocks per SM the register cap is set for
#endif

template <bool ADV, bool PAD>
__global__ void __launch_bounds__(kPairThreads, PNP_JV_PAIR_MINB) k_jv_pair(ElemArgs<float> A, float kappa,
                                                                          float tau_t, float cid, float e2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // warps whose first element is past the end leave together (shuffles need the warp)
  if ((t & ~int64_t(31)) / 2 >= A.n_elem) return;
  const int64_t e = t >> 1;
  const int zb = (int)(t & 1);
  const bool valid = e < A.n_elem;
  int4 ids = make_int4(0, 0, 0, 0);
  int lev = 0;
  if (valid) {
    ids = __ldg(reinterpret_cast<const int4*>(A.conn + 8 * e + 4 * zb));
    lev = A.level[e];
  }
  const int32_t id[4] = {ids.x, ids.y, ids.z, ids.w};
  const float inv_h = pow2f(lev);
  const float szh = zb ? inv_h : -inv_h;
  const float G2 = pow2f(2 * lev + 2);          // (2/h)^2
  const float tau0 = fmaf(cid * G2, G2, tau_t);  // 4/dt^2 + C_I d (2/h)^4

  // z factor of every field at the four corner columns of this lane's Gauss-point level
  float cz[2][4], czd[2][4], pz[4], pzd[4], hz[2][4], vz[3][4], dcz[2][4], dczd[2][4], dpz[4], dpzd[4];
  float4 r0[4], r1[4], dv[4];
  load_corners<PAD>(A, id, valid, r0, r1, dv);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float u[3] = {r0[j].x, r0[j].y, r0[j].z}, hq[2] = {r0[j].w, r1[j].x};
    const float vq[3] = {r1[j].y, r1[j].z, r1[j].w}, d[3] = {dv[j].x, dv[j].y, dv[j].z};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      zstage_vg(u[s], szh, cz[s][j], czd[s][j]);
      hz[s][j] = zstage_v(hq[s]);
      zstage_vg(d[s], szh, dcz[s][j], dczd[s][j]);
    }
    zstage_vg(u[2], szh, pz[j], pzd[j]);
    zstage_vg(d[2], szh, dpz[j], dpzd[j]);
    if constexpr (ADV) {
#pragma unroll
      for (int k = 0; k < 3; ++k) vz[k][j] = zstage_v(vq[k]);
    }
  }

  float Aacc[3][4], Bacc[3][4];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int j = 0; j < 4; ++j) Aacc[f][j] = Bacc[f][j] = 0.0f;

  const float tau_c = rsqrtf(tau0);  // no advection: tau_c depends on the level only
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    YCol yc[2], yp, ydc[2], ydp;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      ystage(cz[s], czd[s], qy, inv_h, yc[s]);
      ystage(dcz[s], dczd[s], qy, inv_h, ydc[s]);
    }
    ystage(pz, pzd, qy, inv_h, yp);
    ystage(dpz, dpzd, qy, inv_h, ydp);
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      float cv[2], gc[2][3], gp[3], dcv[2], dgc[2][3], dgp[3], pv, dpv;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        xstage(yc[s], qx, inv_h, cv[s], gc[s]);
        xstage(ydc[s], qx, inv_h, dcv[s], dgc[s]);
      }
      xstage(yp, qx, inv_h, pv, gp);
      xstage(ydp, qx, inv_h, dpv, dgp);
      float v[3] = {0.0f, 0.0f, 0.0f};
      float tau = tau_c;
      if constexpr (ADV) {
        float vv = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          v[k] = xy_value(vz[k], qx, qy);
          vv = fmaf(v[k], v[k], vv);
        }
        tau = rsqrtf(fmaf(G2, vv, tau0));
      }
      float S[3], Phi[3][3], dR[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float z = s == 0 ? 1.0f : -1.0f;
        const float hqv = xy_value(hz[s], qx, qy);
        float P[3], pg = 0.0f, pdg = 0.0f, gcd = 0.0f, vg = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          P[k] = v[k] - z * gp[k];
          pg = fmaf(P[k], gc[s][k], pg);
          pdg = fmaf(P[k], dgc[s][k], pdg);
          gcd = fmaf(gc[s][k], dgp[k], gcd);
          if constexpr (ADV) vg = fmaf(v[k], dgc[s][k], vg);
        }
        const float R = fmaf(kappa, cv[s], hqv + pg);
        dR[s] = fmaf(kappa, dcv[s], pdg - z * gcd);
        S[s] = fmaf(kappa, dcv[s], vg);
        const float tdR = tau * dR[s];
        const float zdc = z * dcv[s];
        const float zc_tR = z * (cv[s] - tau * R);
#pragma unroll
        for (int k = 0; k < 3; ++k) Phi[s][k] = fmaf(tdR, P[k], fmaf(zc_tR, dgp[k], fmaf(zdc, gp[k], dgc[s][k])));
      }
      S[2] = fmaf(tau, dR[0] - dR[1], dcv[1] - dcv[0]);
#pragma unroll
      for (int k = 0; k < 3; ++k) Phi[2][k] = e2 * dgp[k];
#pragma unroll
      for (int f = 0; f < 3; ++f) test_acc(S[f], Phi[f], qx, qy, inv_h, Aacc[f], Bacc[f]);
      (void)pv;
      (void)dpv;
    }
  }

  // z factor of the test side: this lane's corners take near A + dN B, the partner's
  // corners far A - dN B (sent across the pair)
  const float w = pow2f(-3 * (lev + 1));  // (h/2)^3
  float r[3][4];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float zB = szh * Bacc[f][j];
      const float mine = fmaf(kNear, Aacc[f][j], zB);
      const float send = fmaf(kFar, Aacc[f][j], -zB);
      r[f][j] = w * (mine + partner(send));
    }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t nid = id[j];
    if (nid >= 0) {
      if constexpr (PAD) {
        atomicAdd(A.out4 + nid, make_float4(r[0][j], r[1][j], r[2][j], 0.f));
      } else {
#pragma unroll
        for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)nid + f, r[f][j]);
      }
    } else {
      const int32_t h = -nid - 1;
      const int np = A.hang_np[h];
      const float wgt = np == 2 ? 0.5f : 0.25f;
      for (int p = 0; p < np; ++p) {
        const int32_t pid = A.hang_par[4 * h + p];
        if constexpr (PAD) {
          atomicAdd(A.out4 + pid, make_float4(wgt * r[0][j], wgt * r[1][j], wgt * r[2][j], 0.f));
        } else {
#pragma unroll
          for (int f = 0; f < 3; ++f) atomicAdd(A.out + 3 * (int64_t)pid + f, wgt * r[f][j]);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_jv_pair(const ElemArgs<float>& A, bool advection, cudaStream_t s) {
  if (A.n_elem == 0) return cudaSuccess;
  if (!A.rec || !A.conn) return cudaErrorInvalidValue;
  const bool pad = A.V4 && A.out4;
  if (!pad && (!A.V || !A.out)) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((2 * A.n_elem + kPairThreads - 1) / kPairThreads);
  const float kappa = (float)A.P.kappa, tau_t = (float)A.P.tau_t, cid = (float)(A.P.C_I * 3), e2 = (float)A.P.eps2x2;
  if (advection) {
    if (pad) k_jv_pair<true, true><<<blocks, kPairThreads, 0, s>>>(A, kappa, tau_t, cid, e2);
    else k_jv_pair<true, false><<<blocks, kPairThreads, 0, s>>>(A, kappa, tau_t, cid, e2);
  } else {
    if (pad) k_jv_pair<false, true><<<blocks, kPairThreads, 0, s>>>(A, kappa, tau_t, cid, e2);
    else k_jv_pair<false, false><<<blocks, kPairThreads, 0, s>>>(A, kappa, tau_t, cid, e2);
  }
  note_launch();
  return cudaGetLastError();
}

// floating-point operations per element of k_jv_pair (an FMA counts 2), from the
// formulation it evaluates; per lane: the z factors (value: 3, value and derivative: 4
// per corner), per Gauss-point row qy the y factors (9 per field with gradient), per
// Gauss point the x factors (9 per field with gradient, 6 per plain value), the physics,
// the (x, y) test parts of three fields (26 each), and the z factor of the test side
double jv_pair_flops(bool advection) {
  const double zst = 4.0 * (6 * 4 + (2 + (advection ? 3 : 0)) * 3);
  const double yst = 2.0 * 6 * 9;
  const double xst = 4.0 * (6 * 9 + (2 + (advection ? 3 : 0)) * 6);
  const double tau = advection ? 4.0 * 8 : 0.0;
  const double phys = 4.0 * (2 * (3 * 8 + 6 + 2 + (advection ? 6 : 0) + 3 + 3 * 6) + 5 + 3);
  const double test = 4.0 * 3 * 26;
  const double ztest = 3.0 * 4 * 7;
  return 2.0 * (zst + yst + xst + tau + phys + test + ztest);
}
