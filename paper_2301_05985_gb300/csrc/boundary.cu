// boundary.cu -- species fluxes through a boundary face: the terms of the boundary
// current of Sec. 5.2 (the net species flux through the top boundary of the
// electroconvection cell), out[s] = int_face n . (grad c_s + z_s c_s grad phi) dS with n
// the outward unit normal, z_+ = 1, z_- = -1.
//
// One thread per element (grid-stride over a fixed grid): an element contributes when
// all corners of its side on the face carry the face's boundary bit; the side integral
// uses the tensor Gauss rule with 2^(d-1) points, the Q1 fields gathered through the
// hanging constraints.  Per-block partials are summed in a fixed order.
#include <cstdint>

#include "kernels.h"

namespace {

constexpr double kGs = 0.57735026918962576450914878050196;  // 1/sqrt(3)
constexpr int kFluxThreads = 128;

template <int D>
__global__ void __launch_bounds__(kFluxThreads) k_boundary_flux(int64_t E, const int32_t* __restrict__ conn,
                                                                const uint8_t* __restrict__ level,
                                                                const uint8_t* __restrict__ faces,
                                                                const int32_t* __restrict__ hnode,
                                                                const int32_t* __restrict__ hpar,
                                                                const uint8_t* __restrict__ hnp,
                                                                const double* __restrict__ U, int face,
                                                                double* __restrict__ part) {
  constexpr int NC = 1 << D;
  const int ax = face / 2, high = face & 1;
  const uint8_t fbit = (uint8_t)(1u << face);
  double acc[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t id[NC];
    bool on = true;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      id[c] = conn[e * NC + c];
      if (((c >> ax) & 1) == high) {
        const int32_t node = id[c] >= 0 ? id[c] : hnode[-id[c] - 1];
        on = on && (faces[node] & fbit);
      }
    }
    if (!on) continue;
    // nodal values through the constraints
    double u[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      for (int f = 0; f < 3; ++f) u[c][f] = 0.0;
      if (id[c] >= 0) {
        for (int f = 0; f < 3; ++f) u[c][f] = U[3 * (int64_t)id[c] + f];
      } else {
        const int32_t h = -id[c] - 1;
        const int np = hnp[h];
        const double w = np == 2 ? 0.5 : 0.25;
        for (int p = 0; p < np; ++p)
          for (int f = 0; f < 3; ++f) u[c][f] += w * U[3 * (int64_t)hpar[4 * h + p] + f];
      }
    }
    const int lev = level[e];
    const double h = ldexp(1.0, -lev);
    const double wq = ldexp(1.0, -(D - 1) * (lev + 1));  // (h/2)^(D-1)
    const double nrm = high ? 1.0 : -1.0;
#pragma unroll
    for (int q = 0; q < (1 << (D - 1)); ++q) {
      double xi[3] = {0.0, 0.0, 0.0};
      int bit = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k == ax) {
          xi[k] = high ? 1.0 : -1.0;
        } else {
          xi[k] = ((q >> bit) & 1) ? kGs : -kGs;
          ++bit;
        }
      }
      double val[2] = {0.0, 0.0}, dn[3] = {0.0, 0.0, 0.0};  // c+-, and d/dx_ax of c+, c-, phi
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double N = 1.0, dN = ((c >> ax) & 1) ? 1.0 / h : -1.0 / h;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double f1 = 0.5 * (1.0 + (((c >> k) & 1) ? xi[k] : -xi[k]));
          N *= f1;
          if (k != ax) dN *= f1;
        }
        val[0] += N * u[c][0];
        val[1] += N * u[c][1];
        for (int f = 0; f < 3; ++f) dn[f] += dN * u[c][f];
      }
      acc[0] += wq * nrm * (dn[0] + val[0] * dn[2]);
      acc[1] += wq * nrm * (dn[1] - val[1] * dn[2]);
    }
  }
  __shared__ double sh[2][kFluxThreads];
  sh[0][threadIdx.x] = acc[0];
  sh[1][threadIdx.x] = acc[1];
  __syncthreads();
  for (int o = kFluxThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh[0][0];
    part[2 * blockIdx.x + 1] = sh[1][0];
  }
}

}  // namespace

cudaError_t launch_boundary_flux(int dim, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                 const uint8_t* faces, const int32_t* hnode, const int32_t* hpar, const uint8_t* hnp,
                                 const double* U, int face, double* part, double* out, cudaStream_t s) {
  if (n_elem == 0) return cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
  if (dim == 2)
    k_boundary_flux<2><<<kRedBlocks, kFluxThreads, 0, s>>>(n_elem, conn, level, faces, hnode, hpar, hnp, U, face,
                                                             part);
  else
    k_boundary_flux<3><<<kRedBlocks, kFluxThreads, 0, s>>>(n_elem, conn, level, faces, hnode, hpar, hnp, U, face,
                                                             part);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_parts(kRedBlocks, 2, part, out, s);
}
