// boundary.cu -- the electroconvection diagnostics of Sec. 5.2: the species fluxes through
// a boundary face (the terms of the boundary current, the net species flux through the
// top boundary), out[s] = int_face n . (grad c_s + z_s c_s grad phi) dS with n the
// outward unit normal, z_+ = 1, z_- = -1; and plane integrals of the fields (the
// x-averaged profiles).
//
// Fluxes: one thread per element (grid-stride over a fixed grid): an element contributes when
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

// integral over the plane x_ax = coord (integer units) of the three fields: each point of
// the plane belongs to the one element whose half-open range [a, a + s) along ax holds it
// (the top face, coord = size, to the elements ending there); the element's cross-section
// at xi_ax = 2 (coord - a) / s - 1 is integrated with the 2^(d-1)-point Gauss rule
template <int D>
__global__ void __launch_bounds__(kFluxThreads) k_plane_integral(int64_t E, int L, const int32_t* __restrict__ conn,
                                                                 const uint8_t* __restrict__ level,
                                                                 const int32_t* __restrict__ anchor,
                                                                 const int32_t* __restrict__ hnode,
                                                                 const int32_t* __restrict__ hpar,
                                                                 const uint8_t* __restrict__ hnp,
                                                                 const double* __restrict__ U, int ax, int64_t coord,
                                                                 double* __restrict__ part) {
  constexpr int NC = 1 << D;
  const int64_t size = int64_t(1) << L;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int lev = level[e];
    const int64_t s = int64_t(1) << (L - lev);
    const int64_t a = anchor[e * D + ax];
    const bool inside = (a <= coord && coord < a + s) || (coord == size && a + s == size);
    if (!inside) continue;
    const double xa = 2.0 * (double)(coord - a) / (double)s - 1.0;
    double u[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int32_t id = conn[e * NC + c];
      for (int f = 0; f < 3; ++f) u[c][f] = 0.0;
      if (id >= 0) {
        for (int f = 0; f < 3; ++f) u[c][f] = U[3 * (int64_t)id + f];
      } else {
        const int32_t h = -id - 1;
        const int np = hnp[h];
        const double w = np == 2 ? 0.5 : 0.25;
        for (int p = 0; p < np; ++p)
          for (int f = 0; f < 3; ++f) u[c][f] += w * U[3 * (int64_t)hpar[4 * h + p] + f];
      }
    }
    const double wq = ldexp(1.0, -(D - 1) * (lev + 1));  // (h/2)^(D-1)
#pragma unroll
    for (int q = 0; q < (1 << (D - 1)); ++q) {
      double xi[3] = {0.0, 0.0, 0.0};
      int bit = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k == ax) {
          xi[k] = xa;
        } else {
          xi[k] = ((q >> bit) & 1) ? kGs : -kGs;
          ++bit;
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double N = 1.0;
#pragma unroll
        for (int k = 0; k < D; ++k) N *= 0.5 * (1.0 + (((c >> k) & 1) ? xi[k] : -xi[k]));
        for (int f = 0; f < 3; ++f) acc[f] += wq * N * u[c][f];
      }
    }
  }
  __shared__ double sh[3][kFluxThreads];
  for (int f = 0; f < 3; ++f) sh[f][threadIdx.x] = acc[f];
  __syncthreads();
  for (int o = kFluxThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int f = 0; f < 3; ++f) sh[f][threadIdx.x] += sh[f][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int f = 0; f < 3; ++f) part[3 * blockIdx.x + f] = sh[f][0];
}

// |grad u| of each field at the element centre (the refinement indicator of the octree
// construction): for Q1, du/dx_k there is the mean over the element's 2^(d-1) edges along
// axis k of (u_high - u_low) / h.  One thread per element; out [E][3].
template <int D>
__global__ void k_element_gradient(int64_t E, const int32_t* __restrict__ conn, const uint8_t* __restrict__ level,
                                   const int32_t* __restrict__ hpar, const uint8_t* __restrict__ hnp,
                                   const double* __restrict__ U, double* __restrict__ out) {
  constexpr int NC = 1 << D;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double u[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int32_t id = conn[e * NC + c];
    for (int f = 0; f < 3; ++f) u[c][f] = 0.0;
    if (id >= 0) {
      for (int f = 0; f < 3; ++f) u[c][f] = U[3 * (int64_t)id + f];
    } else {
      const int32_t h = -id - 1;
      const int np = hnp[h];
      const double w = np == 2 ? 0.5 : 0.25;
      for (int p = 0; p < np; ++p)
        for (int f = 0; f < 3; ++f) u[c][f] += w * U[3 * (int64_t)hpar[4 * h + p] + f];
    }
  }
  const double inv = ldexp(1.0, level[e]) / (double)(NC / 2);  // 1 / (h * edges per axis)
  for (int f = 0; f < 3; ++f) {
    double g2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double d = 0.0;
#pragma unroll
      for (int c = 0; c < NC; ++c) d += ((c >> k) & 1) ? u[c][f] : -u[c][f];
      d *= inv;
      g2 += d * d;
    }
    out[3 * e + f] = sqrt(g2);
  }
}

}  // namespace

cudaError_t launch_element_gradient(int dim, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                    const int32_t* hpar, const uint8_t* hnp, const double* U, double* out,
                                    cudaStream_t s) {
  if (n_elem == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n_elem + 255) / 256);
  if (dim == 2) k_element_gradient<2><<<blocks, 256, 0, s>>>(n_elem, conn, level, hpar, hnp, U, out);
  else k_element_gradient<3><<<blocks, 256, 0, s>>>(n_elem, conn, level, hpar, hnp, U, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_plane_integral(int dim, int L, int64_t n_elem, const int32_t* conn, const uint8_t* level,
                                  const int32_t* anchor, const int32_t* hnode, const int32_t* hpar, const uint8_t* hnp,
                                  const double* U, int ax, int64_t coord, double* part, double* out, cudaStream_t s) {
  if (n_elem == 0) return cudaMemsetAsync(out, 0, 3 * sizeof(double), s);
  if (dim == 2)
    k_plane_integral<2><<<kRedBlocks, kFluxThreads, 0, s>>>(n_elem, L, conn, level, anchor, hnode, hpar, hnp, U, ax,
                                                              coord, part);
  else
    k_plane_integral<3><<<kRedBlocks, kFluxThreads, 0, s>>>(n_elem, L, conn, level, anchor, hnode, hpar, hnp, U, ax,
                                                              coord, part);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_parts(kRedBlocks, 3, part, out, s);
}

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
