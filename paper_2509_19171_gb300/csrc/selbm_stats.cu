// Turbulent pipe statistics (Sec. 4, pipe flow): wall shear stress from the wall-face
// nodes and the radially binned mean axial velocity.  Both read the velocity at local
// nodes (moments_kernel output, [E][Np][dim]) of the filtered state.
#include <cuda_runtime.h>

#include "selbm_kernels.cuh"

namespace slb {

// one CTA per element, one thread per wall point of the element: the gradient of u.d at
// the node from the GLL derivative along every reference axis and the chain rule, then
// for every wall face through the node w_s J_s (-mu n.grad(u.d)) and w_s J_s
template <typename Real>
__global__ void wall_stress_kernel(const double *u, int dim, int n, int Np, int affine, const Real *el_drdx,
                                   const Real *drdx, const Real *Dm, const WallPt<Real> *walls, const int32_t *wall_off,
                                   double d0, double d1, double d2, double mu, double *out) {
  const int e = blockIdx.x;
  const int w0 = wall_off[e], nw = wall_off[e + 1] - w0;
  const double dir[3] = {d0, d1, d2};
  for (int k = threadIdx.x; k < nw; k += blockDim.x) {
    const WallPt<Real> &wp = walls[w0 + k];
    const int i = wp.i;
    const int ii[3] = {i % n, (i / n) % n, dim == 3 ? i / (n * n) : 0};
    const int st[3] = {1, n, n * n};
    double dr[3] = {0, 0, 0};
    for (int l = 0; l < dim; ++l) {
      const int base = i - ii[l] * st[l];
      double s = 0;
      for (int q = 0; q < n; ++q) {
        const double *uq = u + ((size_t)e * Np + base + q * st[l]) * dim;
        double ud = 0;
        for (int c = 0; c < dim; ++c) ud += uq[c] * dir[c];
        s += (double)Dm[ii[l] * n + q] * ud;
      }
      dr[l] = s;
    }
    double grad[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c)
      for (int l = 0; l < dim; ++l) {
        const double g = affine ? (double)el_drdx[((size_t)e * dim + l) * dim + c]
                                : (double)drdx[(((size_t)e * Np + i) * dim + l) * dim + c];
        grad[c] += g * dr[l];
      }
    double num = 0, den = 0;
    for (int f = 0; f < wp.nf; ++f) {
      double dn = 0;
      for (int c = 0; c < dim; ++c) dn += (double)wp.n[f][c] * grad[c];
      num += (double)wp.wsJs[f] * (-mu * dn);
      den += (double)wp.wsJs[f];
    }
    out[2 * (w0 + k)] = num;
    out[2 * (w0 + k) + 1] = den;
  }
}

// per-block partial sums over unique nodes: bin b of node g = min(floor(r nbins / R),
// nbins - 1) with r its distance from the axis line; sums of M_g (u.a) and M_g
__global__ void radial_profile_kernel(const double *u, int dim, const int32_t *first, const double *xg,
                                      const double *mass, int G, double o0, double o1, double o2, double a0, double a1,
                                      double a2, double radius, int nbins, double *partial) {
  extern __shared__ double hist[];   // [nbins][2]
  for (int b = threadIdx.x; b < 2 * nbins; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const double o[3] = {o0, o1, o2}, a[3] = {a0, a1, a2};
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    double x[3] = {0, 0, 0}, along = 0;
    for (int c = 0; c < dim; ++c) {
      x[c] = xg[(size_t)g * dim + c] - o[c];
      along += x[c] * a[c];
    }
    double r2 = 0;
    for (int c = 0; c < dim; ++c) {
      const double y = x[c] - along * a[c];
      r2 += y * y;
    }
    int b = (int)floor(sqrt(r2) * nbins / radius);
    b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
    const double *ug = u + (size_t)first[g] * dim;
    double ua = 0;
    for (int c = 0; c < dim; ++c) ua += ug[c] * a[c];
    atomicAdd(&hist[2 * b], mass[g] * ua);
    atomicAdd(&hist[2 * b + 1], mass[g]);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2 * nbins; b += blockDim.x) partial[(size_t)blockIdx.x * 2 * nbins + b] = hist[b];
}

template <typename Real>
cudaError_t launch_wall_stress(const double *u, int dim, int n, int Np, int E, int affine, const Real *el_drdx,
                               const Real *drdx, const Real *Dm, const void *walls, const int32_t *wall_off,
                               const double dir[3], double mu, double *out, cudaStream_t s) {
  wall_stress_kernel<Real><<<E, 64, 0, s>>>(u, dim, n, Np, affine, el_drdx, drdx, Dm, (const WallPt<Real> *)walls,
                                            wall_off, dir[0], dir[1], dir[2], mu, out);
  return cudaGetLastError();
}
template cudaError_t launch_wall_stress<double>(const double *, int, int, int, int, int, const double *, const double *,
                                                const double *, const void *, const int32_t *, const double *, double,
                                                double *, cudaStream_t);
template cudaError_t launch_wall_stress<float>(const double *, int, int, int, int, int, const float *, const float *,
                                               const float *, const void *, const int32_t *, const double *, double,
                                               double *, cudaStream_t);

cudaError_t launch_radial_profile(const double *u, int dim, const int32_t *first, const double *xg, const double *mass,
                                  int G, const double origin[3], const double axis[3], double radius, int nbins,
                                  int blocks, double *partial, cudaStream_t s) {
  radial_profile_kernel<<<blocks, 256, 2 * nbins * sizeof(double), s>>>(
      u, dim, first, xg, mass, G, origin[0], origin[1], origin[2], axis[0], axis[1], axis[2], radius, nbins, partial);
  return cudaGetLastError();
}

}  // namespace slb
