// Allocation-free quadrature integrals of a state given by the caller.
//
// Who needs this: a caller that hands the library device buffers it already
// owns and does not let it allocate -- for instance a host application whose
// own memory pool has reserved the device memory up front, or a monitoring
// hook called every step inside a time loop, where cudaMalloc / cudaFree would
// add an implicit device synchronisation.  selbm_diagnostics cannot serve such
// a caller: it needs a handle, and selbm_create allocates.
//
// The per-element partial sums live in a fixed file-scope device array of
// SELBM_NOALLOC_MAX_ELEMS x 6 doubles (3 MiB), which every GPU that loads the
// library keeps until the process exits.  Host code never uses the array's
// name as an address: the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/selbm.h"
#include "selbm_setup.h"

namespace {

constexpr int kMaxElems = SELBM_NOALLOC_MAX_ELEMS;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_integral_scratch[kMaxElems * 6];

std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

struct VelTable {
  int8_t e[slb::kMaxQ][3];
  int32_t Q, dim;
};

// one block per element: sum over its nodes of w rho, w rho u, w rho0 |u|^2 / 2,
// and the count of non-finite state values; written to scratch[e][0..5]
__global__ void element_integrals_kernel(const double *f, const double *w, int nelem, int np, double rho0,
                                         VelTable vt, double *scratch) {
  __shared__ double red[6][kThreads];
  const int e = blockIdx.x;
  const size_t nloc = (size_t)nelem * np;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const size_t q = (size_t)e * np + i;
    double rho = 0, j[3] = {0, 0, 0};
    for (int a = 0; a < vt.Q; ++a) {
      const double v = f[(size_t)a * nloc + q];
      if (!isfinite(v)) acc[5] += 1.0;
      rho += v;
      for (int k = 0; k < vt.dim; ++k) j[k] += vt.e[a][k] * v;
    }
    const double wq = w[q];
    acc[0] += wq * rho;
    double uu = 0;
    for (int k = 0; k < vt.dim; ++k) {
      acc[1 + k] += wq * j[k];
      uu += (j[k] / rho) * (j[k] / rho);
    }
    acc[4] += 0.5 * rho0 * wq * uu;
  }
  for (int c = 0; c < 6; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 6; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6) scratch[(size_t)e * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// one block: fixed-order sum of the per-element partials -> out[0..5]
__global__ void sum_elements_kernel(const double *scratch, int nelem, double *out) {
  __shared__ double red[6][kThreads];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < nelem; e += blockDim.x)
    for (int c = 0; c < 6; ++c) acc[c] += scratch[(size_t)e * 6 + c];
  for (int c = 0; c < 6; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 6; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = red[threadIdx.x][0];
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_integral_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int selbm_integrals_noalloc(int32_t lattice, int32_t nelem, int32_t np, const double *f, const double *w,
                                       double rho0, double *out, void *cuda_stream) {
  if (!f || !w || !out || nelem <= 0 || np <= 0) return SELBM_ERR_ARG;
  if (nelem > kMaxElems) return SELBM_ERR_ARG;   // scratch holds at most SELBM_NOALLOC_MAX_ELEMS elements
  slb::Lattice L;
  if (!slb::build_lattice(lattice, &L)) return SELBM_ERR_ARG;
  VelTable vt{};
  vt.Q = L.Q;
  vt.dim = L.dim;
  for (int a = 0; a < L.Q; ++a)
    for (int k = 0; k < 3; ++k) vt.e[a][k] = (int8_t)L.e[3 * a + k];
  double *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return SELBM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  element_integrals_kernel<<<nelem, kThreads, 0, s>>>(f, w, nelem, np, rho0, vt, scratch);
  sum_elements_kernel<<<1, kThreads, 0, s>>>(scratch, nelem, out);
  return cudaGetLastError() == cudaSuccess ? SELBM_OK : SELBM_ERR_CUDA;
}
