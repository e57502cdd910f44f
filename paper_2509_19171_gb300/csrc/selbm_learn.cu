// Learned per-element filter control: element features, the control kernel that
// picks each element's filter transfer function, the drift check that falls back
// to the fixed filter, per-element errors against a higher-order run, and the
// MLP training kernels.  The network: 2(N+1) log shell energies -> 64 tanh ->
// 64 tanh -> 2 outputs -> (gamma = 0.5 sigmoid(o0), kc = 2 + (N-3) sigmoid(o1)).
// Parameter vector: W1[64][nin], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "selbm_learn.cuh"
#include "selbm_setup.h"
#include "selbm_lattice.cuh"

namespace slb {

constexpr int kH = 64;
constexpr int kTile = 64;     // samples per training tile

int mlp_nparams(int nin) { return kH * nin + kH + kH * kH + kH + 2 * kH + 2; }

// ---------------------------------------------------------------------------
// learned filter pass (one CTA per element): gather the element tile, features
// from its moments, network -> (gamma, kc) -> transfer function, then (when an
// output is given) filter the tile with V diag(sigma) V^-1 along every axis and
// write element-interior nodes to fout and the weighted share wJ f of boundary
// nodes to the trace, for the mass-weighted assembly of shared nodes.
// ---------------------------------------------------------------------------
template <typename Real, int LAT>
__global__ void __launch_bounds__(256) control_kernel(const ControlArgs<Real> c) {
  constexpr int Q = LT<LAT>::v.Q, DIM = LT<LAT>::v.D;
  constexpr VelTab V = LT<LAT>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = c.n, Np = c.Np, nin = 2 * n;
  Real *sf = reinterpret_cast<Real *>(smem_raw);     // [Q][Np] tile
  Real *q = sf + Q * Np;                               // [2][Np] (rho - rho0, |u|) -> modal
  Real *sVi = q + 2 * Np;                              // [n][n]
  Real *sF = sVi + n * n;                              // [n][n] element filter
  Real *sE = sF + n * n;                               // [2][n] shell energies
  Real *sx = sE + 2 * n;                               // [nin] features, then scaled inputs
  Real *h1 = sx + nin;                                 // [64]
  Real *h2 = h1 + kH;                                  // [64]
  Real *so = h2 + kH;                                  // [2]
  Real *ssig = so + 2;                                 // [n]
  __shared__ double red[2][256];
  __shared__ int in_range;
  const int e = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int32_t *l2g = c.l2g + (size_t)e * Np;
  for (int k = tid; k < n * n; k += T) sVi[k] = c.Vinv[k];
  auto weight = [&](int i) -> Real {
    if (c.affine) {
      const int i0 = i % n, i1 = (i / n) % n, i2 = DIM == 3 ? i / (n * n) : 0;
      return c.el_J[e] * c.gllw[i0] * c.gllw[i1] * (DIM == 3 ? c.gllw[i2] : Real(1));
    }
    return c.wJ[(size_t)e * Np + i];
  };
  double pm = 0.0, pk = 0.0;
  for (int i = tid; i < Np; i += T) {
    const size_t g = l2g[i];
    Real drho = 0, j[3] = {0, 0, 0};
    static_for<0, Q>([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      const Real v = c.f[(size_t)a * c.Gs + g];
      sf[a * Np + i] = v;
      drho += v;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        if (V.e[a][k] > 0) j[k] += v;
        else if (V.e[a][k] < 0) j[k] -= v;
      }
    });
    const Real rho = Real(c.rho0) + drho;
    Real uu = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) uu += (j[k] / rho) * (j[k] / rho);
    q[i] = drho;
    q[Np + i] = sqrt(uu);
    const Real wq = weight(i);
    pm += (double)wq * (double)rho;
    pk += 0.5 * c.rho0 * (double)wq * (double)uu;
  }
  if (c.acc) {
    red[0][tid] = pm;
    red[1][tid] = pk;
  }
  if (tid == 0) in_range = 1;
  __syncthreads();
  if (c.acc) {
    for (int s = T / 2; s > 0; s >>= 1) {
      if (tid < s) { red[0][tid] += red[0][tid + s]; red[1][tid] += red[1][tid + s]; }
      __syncthreads();
    }
    if (tid == 0) { atomicAdd(&c.acc[0], red[0][0]); atomicAdd(&c.acc[1], red[1][0]); }
  }
  // modal coefficients: V^{-1} along every axis, both fields
  const int nl = Np / n;
  for (int axis = 0; axis < DIM; ++axis) {
    const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
    for (int t = tid; t < 2 * nl; t += T) {
      const int fld = t / nl, L = t - fld * nl;
      const int base = axis == 0 ? L * n : (axis == 1 ? (L % n) + n * n * (L / n) : L);
      Real *row = q + fld * Np + base;
      Real v[kMaxN + 1], o[kMaxN + 1];
      for (int k = 0; k < n; ++k) v[k] = row[k * stride];
      for (int m = 0; m < n; ++m) {
        Real s = 0;
        for (int k = 0; k < n; ++k) s += sVi[m * n + k] * v[k];
        o[m] = s;
      }
      for (int m = 0; m < n; ++m) row[m * stride] = o[m];
    }
    __syncthreads();
  }
  // shell energies in a fixed order, then log10 features
  if (tid < 2 * n) {
    const int fld = tid / n, k = tid - fld * n;
    Real s = 0;
    for (int i = 0; i < Np; ++i) {
      const int i0 = i % n, i1 = (i / n) % n, i2 = DIM == 3 ? i / (n * n) : 0;
      if (max(i0, max(i1, i2)) == k) s += q[fld * Np + i] * q[fld * Np + i];
    }
    const Real x = log10(s + Real(1e-30));
    sx[tid] = x;
    if (c.feat_out) c.feat_out[(size_t)e * nin + tid] = (float)x;
    if (c.W) {
      const Real lo = c.lo[tid], hi = c.hi[tid];
      if (!(x >= lo && x <= hi)) in_range = 0;
      sx[tid] = Real(2) * (x - lo) / (hi - lo) - Real(1);
    }
  }
  if (!c.W) return;
  __syncthreads();
  const bool use_net = in_range && !(c.flag && *c.flag);
  if (use_net) {
    const __nv_bfloat16 *W1 = c.W, *b1 = W1 + kH * nin, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + 2 * kH;
    if (tid < kH) {
      Real z = (Real)__bfloat162float(b1[tid]);
      for (int i = 0; i < nin; ++i) z += (Real)__bfloat162float(W1[tid * nin + i]) * sx[i];
      h1[tid] = tanh(z);
    }
    __syncthreads();
    if (tid < kH) {
      Real z = (Real)__bfloat162float(b2[tid]);
      for (int k = 0; k < kH; ++k) z += (Real)__bfloat162float(W2[tid * kH + k]) * h1[k];
      h2[tid] = tanh(z);
    }
    __syncthreads();
    if (tid < 2) {
      Real z = (Real)__bfloat162float(b3[tid]);
      for (int k = 0; k < kH; ++k) z += (Real)__bfloat162float(W3[tid * kH + k]) * h2[k];
      so[tid] = z;
    }
    __syncthreads();
  } else if (tid == 0 && c.n_fallback) {
    atomicAdd(c.n_fallback, 1);
  }
  if (tid < n) {
    Real sig = c.fixed_sigma[tid];
    if (use_net) {
      const Real gam = Real(0.5) / (Real(1) + exp(-so[0]));
      const Real kc = Real(2) + Real(c.N - 3) / (Real(1) + exp(-so[1]));
      sig = Real(1);
      if (tid > kc) {
        const Real r = (Real(tid) - kc) / (Real(c.N) - kc);
        sig = Real(1) - gam * r * r;
      }
    }
    ssig[tid] = sig;
    if (c.sigma_out) c.sigma_out[(size_t)e * n + tid] = sig;
  }
  if (!c.fout) return;
  __syncthreads();
  // F_e = V diag(sigma) V^{-1}; its end rows are exact identity rows
  for (int k = tid; k < n * n; k += T) {
    const int m = k / n, jj = k - m * n;
    Real s = 0;
    for (int qq = 0; qq < n; ++qq) s += c.Vm[m * n + qq] * ssig[qq] * sVi[qq * n + jj];
    if (m == 0 || m == n - 1) s = (m == jj) ? Real(1) : Real(0);
    sF[k] = s;
  }
  __syncthreads();
  for (int axis = 0; axis < DIM; ++axis) {
    const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
    for (int t = tid; t < Q * nl; t += T) {
      const int a = t / nl, L = t - a * nl;
      const int base = axis == 0 ? L * n : (axis == 1 ? (L % n) + n * n * (L / n) : L);
      Real *row = sf + a * Np + base;
      Real v[kMaxN + 1], o[kMaxN + 1];
      for (int k = 0; k < n; ++k) v[k] = row[k * stride];
      for (int m = 0; m < n; ++m) {
        Real s = 0;
        for (int k = 0; k < n; ++k) s += sF[m * n + k] * v[k];
        o[m] = s;
      }
      for (int m = 0; m < n; ++m) row[m * stride] = o[m];
    }
    __syncthreads();
  }
  const size_t EN = (size_t)c.E * c.Nb;
  for (int idx = tid; idx < Q * Np; idx += T) {
    const int a = idx / Np, i = idx - a * Np;
    const int b = c.bslot[i];
    if (b < 0) c.fout[(size_t)a * c.Gs + l2g[i]] = sf[idx];
    else c.T[a * EN + (size_t)e * c.Nb + b] = weight(i) * sf[idx];
  }
}

// drift check after a control pass: fall back to the fixed filter for the rest of
// the run if the relative mass change since the previous step exceeds its bound, or
// (unforced runs, ke_bound > 0) the kinetic energy grew by more than ke_bound
__global__ void drift_check_kernel(double *acc, int *flag, double mass_bound, double ke_bound, int check_ke) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // acc: [0] mass, [1] KE (this step), [2] previous mass, [3] previous KE, [4] have previous
  if (acc[4] != 0.0) {
    const double dm = fabs(acc[0] - acc[2]) / fabs(acc[2]);
    const bool ke_up = check_ke && ke_bound > 0.0 && acc[1] > acc[3] * (1.0 + ke_bound);
    if (dm > mass_bound || ke_up) *flag = 1;
  }
  acc[2] = acc[0];
  acc[3] = acc[1];
  acc[4] = 1.0;
  acc[0] = 0.0;
  acc[1] = 0.0;
}

template <typename Real, int LAT>
static cudaError_t launch_control_t(const ControlArgs<Real> &c, cudaStream_t s) {
  const int Q = LT<LAT>::v.Q;
  const size_t smem = (size_t)(Q * c.Np + 2 * c.Np + 2 * c.n * c.n + 2 * c.n + 2 * c.n + 2 * kH + 2 + c.n) * sizeof(Real);
  auto k = control_kernel<Real, LAT>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<c.E, 256, smem, s>>>(c);
  return cudaGetLastError();
}

size_t control_smem_bytes(int lat, int Np, int n, int real_size) {
  const int Q = lat == SELBM_D2Q9 ? 9 : (lat == SELBM_D3Q19 ? 19 : 27);
  return (size_t)(Q * Np + 2 * Np + 2 * n * n + 4 * n + 2 * kH + 2 + n) * real_size;
}

template <typename Real>
cudaError_t launch_control(int lat, const ControlArgs<Real> &c, cudaStream_t s) {
  switch (lat) {
    case SELBM_D2Q9: return launch_control_t<Real, SELBM_D2Q9>(c, s);
    case SELBM_D3Q19: return launch_control_t<Real, SELBM_D3Q19>(c, s);
    case SELBM_D3Q27: return launch_control_t<Real, SELBM_D3Q27>(c, s);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t launch_control<double>(int, const ControlArgs<double> &, cudaStream_t);
template cudaError_t launch_control<float>(int, const ControlArgs<float> &, cudaStream_t);

cudaError_t launch_drift_check(double *acc, int *flag, double mass_bound, double ke_bound, int check_ke, cudaStream_t s) {
  drift_check_kernel<<<1, 32, 0, s>>>(acc, flag, mass_bound, ke_bound, check_ke);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-element error against a higher-order run on the same mesh
// ---------------------------------------------------------------------------
__global__ void element_errors_kernel(int dim, int n, int nR, const double *rho, const double *u, const double *rhoR,
                                      const double *uR, const double *I, const double *wq, double *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Np = dim == 3 ? n * n * n : n * n, NpR = dim == 3 ? nR * nR * nR : nR * nR;
  const int cap = NpR > Np ? NpR : Np;
  double *A = reinterpret_cast<double *>(smem_raw);
  double *B = A + cap * 1;
  double *sI = A + 2 * cap * 1;   // [n][nR]
  __shared__ double red[256];
  const int e = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  for (int k = tid; k < n * nR; k += T) sI[k] = I[k];
  double acc = 0.0;
  for (int fld = 0; fld <= dim; ++fld) {
    __syncthreads();
    for (int i = tid; i < NpR; i += T)
      A[i] = fld == 0 ? rhoR[(size_t)e * NpR + i] : uR[((size_t)e * NpR + i) * dim + fld - 1];
    __syncthreads();
    // sizes along (axis0, axis1, axis2): start (nR, nR, nR); interpolate one axis at a time
    int d0 = nR, d1 = nR, d2 = dim == 3 ? nR : 1;
    double *src = A, *dst = B;
    for (int axis = 0; axis < dim; ++axis) {
      const int o0 = axis == 0 ? n : d0, o1 = axis == 1 ? n : d1, o2 = axis == 2 ? n : d2;
      for (int t = tid; t < o0 * o1 * o2; t += T) {
        const int a0 = t % o0, a1 = (t / o0) % o1, a2 = t / (o0 * o1);
        double s = 0.0;
        for (int k = 0; k < nR; ++k) {
          int b0 = a0, b1 = a1, b2 = a2;
          int row;
          if (axis == 0) { b0 = k; row = a0; } else if (axis == 1) { b1 = k; row = a1; } else { b2 = k; row = a2; }
          s += sI[row * nR + k] * src[b0 + d0 * (b1 + d1 * b2)];
        }
        dst[t] = s;
      }
      __syncthreads();
      d0 = o0; d1 = o1; d2 = o2;
      double *tmp = src; src = dst; dst = tmp;
    }
    for (int i = tid; i < Np; i += T) {
      const double v = fld == 0 ? rho[(size_t)e * Np + i] : u[((size_t)e * Np + i) * dim + fld - 1];
      const double dlt = v - src[i];
      acc += wq[(size_t)e * Np + i] * dlt * dlt;
    }
  }
  red[tid] = acc;
  __syncthreads();
  for (int s = T / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) err[e] = red[0];
}

cudaError_t launch_element_errors(int E, int dim, int n, int nR, const double *rho, const double *u, const double *rhoR,
                                  const double *uR, const double *I, const double *wq, double *err, cudaStream_t s) {
  const int Np = dim == 3 ? n * n * n : n * n, NpR = dim == 3 ? nR * nR * nR : nR * nR;
  const int cap = std::max(Np, NpR);
  const size_t smem = (size_t)(2 * cap + n * nR) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(element_errors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  element_errors_kernel<<<E, 256, smem, s>>>(dim, n, nR, rho, u, rhoR, uR, I, wq, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MLP training: one CTA per 64-sample tile computes the tile's loss and gradient sums
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix32(uint32_t x, uint64_t key, uint32_t r) {
  uint64_t z = (uint64_t)x ^ (key + 0x9E3779B97F4A7C15ull * (r + 1));
  z ^= z >> 31; z *= 0x7FB5D329728EA185ull;
  z ^= z >> 27; z *= 0x81DADEF4BC2DD44Dull;
  z ^= z >> 33;
  return (uint32_t)z;
}

// bijection of [0, M): four-round Feistel network on 2h bits (4^h >= M), cycle walking
__device__ int64_t shuffle_index(int64_t i, int64_t M, int h, uint64_t key) {
  const uint32_t mask = (1u << h) - 1u;
  uint64_t x = (uint64_t)i;
  for (int walk = 0; walk < 4096; ++walk) {
    uint32_t L = (uint32_t)(x >> h) & mask, R = (uint32_t)x & mask;
    for (uint32_t r = 0; r < 4; ++r) {
      const uint32_t nL = R, nR = L ^ (mix32(R, key, r) & mask);
      L = nL; R = nR;
    }
    x = ((uint64_t)L << h) | R;
    if ((int64_t)x < M) return (int64_t)x;
  }
  return i;   // unreachable for a bijection in practice; keeps the loop bounded
}

struct TileArgs {
  const float *params;
  int nin, N;
  const float *X, *Y;     // [M][nin] scaled inputs, [M][2] targets (gamma, kc)
  int64_t M, start, count;   // samples [start, start + count) of the (shuffled) order
  int h;                   // shuffle bits per half, 0 = identity order
  uint64_t key;
  float *gpart, *lpart;    // [tiles][P], [tiles]
  float *out;              // forward mode: [M][2] (gamma, kc)
  int bf16;                // forward mode: round weights to bfloat16
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(256) mlp_tile_kernel(const TileArgs a, int forward_only) {
  extern __shared__ __align__(16) float sm[];
  const int nin = a.nin, P = kH * nin + kH + kH * kH + kH + 2 * kH + 2;
  float *W = sm;                       // [P]
  float *S = W + P;                    // [64][nin]
  float *H1 = S + kTile * nin;         // [64][64]
  float *H2 = H1 + kTile * kH;         // [64][64]
  float *D2 = H2 + kTile * kH;         // [64][64]  dZ2
  float *D1 = D2 + kTile * kH;         // [64][64]  dZ1
  float *O = D1 + kTile * kH;          // [64][2]
  float *dO = O + kTile * 2;           // [64][2]
  float *Yt = dO + kTile * 2;          // [64][2]
  int *idx = reinterpret_cast<int *>(Yt + kTile * 2);   // [64] sample index or -1
  const int tid = threadIdx.x, T = blockDim.x;
  const float *W1 = W, *b1 = W1 + kH * nin, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + 2 * kH;
  for (int k = tid; k < P; k += T) W[k] = a.bf16 ? bf16r(a.params[k]) : a.params[k];
  for (int s = tid; s < kTile; s += T) {
    const int64_t pos = (int64_t)blockIdx.x * kTile + s;
    int64_t sidx = -1;
    if (pos < a.count) {
      const int64_t g = a.start + pos;
      sidx = a.h > 0 ? shuffle_index(g, a.M, a.h, a.key) : g;
    }
    idx[s] = (int)sidx;
  }
  __syncthreads();
  for (int k = tid; k < kTile * nin; k += T) {
    const int s = k / nin, i = k - s * nin;
    S[k] = idx[s] >= 0 ? a.X[(size_t)idx[s] * nin + i] : 0.f;
  }
  for (int k = tid; k < kTile * 2; k += T) {
    const int s = k / 2;
    Yt[k] = (idx[s] >= 0 && !forward_only) ? a.Y[(size_t)idx[s] * 2 + (k & 1)] : 0.f;
  }
  __syncthreads();
  for (int k = tid; k < kTile * kH; k += T) {
    const int s = k / kH, j = k - s * kH;
    float z = b1[j];
    for (int i = 0; i < nin; ++i) z += W1[j * nin + i] * S[s * nin + i];
    H1[k] = tanhf(z);
  }
  __syncthreads();
  for (int k = tid; k < kTile * kH; k += T) {
    const int s = k / kH, j = k - s * kH;
    float z = b2[j];
    for (int m = 0; m < kH; ++m) z += W2[j * kH + m] * H1[s * kH + m];
    H2[k] = tanhf(z);
  }
  __syncthreads();
  const float Nm3 = (float)(a.N - 3);
  for (int k = tid; k < kTile * 2; k += T) {
    const int s = k / 2, c = k & 1;
    float z = b3[c];
    for (int m = 0; m < kH; ++m) z += W3[c * kH + m] * H2[s * kH + m];
    const float sg = 1.f / (1.f + expf(-z));
    const float val = c == 0 ? 0.5f * sg : 2.f + Nm3 * sg;
    O[k] = val;
    if (forward_only) {
      if (idx[s] >= 0) a.out[(size_t)idx[s] * 2 + c] = val;
    } else {
      const float scale = c == 0 ? 0.5f : Nm3;
      const float r = idx[s] >= 0 ? (val - Yt[k]) / scale : 0.f;
      dO[k] = 2.f * r / scale * (c == 0 ? 0.5f : Nm3) * sg * (1.f - sg);   // dL/dz (unscaled by batch)
      O[k] = r * r;
    }
  }
  if (forward_only) return;
  __syncthreads();
  float *g = a.gpart + (size_t)blockIdx.x * P;
  float *gW1 = g, *gb1 = gW1 + kH * nin, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gW3 = gb2 + kH, *gb3 = gW3 + 2 * kH;
  if (tid == 0) {
    float l = 0.f;
    for (int k = 0; k < kTile * 2; ++k) l += O[k];
    a.lpart[blockIdx.x] = l;
  }
  // output layer
  for (int k = tid; k < 2 * kH; k += T) {
    const int c = k / kH, m = k - c * kH;
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += dO[t * 2 + c] * H2[t * kH + m];
    gW3[k] = s;
  }
  if (tid < 2) {
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += dO[t * 2 + tid];
    gb3[tid] = s;
  }
  for (int k = tid; k < kTile * kH; k += T) {
    const int s = k / kH, m = k - s * kH;
    const float dh = dO[s * 2] * W3[m] + dO[s * 2 + 1] * W3[kH + m];
    D2[k] = dh * (1.f - H2[k] * H2[k]);
  }
  __syncthreads();
  for (int k = tid; k < kH * kH; k += T) {
    const int j = k / kH, m = k - j * kH;
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += D2[t * kH + j] * H1[t * kH + m];
    gW2[k] = s;
  }
  for (int j = tid; j < kH; j += T) {
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += D2[t * kH + j];
    gb2[j] = s;
  }
  for (int k = tid; k < kTile * kH; k += T) {
    const int s = k / kH, m = k - s * kH;
    float dh = 0.f;
    for (int j = 0; j < kH; ++j) dh += D2[s * kH + j] * W2[j * kH + m];
    D1[k] = dh * (1.f - H1[k] * H1[k]);
  }
  __syncthreads();
  for (int k = tid; k < kH * nin; k += T) {
    const int j = k / nin, i = k - j * nin;
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += D1[t * kH + j] * S[t * nin + i];
    gW1[k] = s;
  }
  for (int j = tid; j < kH; j += T) {
    float s = 0.f;
    for (int t = 0; t < kTile; ++t) s += D1[t * kH + j];
    gb1[j] = s;
  }
}

// sum tile partials in tile order (deterministic), scale, then optionally Adam
__global__ void mlp_reduce_kernel(const float *gpart, const float *lpart, int tiles, int P, float scale, float *grad,
                                  float *loss, float *params, float *m, float *v, float lr, float b1c, float b2c,
                                  int adam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss) {
    float l = 0.f;
    for (int t = 0; t < tiles; ++t) l += lpart[t];
    *loss = l * scale;
  }
  if (p >= P) return;
  float gs = 0.f;
  for (int t = 0; t < tiles; ++t) gs += gpart[(size_t)t * P + p];
  gs *= scale;
  if (grad) grad[p] = gs;
  if (adam) {
    const float mm = 0.9f * m[p] + 0.1f * gs;
    const float vv = 0.999f * v[p] + 0.001f * gs * gs;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm / b1c) / (sqrtf(vv / b2c) + 1e-8f);
  }
}

static size_t tile_smem(int nin) {
  const int P = mlp_nparams(nin);
  return (size_t)(P + kTile * nin + 4 * kTile * kH + 6 * kTile) * sizeof(float) + kTile * sizeof(int);
}

static cudaError_t tile_attr(int nin) {
  return cudaFuncSetAttribute(mlp_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem(nin));
}

cudaError_t mlp_grad(const float *params, int nin, int N, const float *X, const float *Y, int64_t M, float *grad,
                     float *loss, cudaStream_t s) {
  const int P = mlp_nparams(nin);
  const int tiles = (int)((M + kTile - 1) / kTile);
  float *gpart = nullptr, *lpart = nullptr;
  cudaError_t e = cudaMalloc(&gpart, (size_t)tiles * P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&lpart, (size_t)tiles * sizeof(float));
  if (e == cudaSuccess) e = tile_attr(nin);
  if (e == cudaSuccess) {
    TileArgs a{params, nin, N, X, Y, M, 0, M, 0, 0, gpart, lpart, nullptr, 0};
    mlp_tile_kernel<<<tiles, 256, tile_smem(nin), s>>>(a, 0);
    mlp_reduce_kernel<<<(P + 255) / 256, 256, 0, s>>>(gpart, lpart, tiles, P, 1.f / (float)M, grad, loss, nullptr,
                                                     nullptr, nullptr, 0.f, 1.f, 1.f, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(gpart);
  cudaFree(lpart);
  return e;
}

cudaError_t mlp_forward(const float *params, int nin, int N, const float *X, int64_t M, int bf16, float *out,
                        cudaStream_t s) {
  cudaError_t e = tile_attr(nin);
  if (e != cudaSuccess) return e;
  const int tiles = (int)((M + kTile - 1) / kTile);
  TileArgs a{params, nin, N, X, nullptr, M, 0, M, 0, 0, nullptr, nullptr, out, bf16};
  mlp_tile_kernel<<<tiles, 256, tile_smem(nin), s>>>(a, 1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t mlp_train(float *params, float *m, float *v, int nin, int N, const float *X, const float *Y, int64_t M,
                      int batch, int epochs, float lr, uint64_t seed, int64_t *adam_t, float *loss_hist,
                      cudaStream_t s) {
  const int P = mlp_nparams(nin);
  const int tiles = (batch + kTile - 1) / kTile;
  int h = 1;
  while ((int64_t)1 << (2 * h) < M) ++h;
  float *gpart = nullptr, *lpart = nullptr, *dloss = nullptr;
  cudaError_t e = cudaMalloc(&gpart, (size_t)tiles * P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&lpart, (size_t)tiles * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dloss, sizeof(float));
  if (e == cudaSuccess) e = tile_attr(nin);
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    double lsum = 0.0;
    int64_t nb = 0;
    const uint64_t key = seed * 0x9E3779B97F4A7C15ull + (uint64_t)ep;
    for (int64_t start = 0; start < M && e == cudaSuccess; start += batch) {
      const int64_t cnt = std::min<int64_t>(batch, M - start);
      const int tl = (int)((cnt + kTile - 1) / kTile);
      TileArgs a{params, nin, N, X, Y, M, start, cnt, h, key, gpart, lpart, nullptr, 0};
      mlp_tile_kernel<<<tl, 256, tile_smem(nin), s>>>(a, 0);
      const int64_t t = ++(*adam_t);
      const float b1c = 1.f - powf(0.9f, (float)t), b2c = 1.f - powf(0.999f, (float)t);
      mlp_reduce_kernel<<<(P + 255) / 256, 256, 0, s>>>(gpart, lpart, tl, P, 1.f / (float)cnt, nullptr, dloss, params,
                                                       m, v, lr, b1c, b2c, 1);
      e = cudaGetLastError();
      if (loss_hist && e == cudaSuccess) {
        float l = 0.f;
        e = cudaMemcpyAsync(&l, dloss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        lsum += l * (double)cnt;
        nb += cnt;
      }
    }
    if (loss_hist && nb > 0) loss_hist[ep] = (float)(lsum / (double)nb);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(gpart);
  cudaFree(lpart);
  cudaFree(dloss);
  return e;
}

}  // namespace slb
