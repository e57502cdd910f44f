// Hot-path kernels of the filtered SELBM (paper Sec. 2): per-stage element
// kernel (optional filter + BGK collision in stage 1, tensor-product GLL
// derivative with metrics, flux bounce-back, Runge-Kutta combination at
// element-interior nodes, weighted contributions of element-boundary nodes),
// and the assembly kernel that finishes the shared nodes.
#include <cstdio>

#include "selbm_kernels.cuh"
#include "selbm_setup.h"

namespace slb {

template <int LAT> struct Lat;
template <> struct Lat<SELBM_D2Q9> { static constexpr int Q = 9, D = 2; };
template <> struct Lat<SELBM_D3Q19> { static constexpr int Q = 19, D = 3; };
template <> struct Lat<SELBM_D3Q27> { static constexpr int Q = 27, D = 3; };

__constant__ int8_t c_e[3][kMaxQ][3];
__constant__ double c_td[3][kMaxQ];
__constant__ float c_tf[3][kMaxQ];
__constant__ int8_t c_opp[3][kMaxQ];

void upload_lattice_constants() {
  int8_t e[3][kMaxQ][3] = {};
  double td[3][kMaxQ] = {};
  float tf[3][kMaxQ] = {};
  int8_t opp[3][kMaxQ] = {};
  for (int l = 0; l < 3; ++l) {
    Lattice L;
    build_lattice(l, &L);
    for (int a = 0; a < L.Q; ++a) {
      for (int k = 0; k < 3; ++k) e[l][a][k] = (int8_t)L.e[3 * a + k];
      td[l][a] = L.t[a];
      tf[l][a] = (float)L.t[a];
      opp[l][a] = (int8_t)L.opp[a];
    }
  }
  cudaMemcpyToSymbol(c_e, e, sizeof(e));
  cudaMemcpyToSymbol(c_td, td, sizeof(td));
  cudaMemcpyToSymbol(c_tf, tf, sizeof(tf));
  cudaMemcpyToSymbol(c_opp, opp, sizeof(opp));
}

template <typename Real> __device__ __forceinline__ Real wt(int lat, int a);
template <> __device__ __forceinline__ double wt<double>(int lat, int a) { return c_td[lat][a]; }
template <> __device__ __forceinline__ float wt<float>(int lat, int a) { return c_tf[lat][a]; }

constexpr int kMaxN1 = kMaxN + 1;

size_t stage_smem_bytes(int lat, int Np, int n, int real_size) {
  const int Q = lat == SELBM_D2Q9 ? 9 : (lat == SELBM_D3Q19 ? 19 : 27);
  return (size_t)(Q * Np + 2 * n * n + Np) * real_size;
}

// ---------------------------------------------------------------------------
// element-tile helpers (tile sf[Q][Np] in shared memory, r index fastest)
// ---------------------------------------------------------------------------

// base index and stride of the line through line-number L along `axis`
__device__ __forceinline__ void line_base(int axis, int L, int n, int *base, int *stride) {
  if (axis == 0) { *base = L * n; *stride = 1; }
  else if (axis == 1) { *base = (L % n) + n * n * (L / n); *stride = n; }
  else { *base = L; *stride = n * n; }
}

// one 1D filter pass along `axis` for every population (lines are disjoint)
template <typename Real, int Q>
__device__ void filter_pass(Real *sf, const Real *sF, int n, int Np, int axis) {
  const int nl = Np / n;
  for (int idx = threadIdx.x; idx < Q * nl; idx += blockDim.x) {
    const int a = idx / nl, L = idx - a * nl;
    int base, stride;
    line_base(axis, L, n, &base, &stride);
    Real *row = sf + a * Np + base;
    Real v[kMaxN1];
#pragma unroll
    for (int k = 0; k < kMaxN1; ++k)
      if (k < n) v[k] = row[k * stride];
    for (int m = 0; m < n; ++m) {
      Real s = 0;
#pragma unroll
      for (int k = 0; k < kMaxN1; ++k)
        if (k < n) s += sF[m * n + k] * v[k];
      row[m * stride] = s;
    }
  }
}

// BGK collision with the higher-order force at local node i (deviation form:
// the tile holds g = f_bar - t rho0).  Sec. 2.1:
//   f_bar^eq = f^eq - dt/2 F**,  f* = f_bar - omega (f_bar - f_bar^eq) + dt F**,  omega = 1/(tau + 1/2)
template <typename Real, int LAT>
__device__ void collide_node(Real *sf, int i, const KParams<Real> &p, Real *srho, int e) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  const int Np = p.Np;
  Real drho = 0, j[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const Real v = sf[a * Np + i];
    drho += v;
#pragma unroll
    for (int k = 0; k < DIM; ++k) j[k] += (Real)c_e[LAT][a][k] * v;
  }
  const Real rho = p.rho0 + drho;
  const Real inv = Real(1) / rho;
  const size_t gid = p.l2g[(size_t)e * Np + i];
  Real ga[3];
  node_accel(p, gid, ga);
  Real u[3] = {0, 0, 0}, F[3] = {0, 0, 0};
  Real uu = 0, uF = 0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    u[k] = j[k] * inv;
    uu += u[k] * u[k];
    if (p.has_force) { F[k] = rho * ga[k]; uF += u[k] * F[k]; }
  }
  const Real ics2 = Real(3), ics4 = Real(9);
  const bool own = p.owner[(size_t)e * Np + i] != 0;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    Real eu = 0, eF = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { eu += (Real)c_e[LAT][a][k] * u[k]; eF += (Real)c_e[LAT][a][k] * F[k]; }
    const Real t = wt<Real>(LAT, a);
    Real feq = t * (drho + rho * (eu * ics2 + Real(0.5) * eu * eu * ics4 - Real(0.5) * uu * ics2));
    Real Fss = 0;
    if (p.has_force) {
      Fss = t * (eu * eF * ics4 - uF * ics2);
      feq -= p.half_dt * Fss;
    }
    const Real v = sf[a * Np + i];
    const Real out = v - p.omega * (v - feq) + p.dt * Fss;
    sf[a * Np + i] = out;
    if (own) p.f0out[a * (size_t)p.Gs + gid] = out;
  }
  srho[i] = rho;
  if (own && p.has_force) p.rho[gid] = rho;
}

// ---------------------------------------------------------------------------
// stage kernel: one CTA per element
// ---------------------------------------------------------------------------
template <typename Real, int LAT, bool AFFINE>
__global__ void __launch_bounds__(512) stage_kernel(const KParams<Real> p) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, Np = p.Np;
  Real *sf = reinterpret_cast<Real *>(smem_raw);
  Real *sD = sf + Q * Np;
  Real *sF = sD + n * n;
  Real *srho = sF + n * n;
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < n * n; k += nt) { sD[k] = p.Dm[k]; sF[k] = p.Fm[k]; }
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  for (int idx = tid; idx < Q * Np; idx += nt) {
    const int a = idx / Np, i = idx - a * Np;
    sf[idx] = p.fin[(size_t)a * p.Gs + l2g[i]];
  }
  __syncthreads();
  if (p.stage == 1) {
    if (p.apply_filter) {
      for (int axis = 0; axis < DIM; ++axis) {
        filter_pass<Real, Q>(sf, sF, n, Np, axis);
        __syncthreads();
      }
    }
    for (int i = tid; i < Np; i += nt) collide_node<Real, LAT>(sf, i, p, srho, e);
    __syncthreads();
  }

  // metric coefficients of the element (affine case)
  Real em[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  Real Je = 0;
  if (AFFINE) {
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int k = 0; k < DIM; ++k) em[l][k] = p.el_drdx[((size_t)e * DIM + l) * DIM + k];
    Je = p.el_J[e];
  }
  const Real ics2 = Real(3);
  const size_t EN = (size_t)p.E * p.Nb;
  for (int idx = tid; idx < Q * Np; idx += nt) {
    const int a = idx / Np, i = idx - a * Np;
    int ii[3] = {i % n, (i / n) % n, DIM == 3 ? i / (n * n) : 0};
    const int strides[3] = {1, n, n * n};
    // e_alpha . grad f = sum_l (sum_k e_k dr_l/dx_k) (D_l f)   (chain rule, Sec. 2.2)
    Real adv = 0;
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      Real coef = 0;
      if (AFFINE) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) coef += (Real)c_e[LAT][a][k] * em[l][k];
      } else {
        const Real *gm = p.drdx + (((size_t)e * Np + i) * DIM + l) * DIM;
#pragma unroll
        for (int k = 0; k < DIM; ++k) coef += (Real)c_e[LAT][a][k] * gm[k];
      }
      if (coef != Real(0)) {
        const Real *row = sf + a * Np + (i - ii[l] * strides[l]);
        const Real *drow = sD + ii[l] * n;
        Real d = 0;
#pragma unroll
        for (int k = 0; k < kMaxN1; ++k)
          if (k < n) d += drow[k] * row[k * strides[l]];
        adv += coef * d;
      }
    }
    const int b = p.bslot[i];
    const size_t gid = l2g[i];
    if (b < 0) {
      Real Fs = 0;
      if (p.has_force) {
        const Real rho_i = p.stage == 1 ? srho[i] : p.rho[gid];
        Real ga[3];
        node_accel(p, gid, ga);
        Real eg = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) eg += (Real)c_e[LAT][a][k] * ga[k];
        Fs = wt<Real>(LAT, a) * eg * rho_i * ics2;
      }
      const Real fprev = sf[idx];
      const Real f0v = p.stage == 1 ? fprev : p.f0[(size_t)a * p.Gs + gid];
      p.fout[(size_t)a * p.Gs + gid] = p.A * f0v + p.B * (fprev + p.dt * (Fs - adv));
    } else {
      Real wJi;
      if (AFFINE) {
        wJi = Je * p.gllw[ii[0]] * p.gllw[ii[1]];
        if (DIM == 3) wJi *= p.gllw[ii[2]];
      } else {
        wJi = p.wJ[(size_t)e * Np + i];
      }
      p.T[a * EN + (size_t)e * p.Nb + b] = -(p.B * p.dt) * wJi * adv;
    }
  }
  // flux bounce-back on the element's wall nodes (Sec. 2.2.1):
  //   + w_s J_s (n.e_a) [f_a - f_opp(a) - 2 t_a rho0 (e_a.u_b)/cs2]  for n.e_a < 0
  const int w0 = p.wall_off[e], w1 = p.wall_off[e + 1];
  if (w1 > w0) {
    __syncthreads();
    for (int idx = tid; idx < Q * (w1 - w0); idx += nt) {
      const int a = idx % Q;
      const WallPt<Real> &wp = p.walls[w0 + idx / Q];
      const int oa = c_opp[LAT][a];
      Real sum = 0;
      for (int f = 0; f < wp.nf; ++f) {
        Real ne = 0, eu = 0;
        const Real *ub = p.wall_u + 3 * (wp.wid[f] - 1);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          ne += wp.n[f][k] * (Real)c_e[LAT][a][k];
          eu += (Real)c_e[LAT][a][k] * ub[k];
        }
        if (ne < Real(0)) {
          const Real jump = sf[a * Np + wp.i] - sf[oa * Np + wp.i] - Real(2) * wt<Real>(LAT, a) * p.rho0 * eu * ics2;
          sum += wp.wsJs[f] * ne * jump;
        }
      }
      p.T[a * EN + (size_t)e * p.Nb + wp.b] += (p.B * p.dt) * sum;
    }
  }
}

// ---------------------------------------------------------------------------
// assembly of element-boundary nodes: f^s = A f^0 + B f^{s-1} + sum_c T_c / M + B dt F*,
// where T_c = B dt x (weighted contribution of copy c); copies summed in ascending (element, local node) order
// ---------------------------------------------------------------------------
template <typename Real, int LAT>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 2) dss_kernel(const KParams<Real> p) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  const Real Bdt = p.B * p.dt;
  const size_t EN = (size_t)p.E * p.Nb;
  const Real *__restrict__ Tr = p.T;
  const Real *__restrict__ fin = p.fin;
  const Real *__restrict__ f0 = p.f0;
  Real *__restrict__ fout = p.fout;
  const size_t G = p.Gs;                 // population stride
  const bool use_f0 = p.A != Real(0);
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < p.Gb; u += gridDim.x * blockDim.x) {
    const int c0 = p.bnode_off[u], c1 = p.bnode_off[u + 1];
    const size_t gid = p.bnode_g[u];
    const Real minv = p.bnode_minv[u];
    const Real rho = p.has_force ? p.rho[gid] : Real(0);
    Real ga[3] = {0, 0, 0};
    if (p.has_force) node_accel(p, gid, ga);
    // populations in two halves; two copies per iteration, their loads in flight together,
    // added in ascending copy order
    constexpr int QH = (Q + 1) / 2;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int a0 = hh * QH;
      Real s[QH];
#pragma unroll
      for (int a = 0; a < QH; ++a) s[a] = 0;
      int c = c0;
      for (; c + 1 < c1; c += 2) {
        const Real *t0 = Tr + p.bnode_slot[c] + (size_t)a0 * EN, *t1 = Tr + p.bnode_slot[c + 1] + (size_t)a0 * EN;
        Real v0[QH], v1[QH];
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) { v0[a] = t0[a * EN]; v1[a] = t1[a * EN]; }
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) { s[a] += v0[a]; s[a] += v1[a]; }
      }
      if (c < c1) {
        const Real *t0 = Tr + p.bnode_slot[c] + (size_t)a0 * EN;
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) s[a] += t0[a * EN];
      }
#pragma unroll
      for (int al = 0; al < QH; ++al) {
        const int a = a0 + al;
        if (a >= Q) break;
        Real Fs = 0;
        if (p.has_force) {
          Real eg = 0;
#pragma unroll
          for (int k = 0; k < DIM; ++k) eg += (Real)c_e[LAT][a][k] * ga[k];
          Fs = wt<Real>(LAT, a) * eg * rho * Real(3);
        }
        const Real base = use_f0 ? p.A * f0[(size_t)a * G + gid] : Real(0);   // stage 1: A = 0
        fout[(size_t)a * G + gid] = base + p.B * fin[(size_t)a * G + gid] + s[al] * minv + Bdt * Fs;
      }
    }
  }
}

// filtered copy (owners write) used to read the state back between steps
template <typename Real, int LAT>
__global__ void __launch_bounds__(512) finalize_kernel(const KParams<Real> p) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = p.n, Np = p.Np;
  Real *sf = reinterpret_cast<Real *>(smem_raw);
  Real *sF = sf + Q * Np + n * n;
  const int e = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < n * n; k += nt) sF[k] = p.Fm[k];
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  for (int idx = tid; idx < Q * Np; idx += nt) {
    const int a = idx / Np, i = idx - a * Np;
    sf[idx] = p.fin[(size_t)a * p.Gs + l2g[i]];
  }
  __syncthreads();
  if (p.apply_filter) {
    for (int axis = 0; axis < DIM; ++axis) {
      filter_pass<Real, Q>(sf, sF, n, Np, axis);
      __syncthreads();
    }
  }
  for (int idx = tid; idx < Q * Np; idx += nt) {
    const int a = idx / Np, i = idx - a * Np;
    if (p.owner[(size_t)e * Np + i]) p.fout[(size_t)a * p.Gs + l2g[i]] = sf[idx];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int block_for(int lat) { return lat == SELBM_D2Q9 ? 256 : 512; }

template <typename Real, int LAT, bool AFF>
static cudaError_t launch_stage_t(const KParams<Real> &p, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(LAT, p.Np, p.n, sizeof(Real));
  auto k = stage_kernel<Real, LAT, AFF>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<p.E, block_for(LAT), smem, s>>>(p);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_stage(int lat, bool affine, const KParams<Real> &p, cudaStream_t s) {
  switch (lat) {
    case SELBM_D2Q9: return affine ? launch_stage_t<Real, SELBM_D2Q9, true>(p, s) : launch_stage_t<Real, SELBM_D2Q9, false>(p, s);
    case SELBM_D3Q19: return affine ? launch_stage_t<Real, SELBM_D3Q19, true>(p, s) : launch_stage_t<Real, SELBM_D3Q19, false>(p, s);
    case SELBM_D3Q27: return affine ? launch_stage_t<Real, SELBM_D3Q27, true>(p, s) : launch_stage_t<Real, SELBM_D3Q27, false>(p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename Real, int LAT>
static cudaError_t launch_dss_t(const KParams<Real> &p, cudaStream_t s) {
  if (p.Gb == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)std::min<size_t>(((size_t)p.Gb + threads - 1) / threads, 152 * 32);
  dss_kernel<Real, LAT><<<blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_dss(int lat, const KParams<Real> &p, cudaStream_t s) {
  switch (lat) {
    case SELBM_D2Q9: return launch_dss_t<Real, SELBM_D2Q9>(p, s);
    case SELBM_D3Q19: return launch_dss_t<Real, SELBM_D3Q19>(p, s);
    case SELBM_D3Q27: return launch_dss_t<Real, SELBM_D3Q27>(p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename Real, int LAT>
static cudaError_t launch_finalize_t(const KParams<Real> &p, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(LAT, p.Np, p.n, sizeof(Real));
  auto k = finalize_kernel<Real, LAT>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<p.E, block_for(LAT), smem, s>>>(p);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_finalize(int lat, const KParams<Real> &p, cudaStream_t s) {
  switch (lat) {
    case SELBM_D2Q9: return launch_finalize_t<Real, SELBM_D2Q9>(p, s);
    case SELBM_D3Q19: return launch_finalize_t<Real, SELBM_D3Q19>(p, s);
    case SELBM_D3Q27: return launch_finalize_t<Real, SELBM_D3Q27>(p, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// state import / export and diagnostics
// ---------------------------------------------------------------------------

// f_bar = f^eq(rho, u) - dt/2 F** stored as g = f_bar - t rho0 (Sec. 2.1, f at equilibrium)
template <typename Real, int LAT>
__global__ void init_kernel(const double *rho, const double *u, const int32_t *first, int G, int Gs, double rho0,
                            double half_dt, double gx, double gy, double gz, int has_force, const Real *fS,
                            double amp, Real *out) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const size_t q = first[g];
    const double r = rho[q];
    double uv[3] = {0, 0, 0}, F[3] = {0, 0, 0}, gg[3] = {gx, gy, gz};
    if (fS)
      for (int k = 0; k < 3; ++k) gg[k] += amp * (double)fS[(size_t)k * G + g];
    double uu = 0, uF = 0;
    for (int k = 0; k < DIM; ++k) {
      uv[k] = u[q * DIM + k];
      uu += uv[k] * uv[k];
      F[k] = has_force ? r * gg[k] : 0.0;
      uF += uv[k] * F[k];
    }
    for (int a = 0; a < Q; ++a) {
      double eu = 0, eF = 0;
      for (int k = 0; k < DIM; ++k) { eu += c_e[LAT][a][k] * uv[k]; eF += c_e[LAT][a][k] * F[k]; }
      const double t = c_td[LAT][a];
      const double feq = t * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
      const double Fss = t * (9.0 * eu * eF - 3.0 * uF);
      out[(size_t)a * Gs + g] = (Real)(feq - half_dt * Fss - t * rho0);
    }
  }
}

template <typename Real, int LAT>
__global__ void set_state_kernel(const double *f, const int32_t *first, int G, int Gs, size_t nloc, double rho0, Real *out) {
  constexpr int Q = Lat<LAT>::Q;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    for (int a = 0; a < Q; ++a) out[(size_t)a * Gs + g] = (Real)(f[(size_t)a * nloc + first[g]] - c_td[LAT][a] * rho0);
}

template <typename Real, int LAT>
__global__ void get_state_kernel(const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *f) {
  constexpr int Q = Lat<LAT>::Q;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nloc; q += (size_t)gridDim.x * blockDim.x)
    for (int a = 0; a < Q; ++a) f[(size_t)a * nloc + q] = (double)buf[(size_t)a * Gs + l2g[q]] + c_td[LAT][a] * rho0;
}

// rho = sum f_bar, rho u = sum e f_bar at every local node (FP64 sums)
template <typename Real, int LAT>
__global__ void moments_kernel(const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *rho, double *u) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nloc; q += (size_t)gridDim.x * blockDim.x) {
    const size_t g = l2g[q];
    double d = 0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q; ++a) {
      const double v = (double)buf[(size_t)a * Gs + g];
      d += v;
      for (int k = 0; k < DIM; ++k) j[k] += c_e[LAT][a][k] * v;
    }
    const double r = rho0 + d;
    rho[q] = r;
    for (int k = 0; k < DIM; ++k) u[q * DIM + k] = j[k] / r;
  }
}

// non-equilibrium second moment at every local node, Pi_ij = factor sum_a e_ai e_aj (f_a - f_a^eq
// + dt/2 F**_a), factor = tau / (tau + 1/2); the buffer holds deviations f - t rho0; acceleration
// g + amp S_g (amp the field's time factor at the read-back time)
template <typename Real, int LAT>
__global__ void stress_kernel(const Real *buf, const int32_t *l2g, int G, int Gs, size_t nloc, double rho0, double half_dt,
                              double factor, double g0, double g1, double g2, int has_force, const Real *fS, double amp,
                              double *out) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nloc; q += (size_t)gridDim.x * blockDim.x) {
    const size_t g = l2g[q];
    double d = 0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q; ++a) {
      const double v = (double)buf[(size_t)a * Gs + g];
      d += v;
      for (int k = 0; k < DIM; ++k) j[k] += c_e[LAT][a][k] * v;
    }
    const double r = rho0 + d;
    double u[3] = {0, 0, 0}, F[3] = {0, 0, 0}, acc[3] = {g0, g1, g2}, uu = 0, uF = 0;
    if (fS)
      for (int k = 0; k < 3; ++k) acc[k] += amp * (double)fS[(size_t)k * G + g];
    for (int k = 0; k < DIM; ++k) {
      u[k] = j[k] / r;
      uu += u[k] * u[k];
      F[k] = has_force ? r * acc[k] : 0.0;
      uF += u[k] * F[k];
    }
    double pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < Q; ++a) {
      double eu = 0, eF = 0;
      for (int k = 0; k < DIM; ++k) { eu += c_e[LAT][a][k] * u[k]; eF += c_e[LAT][a][k] * F[k]; }
      const double t = c_td[LAT][a];
      // f - f^eq with f = buf + t rho0 and f^eq = t rho (1 + 3 eu + 4.5 eu^2 - 1.5 uu), rho = rho0 + d;
      // f_bar^eq = f^eq - dt/2 F** enters as + dt/2 F** without the 3 e.F term of F**: that
      // term's second moment sum_a t_a e_ai e_aj e_ak F_k vanishes, so it cannot change Pi
      const double neq = (double)buf[(size_t)a * Gs + g] - t * (d + r * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu)) +
                         half_dt * t * (9.0 * eu * eF - 3.0 * uF);
      for (int i = 0; i < DIM; ++i)
        for (int k = 0; k < DIM; ++k) pi[i][k] += (double)(c_e[LAT][a][i] * c_e[LAT][a][k]) * neq;
    }
    for (int i = 0; i < DIM; ++i)
      for (int k = 0; k < DIM; ++k) out[(q * DIM + i) * DIM + k] = factor * pi[i][k];
  }
}

// per-block partial sums: mass, momentum[3], KE, non-finite count (deterministic two-pass)
template <typename Real, int LAT>
__global__ void diag_partial_kernel(const Real *buf, const double *mass, int G, int Gs, double rho0, double *partial) {
  constexpr int Q = Lat<LAT>::Q, DIM = Lat<LAT>::D;
  __shared__ double red[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    double d = 0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q; ++a) {
      const double v = (double)buf[(size_t)a * Gs + g];
      if (!isfinite(v)) acc[5] += 1.0;
      d += v;
      for (int k = 0; k < DIM; ++k) j[k] += c_e[LAT][a][k] * v;
    }
    const double r = rho0 + d, M = mass[g];
    acc[0] += M * r;
    double uu = 0;
    for (int k = 0; k < DIM; ++k) { acc[1 + k] += M * j[k]; uu += (j[k] / r) * (j[k] / r); }
    acc[4] += 0.5 * rho0 * M * uu;
  }
  for (int c = 0; c < 6; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < 6; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; ++c) partial[blockIdx.x * 6 + c] = red[c][0];
}

// viscous dissipation integral of the velocity u [E][Np][dim] (local nodes):
// eps = 2 mu sum_i (d_i u_i)^2 - (2/3) mu (div u)^2 + mu sum_{i<j} (d_i u_j + d_j u_i)^2,
// gradients by D_hat along each reference axis and the chain rule; one CTA per element,
// per-element sums into partial[e] (summed in element order afterwards)
template <typename Real>
__global__ void eps_kernel(const double *u, int dim, int n, int Np, int affine, const Real *el_drdx, const Real *drdx,
                           const Real *el_J, const Real *wJ, const Real *gllw, const Real *Dm, double mu,
                           double *partial) {
  __shared__ double red[256];
  const int e = blockIdx.x, tid = threadIdx.x;
  double acc = 0.0;
  for (int i = tid; i < Np; i += blockDim.x) {
    const int ii[3] = {i % n, (i / n) % n, dim == 3 ? i / (n * n) : 0};
    const int st[3] = {1, n, n * n};
    double dr[3][3];   // dr[l][c] = d u_c / d r_l
    for (int l = 0; l < dim; ++l)
      for (int c = 0; c < dim; ++c) {
        double s = 0.0;
        const int base = i - ii[l] * st[l];
        for (int k = 0; k < n; ++k) s += (double)Dm[ii[l] * n + k] * u[((size_t)e * Np + base + k * st[l]) * dim + c];
        dr[l][c] = s;
      }
    double g[3][3];    // g[k][c] = d u_c / d x_k = sum_l dr_l/dx_k d u_c/d r_l
    for (int k = 0; k < dim; ++k)
      for (int c = 0; c < dim; ++c) {
        double s = 0.0;
        for (int l = 0; l < dim; ++l) {
          const double m = affine ? (double)el_drdx[((size_t)e * dim + l) * dim + k]
                                  : (double)drdx[(((size_t)e * Np + i) * dim + l) * dim + k];
          s += m * dr[l][c];
        }
        g[k][c] = s;
      }
    double div = 0.0, diag = 0.0, off = 0.0;
    for (int k = 0; k < dim; ++k) { div += g[k][k]; diag += g[k][k] * g[k][k]; }
    for (int a = 0; a < dim; ++a)
      for (int b = a + 1; b < dim; ++b) off += (g[a][b] + g[b][a]) * (g[a][b] + g[b][a]);
    const double dens = 2.0 * mu * diag - (2.0 / 3.0) * mu * div * div + mu * off;
    double w;
    if (affine) {
      w = (double)el_J[e] * (double)gllw[ii[0]] * (double)gllw[ii[1]] * (dim == 3 ? (double)gllw[ii[2]] : 1.0);
    } else {
      w = (double)wJ[(size_t)e * Np + i];
    }
    acc += w * dens;
  }
  red[tid] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) partial[e] = red[0];
}

__global__ void sum_kernel(const double *partial, int count, double *out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) acc += partial[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <typename Real>
cudaError_t launch_eps(const double *u, int dim, int n, int Np, int E, int affine, const Real *el_drdx, const Real *drdx,
                       const Real *el_J, const Real *wJ, const Real *gllw, const Real *Dm, double mu, double *partial,
                       double *out, cudaStream_t s) {
  eps_kernel<Real><<<E, 256, 0, s>>>(u, dim, n, Np, affine, el_drdx, drdx, el_J, wJ, gllw, Dm, mu, partial);
  sum_kernel<<<1, 256, 0, s>>>(partial, E, out);
  return cudaGetLastError();
}
template cudaError_t launch_eps<double>(const double *, int, int, int, int, int, const double *, const double *,
                                        const double *, const double *, const double *, const double *, double,
                                        double *, double *, cudaStream_t);
template cudaError_t launch_eps<float>(const double *, int, int, int, int, int, const float *, const float *,
                                       const float *, const float *, const float *, const float *, double, double *,
                                       double *, cudaStream_t);

__global__ void diag_final_kernel(const double *partial, int nblocks, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int c = 0; c < 6; ++c) acc[c] += partial[b * 6 + c];
    for (int c = 0; c < 6; ++c) out[c] = acc[c];
  }
}

static int grid_for(size_t n, int threads) { return (int)std::min<size_t>((n + threads - 1) / threads, 152 * 16); }

#define SELBM_LAT_SWITCH(lat, CALL)                  \
  switch (lat) {                                     \
    case SELBM_D2Q9: { constexpr int L = SELBM_D2Q9; CALL; } break;  \
    case SELBM_D3Q19: { constexpr int L = SELBM_D3Q19; CALL; } break; \
    case SELBM_D3Q27: { constexpr int L = SELBM_D3Q27; CALL; } break; \
    default: return cudaErrorInvalidValue;           \
  }

template <typename Real>
cudaError_t launch_init(int lat, const double *rho, const double *u, const int32_t *first, int G, int Gs, double rho0,
                        double half_dt, const double g[3], int has_force, const Real *fS, double amp, Real *out,
                        cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (init_kernel<Real, L><<<grid_for(G, 256), 256, 0, s>>>(rho, u, first, G, Gs, rho0, half_dt, g[0], g[1], g[2], has_force, fS, amp, out)));
  return cudaGetLastError();
}

template <typename Real>
__global__ void combine_kernel(size_t n, const Real *f0, const Real *f1, const Real *f2, const Real *f3, int m,
                               Real c0, Real c1, Real c2, Real c3, const Real *base, Real cb, Real *g, Real *b) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    Real v = c0 * f0[i];
    if (m > 1) v += c1 * f1[i];
    if (m > 2) v += c2 * f2[i];
    if (m > 3) v += c3 * f3[i];
    g[i] = v;
    b[i] = base[i] - cb * v;
  }
}
template <typename Real>
cudaError_t launch_combine(size_t n, const Real *f0, const Real *f1, const Real *f2, const Real *f3, int m,
                           const double c[4], const Real *base, double cb, Real *g, Real *b, cudaStream_t s) {
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  combine_kernel<Real><<<blocks, 256, 0, s>>>(n, f0, f1, f2, f3, m, (Real)c[0], (Real)c[1], (Real)c[2], (Real)c[3],
                                              base, (Real)cb, g, b);
  return cudaGetLastError();
}

// per-node acceleration field on unique nodes from the first local copy of each node
template <typename Real>
__global__ void force_field_kernel(const double *S, const int32_t *first, int G, int dim, Real *fS) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const size_t q = first[g];
    for (int k = 0; k < 3; ++k) fS[(size_t)k * G + g] = k < dim ? (Real)S[q * dim + k] : Real(0);
  }
}
template <typename Real>
cudaError_t launch_force_field(const double *S, const int32_t *first, int G, int dim, Real *fS, cudaStream_t s) {
  force_field_kernel<Real><<<grid_for(G, 256), 256, 0, s>>>(S, first, G, dim, fS);
  return cudaGetLastError();
}

// A(t) = sin(2 pi t / period) while t < t_end (1 for period <= 0), 0 after; t = ft[0] is the
// time at the start of the step, advanced by dt here so that graph replays keep the clock
template <typename Real>
__global__ void force_amp_kernel(double *ft, Real *amp, double dt, double period, double t_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double t = ft[0];
  double A = 0.0;
  if (t < t_end) A = period > 0.0 ? sin(2.0 * 3.14159265358979323846 * t / period) : 1.0;
  *amp = (Real)A;
  ft[0] = t + dt;
}
template <typename Real>
cudaError_t launch_force_amp(double *ft, Real *amp, double dt, double period, double t_end, cudaStream_t s) {
  force_amp_kernel<Real><<<1, 32, 0, s>>>(ft, amp, dt, period, t_end);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_set_state(int lat, const double *f, const int32_t *first, int G, int Gs, size_t nloc, double rho0, Real *out, cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (set_state_kernel<Real, L><<<grid_for(G, 256), 256, 0, s>>>(f, first, G, Gs, nloc, rho0, out)));
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_get_state(int lat, const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *f, cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (get_state_kernel<Real, L><<<grid_for(nloc, 256), 256, 0, s>>>(buf, l2g, Gs, nloc, rho0, f)));
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_moments(int lat, const Real *buf, const int32_t *l2g, int Gs, size_t nloc, double rho0, double *rho, double *u, cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (moments_kernel<Real, L><<<grid_for(nloc, 256), 256, 0, s>>>(buf, l2g, Gs, nloc, rho0, rho, u)));
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_stress(int lat, const Real *buf, const int32_t *l2g, int G, int Gs, size_t nloc, double rho0, double half_dt,
                          double factor, const double g[3], int has_force, const Real *fS, double amp, double *out,
                          cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (stress_kernel<Real, L><<<grid_for(nloc, 256), 256, 0, s>>>(
                             buf, l2g, G, Gs, nloc, rho0, half_dt, factor, g[0], g[1], g[2], has_force, fS, amp, out)));
  return cudaGetLastError();
}
int diag_blocks() { return 152 * 4; }
template <typename Real>
cudaError_t launch_diag(int lat, const Real *buf, const double *mass, int G, int Gs, double rho0, double *partial, double *out, cudaStream_t s) {
  SELBM_LAT_SWITCH(lat, (diag_partial_kernel<Real, L><<<diag_blocks(), 256, 0, s>>>(buf, mass, G, Gs, rho0, partial)));
  diag_final_kernel<<<1, 32, 0, s>>>(partial, diag_blocks(), out);
  return cudaGetLastError();
}

#define SELBM_INST_UTIL(Real)                                                                                              \
  template cudaError_t launch_init<Real>(int, const double *, const double *, const int32_t *, int, int, double, double,      \
                                         const double[3], int, const Real *, double, Real *, cudaStream_t);              \
  template cudaError_t launch_force_field<Real>(const double *, const int32_t *, int, int, Real *, cudaStream_t);         \
  template cudaError_t launch_combine<Real>(size_t, const Real *, const Real *, const Real *, const Real *, int,         \
                                            const double[4], const Real *, double, Real *, Real *, cudaStream_t);        \
  template cudaError_t launch_force_amp<Real>(double *, Real *, double, double, double, cudaStream_t);                    \
  template cudaError_t launch_stress<Real>(int, const Real *, const int32_t *, int, int, size_t, double, double, double,        \
                                           const double[3], int, const Real *, double, double *, cudaStream_t);          \
  template cudaError_t launch_set_state<Real>(int, const double *, const int32_t *, int, int, size_t, double, Real *, cudaStream_t); \
  template cudaError_t launch_get_state<Real>(int, const Real *, const int32_t *, int, size_t, double, double *, cudaStream_t); \
  template cudaError_t launch_moments<Real>(int, const Real *, const int32_t *, int, size_t, double, double *, double *, cudaStream_t); \
  template cudaError_t launch_diag<Real>(int, const Real *, const double *, int, int, double, double *, double *, cudaStream_t);
SELBM_INST_UTIL(double)
SELBM_INST_UTIL(float)

template cudaError_t launch_stage<double>(int, bool, const KParams<double> &, cudaStream_t);
template cudaError_t launch_stage<float>(int, bool, const KParams<float> &, cudaStream_t);
template cudaError_t launch_dss<double>(int, const KParams<double> &, cudaStream_t);
template cudaError_t launch_dss<float>(int, const KParams<float> &, cudaStream_t);
template cudaError_t launch_finalize<double>(int, const KParams<double> &, cudaStream_t);
template cudaError_t launch_finalize<float>(int, const KParams<float> &, cudaStream_t);

}  // namespace slb
