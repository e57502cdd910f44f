// Population-split step for hexahedral meshes (compile-time order N and lattice).
//
// Once the collision is done, the three Runge-Kutta stages only advect, and every
// population advects independently of the others.  The step therefore runs as
//   prologue_kernel   one CTA per element: the pending filter of the previous step
//                     (fixed, or chosen per element by the learned control) and the
//                     BGK collision; writes f^0 on unique nodes
//   stage_split_kernel  per stage, one CTA per (element, group of PB populations):
//                     gather the group's tile, -B dt e.grad f by sum factorisation,
//                     stage combination, element-interior nodes to f^s and weighted
//                     boundary shares to the assembly trace (+ flux bounce-back)
//   dss_kernel        assembly of shared nodes (unchanged)
// The split CTAs are small (PB (N+1)^3 values), a single round of (population,
// r-line) tasks covers them, and several CTAs per SM overlap their gathers with
// each other's arithmetic.
//
// With the learned control, three kernels choose each element's transfer function first
// (node_features_kernel: rho - rho0, |u| and the drift integrals on unique nodes;
// element_features_kernel: modal shell energies, one warp per element; mlp_sigma_kernel: the
// network over 16 elements per CTA).  Copies of a shared node are then filtered by different
// element filters: the prologue writes their weighted shares wJ f to the trace and
// dss_collide_kernel forms the mass-weighted average and collides it.
#pragma once
#include <cuda_bf16.h>

#include <algorithm>

#include "selbm_collide.cuh"
#include "selbm_fast.cuh"
#include "selbm_split_stage.cuh"

namespace slb {

// ---------------------------------------------------------------------------
// prologue: pending filter + collision, one CTA per element with all Q populations
// ---------------------------------------------------------------------------
// learned control inputs of the prologue (network: 2n -> 64 tanh -> 64 tanh -> 2)
template <typename Real, int n>
struct LearnedIn {
  Real Vm[n * n];               // modal -> nodal
  Real Vinv[n * n];             // nodal -> modal
  Real fixed_sigma[n];          // transfer function of the fixed filter (fallback)
  const __nv_bfloat16 *W;       // parameters; NULL = features only
  const Real *lo, *hi;          // [2n] training range of the features
  const int *flag;              // sticky drift fallback flag or NULL
  double *acc;                  // drift accumulators (mass, KE) or NULL
  Real *sigma_out;              // [E][n] or NULL
  float *feat_out;              // [E][2n] or NULL
  int *n_fallback;              // counter of elements that kept the fixed filter, or NULL
  int outputs;                  // 0: features / transfer functions only
};

constexpr int kProThreads = 256;
constexpr int kHidden = 64;

template <typename Real, int LAT, int n, bool AFFINE, int MODE>
constexpr size_t prologue_smem_bytes() {
  using TI = Tile<Real, n, 3>;
  constexpr int Q = LT<LAT>::v.Q;
  size_t reals = (size_t)Q * TI::PS + 2 * n * n;                   // tile; U, W or F_e, V^-1
  if (MODE == PRO_LEARNED) reals += 2 * n * n + n;                  // V, W (or F_e^T), sigma_e
  return reals * sizeof(Real);
}

// y <- (A x A x A) y on NP populations of a tile, one 1D pass per axis; op maps the n
// values of one line in place.  PAIRS: on the swizzled FP32 tile, the s- and t-passes take
// two adjacent columns per task with 8-byte accesses (for light ops; heavy ops spill)
template <typename Real, int n, int NP, int T, bool PAIRS = false, typename Op>
__device__ __forceinline__ void tile_pass3(Real *sf, int tid, Op op) {
  using TI = Tile<Real, n, 3>;
  constexpr int NL = n * n, PS = TI::PS;
  for (int t = tid; t < NP * NL; t += T) {          // r-lines
    const int a = t / NL, L = t - a * NL;
    const int i1 = L % n, i2 = L / n;
    Real v[n];
    Real *base = sf + a * PS + TI::line(i1, i2);
    load_line<Real, n>(base, TI::sw(i1), v);
    op(v);
    store_line<Real, n>(base, TI::sw(i1), v);
  }
  __syncthreads();
  if constexpr (TI::SW && PAIRS) {
    // swizzled FP32 tile: two adjacent columns per task (i0 = 2q, 2q + 1 sit in one aligned
    // 8-byte pair of every line), one vector access per line
    auto pair_pass = [&](auto addr) {
      for (int t = tid; t < NP * NL / 2; t += T) {
        const int a = t / (NL / 2), r = t - a * (NL / 2), q = r & 3, w = r >> 2;
        float2 v2[n];
#pragma unroll
        for (int k = 0; k < n; ++k) v2[k] = *reinterpret_cast<const float2 *>(sf + a * PS + addr(w, k, q));
        {
          Real v[n];
#pragma unroll
          for (int k = 0; k < n; ++k) v[k] = v2[k].x;
          op(v);
#pragma unroll
          for (int k = 0; k < n; ++k) v2[k].x = v[k];
        }
        {
          Real v[n];
#pragma unroll
          for (int k = 0; k < n; ++k) v[k] = v2[k].y;
          op(v);
#pragma unroll
          for (int k = 0; k < n; ++k) v2[k].y = v[k];
        }
#pragma unroll
        for (int k = 0; k < n; ++k) *reinterpret_cast<float2 *>(sf + a * PS + addr(w, k, q)) = v2[k];
      }
    };
    // s-lines (i0 pair, k, i2 = w) and t-lines (i0 pair, i1 = w, k)
    pair_pass([](int w, int k, int q) { return TI::line(k, w) + ((2 * q) ^ TI::sw(k)); });
    __syncthreads();
    pair_pass([](int w, int k, int q) { return TI::line(w, k) + ((2 * q) ^ TI::sw(w)); });
    __syncthreads();
  } else {
    for (int t = tid; t < NP * NL; t += T) {          // s-lines
      const int a = t / NL, r = t - a * NL, i0 = r % n, i2 = r / n;
      Real v[n];
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = sf[a * PS + TI::at(i0, k, i2)];
      op(v);
#pragma unroll
      for (int k = 0; k < n; ++k) sf[a * PS + TI::at(i0, k, i2)] = v[k];
    }
    __syncthreads();
    for (int t = tid; t < NP * NL; t += T) {          // t-lines
      const int a = t / NL, r = t - a * NL, i0 = r % n, i1 = r / n;
      Real v[n];
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = sf[a * PS + TI::at(i0, i1, k)];
      op(v);
#pragma unroll
      for (int k = 0; k < n; ++k) sf[a * PS + TI::at(i0, i1, k)] = v[k];
    }
    __syncthreads();
  }
}

// v <- v + U (W v) with U^T and W stored by rows in shared memory (row stride n), the
// rows read as vectors
template <typename Real, int n>
__device__ __forceinline__ void filter_rows(Real (&v)[n], const Real *UT, const Real *W, int r) {
  Real o[n];
#pragma unroll
  for (int j = 0; j < n; ++j) o[j] = v[j];
  for (int q = 0; q < r; ++q) {
    Real row[n];
    load_line<Real, n>(W + q * n, 0, row);
    Real s = 0;
#pragma unroll
    for (int k = 0; k < n; ++k) s += row[k] * v[k];
    load_line<Real, n>(UT + q * n, 0, row);
#pragma unroll
    for (int j = 0; j < n; ++j) o[j] += row[j] * s;
  }
#pragma unroll
  for (int j = 0; j < n; ++j) v[j] = o[j];
}

// y <- ((I + U W) x (I + U W) x (I + U W)) y on NP populations of a tile, U^T and W (r rows of
// n) in shared memory.  On the swizzled FP32 tile the s- and t-passes take two adjacent columns
// per task and share each row of U^T and W between them (packed FMAs).
template <typename Real, int n, int NP, int T>
__device__ __forceinline__ void tile_lowrank3(Real *sf, int tid, const Real *UT, const Real *W, int r) {
  using TI = Tile<Real, n, 3>;
  if constexpr (!TI::SW) {
    tile_pass3<Real, n, NP, T>(sf, tid, [&](Real (&v)[n]) { filter_rows<Real, n>(v, UT, W, r); });
  } else {
    constexpr int NL = n * n, PS = TI::PS;
    for (int t = tid; t < NP * NL; t += T) {          // r-lines
      const int a = t / NL, L = t - a * NL;
      const int i1 = L % n, i2 = L / n;
      Real v[n];
      Real *base = sf + a * PS + TI::line(i1, i2);
      load_line<Real, n>(base, TI::sw(i1), v);
      filter_rows<Real, n>(v, UT, W, r);
      store_line<Real, n>(base, TI::sw(i1), v);
    }
    __syncthreads();
    auto pair_pass = [&](auto addr) {
      for (int t = tid; t < NP * NL / 2; t += T) {
        const int a = t / (NL / 2), rr = t - a * (NL / 2), q = rr & 3, w = rr >> 2;
        Real *base = sf + a * PS;
        float2 v2[n], o2[n];
#pragma unroll
        for (int k = 0; k < n; ++k) {
          v2[k] = *reinterpret_cast<const float2 *>(base + addr(w, k, q));
          o2[k] = v2[k];
        }
        for (int m = 0; m < r; ++m) {
          Real row[n];
          load_line<Real, n>(W + m * n, 0, row);
          float2 s2 = __fmul2_rn(make_float2(row[0], row[0]), v2[0]);
#pragma unroll
          for (int k = 1; k < n; ++k) s2 = __ffma2_rn(make_float2(row[k], row[k]), v2[k], s2);
          load_line<Real, n>(UT + m * n, 0, row);
#pragma unroll
          for (int j = 0; j < n; ++j) o2[j] = __ffma2_rn(make_float2(row[j], row[j]), s2, o2[j]);
        }
#pragma unroll
        for (int j = 0; j < n; ++j) *reinterpret_cast<float2 *>(base + addr(w, j, q)) = o2[j];
      }
    };
    pair_pass([](int w, int k, int q) { return TI::line(k, w) + ((2 * q) ^ TI::sw(k)); });
    __syncthreads();
    pair_pass([](int w, int k, int q) { return TI::line(w, k) + ((2 * q) ^ TI::sw(w)); });
    __syncthreads();
  }
}

template <typename Real, int n>
__device__ __forceinline__ void dense_vals(Real (&v)[n], const Real *M) {
  Real o[n];
#pragma unroll
  for (int j = 0; j < n; ++j) {
    Real s = 0;
#pragma unroll
    for (int k = 0; k < n; ++k) s += M[j * n + k] * v[k];
    o[j] = s;
  }
#pragma unroll
  for (int j = 0; j < n; ++j) v[j] = o[j];
}

// y <- (M x M x M) y on NP populations of a tile, M (row-major) and its transpose MT in
// shared memory.  On the swizzled FP32 tile the s- and t-passes take two adjacent columns
// per task (8-byte accesses) and accumulate the columns of M with packed FMAs.
template <typename Real, int n, int NP, int T>
__device__ __forceinline__ void tile_dense3(Real *sf, int tid, const Real *M, const Real *MT) {
  using TI = Tile<Real, n, 3>;
  if constexpr (!TI::SW) {
    tile_pass3<Real, n, NP, T>(sf, tid, [&](Real (&v)[n]) { dense_vals<Real, n>(v, M); });
  } else {
    constexpr int NL = n * n, PS = TI::PS;
    for (int t = tid; t < NP * NL; t += T) {          // r-lines
      const int a = t / NL, L = t - a * NL;
      const int i1 = L % n, i2 = L / n;
      Real v[n];
      Real *base = sf + a * PS + TI::line(i1, i2);
      load_line<Real, n>(base, TI::sw(i1), v);
      dense_vals<Real, n>(v, M);
      store_line<Real, n>(base, TI::sw(i1), v);
    }
    __syncthreads();
    auto pair_pass = [&](auto addr) {
      for (int t = tid; t < NP * NL / 2; t += T) {
        const int a = t / (NL / 2), r = t - a * (NL / 2), q = r & 3, w = r >> 2;
        Real *base = sf + a * PS;
        float2 d[n];
#pragma unroll
        for (int j = 0; j < n; ++j) d[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const float2 vk = *reinterpret_cast<const float2 *>(base + addr(w, k, q));
          Real col[n];
          load_line<Real, n>(MT + k * n, 0, col);
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = __ffma2_rn(make_float2(col[j], col[j]), vk, d[j]);
        }
#pragma unroll
        for (int j = 0; j < n; ++j) *reinterpret_cast<float2 *>(base + addr(w, j, q)) = d[j];
      }
    };
    // s-lines (i0 pair, k, i2 = w) and t-lines (i0 pair, i1 = w, k)
    pair_pass([](int w, int k, int q) { return TI::line(k, w) + ((2 * q) ^ TI::sw(k)); });
    __syncthreads();
    pair_pass([](int w, int k, int q) { return TI::line(w, k) + ((2 * q) ^ TI::sw(w)); });
    __syncthreads();
  }
}

template <typename Real, int LAT, int n, bool AFFINE, int MODE>
__global__ void __launch_bounds__(kProThreads, sizeof(Real) == 4 ? 4 : 2)
prologue_kernel(const KParams<Real> p, const FastMats<Real, n> m, const LearnedIn<Real, n> c) {
  constexpr int Q = LT<LAT>::v.Q, DIM = 3, Np = n * n * n, T = kProThreads;
  using TI = Tile<Real, n, DIM>;
  constexpr int PS = TI::PS;
  constexpr bool LEARNED = MODE == PRO_LEARNED;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sf = reinterpret_cast<Real *>(smem_raw);   // [Q][PS]
  Real *sM0 = sf + Q * PS;                          // learned: [n][n] F_e or U_e^T
  Real *sM1 = sM0 + n * n;                          // learned: [n][n] V^-1
  Real *sVm = sM1 + n * n;                          // learned: [n][n]
  Real *sW = sVm + n * n;                           // learned: [n][n] W or F_e^T
  Real *ssig = sW + n * n;                          // learned: [n] sigma_e of this element
  __shared__ int s_r, s_mode[n];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t G = p.Gs;                            // population stride of the state
  auto weight = [&](int i) -> Real {
    if (AFFINE) {
      const int i0 = i % n, i1 = (i / n) % n, i2 = i / (n * n);
      return p.el_J[e] * p.gllw[i0] * p.gllw[i1] * p.gllw[i2];
    }
    return p.wJ[(size_t)e * Np + i];
  };
  if (LEARNED) {
    // the element's transfer function, chosen by the control kernels (mlp_sigma_kernel)
    for (int k = tid; k < n * n; k += T) { sM1[k] = c.Vinv[k]; sVm[k] = c.Vm[k]; }
    if (tid < n) ssig[tid] = c.sigma_out[(size_t)e * n + tid];
  }
  // ---- gather with asynchronous copies (all Q populations of the thread's nodes in
  //      flight at once)
  {
    const unsigned s_f = (unsigned)__cvta_generic_to_shared(sf);
    for (int i = tid; i < Np; i += T) {
      const Real *src = p.fin + l2g[i];
      const unsigned d = s_f + (unsigned)TI::node(i) * (unsigned)sizeof(Real);
#pragma unroll
      for (int a = 0; a < Q; ++a) cp_async_s<Real>(d + a * PS * (unsigned)sizeof(Real), src + a * G);
    }
    cp_async_wait_all();
  }
  __syncthreads();

  if (LEARNED) {
    // F_e = V diag(sigma) V^-1 with exact identity end rows, = I + U W with U = V[:, d]
    // diag(sigma_d - 1) (end rows zero) and W = V^-1[d, :] over the damped modes d: the
    // low-rank form when it is cheaper (2 r n < n^2 multiply-adds per line)
    if (tid == 0) {
      int r = 0;
      for (int k = 0; k < n; ++k)
        if (ssig[k] != Real(1)) s_mode[r++] = k;
      s_r = r;
    }
    __syncthreads();
    const int r = s_r;
    if (2 * r < n) {
      for (int idx = tid; idx < n * r; idx += T) {       // U^T [q][j]
        const int q = idx / n, j = idx - q * n, k = s_mode[q];
        sM0[q * n + j] = (j == 0 || j == n - 1) ? Real(0) : sVm[j * n + k] * (ssig[k] - Real(1));
      }
      for (int idx = tid; idx < r * n; idx += T) {       // W [q][k]
        const int q = idx / n, jj = idx - q * n;
        sW[q * n + jj] = sM1[s_mode[q] * n + jj];
      }
      __syncthreads();
      tile_lowrank3<Real, n, Q, T>(sf, tid, sM0, sW, r);
    } else {
      for (int k = tid; k < n * n; k += T) {
        const int rr = k / n, jj = k - rr * n;
        Real s = 0;
#pragma unroll
        for (int q = 0; q < n; ++q) s += sVm[rr * n + q] * ssig[q] * sM1[q * n + jj];
        if (rr == 0 || rr == n - 1) s = (rr == jj) ? Real(1) : Real(0);
        sM0[k] = s;
        sW[jj * n + rr] = s;                            // F_e^T
      }
      __syncthreads();
      tile_dense3<Real, n, Q, T>(sf, tid, sM0, sW);
    }
  } else if (MODE == PRO_FIXED) {
    // U and W are the same for every element: read them as kernel-parameter constants
    const int r = m.r;
    tile_pass3<Real, n, Q, T, true>(sf, tid, [&](Real (&v)[n]) { filter_vals<Real, n>(v, m.U, m.W, r); });
  }

  // ---- collision at every node this element writes: owned copies (one filter for
  //      all elements, so copies agree), or element-interior nodes with the learned
  //      control, whose element-boundary copies go to the trace as wJ f for the
  //      mass-weighted assembly of shared nodes
  const size_t EN = (size_t)p.E * p.Nb;
  for (int i = tid; i < Np; i += T) {
    const int ti = TI::node(i);
    const size_t g = l2g[i];
    if (LEARNED) {
      const int b = p.bslot[i];
      if (b >= 0) {
        const Real wq = weight(i);
        Real *tp = p.T + (size_t)e * p.Nb + b;
#pragma unroll
        for (int a = 0; a < Q; ++a) tp[a * EN] = wq * sf[a * PS + ti];
        continue;
      }
    } else if (!p.owner[(size_t)e * Np + i]) {
      continue;
    }
    Real fr[Q], gacc[3];
#pragma unroll
    for (int a = 0; a < Q; ++a) fr[a] = sf[a * PS + ti];
    node_accel(p, g, gacc);
    const Real rho = bgk_collide<Real, LAT>(fr, p.rho0, p.omega, p.dt, p.half_dt, gacc, p.has_force != 0);
#pragma unroll
    for (int a = 0; a < Q; ++a) p.f0out[(size_t)a * G + g] = fr[a];
    if (p.has_force) p.rho[g] = rho;
  }
}

// ---------------------------------------------------------------------------
// learned control, split form: node features, then the per-element network
// ---------------------------------------------------------------------------
// rho - rho0 and |u| at every unique node of the state the pending filter acts on, q [2][Gs],
// and its drift integrals sum M_g rho_g and sum M_g rho0 |u_g|^2 / 2 (added to acc[0], acc[1])
template <typename Real, int LAT>
__global__ void __launch_bounds__(256) node_features_kernel(const KParams<Real> p, Real *q, const double *mass,
                                                            double *acc) {
  constexpr VelTab V = LT<LAT>::v;
  constexpr int Q = V.Q, DIM = V.D;
  __shared__ double red[8][2];
  const size_t Gs = p.Gs;
  double pm = 0.0, pk = 0.0;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (size_t)p.G; g += (size_t)gridDim.x * blockDim.x) {
    Real drho = 0, j[3] = {0, 0, 0};
    static_for<0, Q>([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      const Real v = p.fin[(size_t)a * Gs + g];
      drho += v;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        if (V.e[a][k] > 0) j[k] += v;
        else if (V.e[a][k] < 0) j[k] -= v;
      }
    });
    const Real rho = p.rho0 + drho;
    Real uu = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) uu += (j[k] / rho) * (j[k] / rho);
    q[g] = drho;
    q[Gs + g] = sqrt(uu);
    if (acc) {
      pm += mass[g] * (double)rho;
      pk += 0.5 * (double)p.rho0 * mass[g] * (double)uu;
    }
  }
  if (!acc) return;
  pm = warp_sum(pm);
  pk = warp_sum(pk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[wid][0] = pm; red[wid][1] = pk; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sm = 0.0, sk = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sm += red[w][0]; sk += red[w][1]; }
    atomicAdd(&acc[0], sm);
    atomicAdd(&acc[1], sk);
  }
}

// One warp per element (kCtlWarps elements per CTA): the fields at its local nodes, modal
// coefficients (V^-1 along every axis), shell energies E_k (largest modal index k) and the
// features x = log10(E_k + 1e-30) of rho - rho0 and |u| -> X [E][2n]
constexpr int kCtlWarps = 4;
template <typename Real, int n>
__global__ void __launch_bounds__(32 * kCtlWarps, sizeof(Real) == 4 ? 4 : 2)
element_features_kernel(const KParams<Real> p, const LearnedIn<Real, n> c, const Real *q, Real *X) {
  constexpr int Np = n * n * n, NL = n * n, nin = 2 * n, WPB = kCtlWarps;
  static_assert(nin <= 32, "one lane per feature");
  __shared__ __align__(16) Real sq[WPB][2][Np];
  __shared__ Real sVi[n * n];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) sVi[k] = c.Vinv[k];
  __syncthreads();                                   // the only block-wide barrier
  const int e = blockIdx.x * WPB + wid;
  if (e >= p.E) return;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t Gs = p.Gs;
  Real *f0 = sq[wid][0], *f1 = sq[wid][1];
  {
    // all of the lane's index and field loads in flight together (one dependent round trip)
    constexpr int NPL = (Np + 31) / 32, HALF = (NPL + 1) / 2;
#pragma unroll
    for (int r0 = 0; r0 < NPL; r0 += HALF) {
      int32_t gi[HALF];
#pragma unroll
      for (int r = 0; r < HALF; ++r) {
        const int i = lane + 32 * (r0 + r);
        gi[r] = (r0 + r < NPL && i < Np) ? l2g[i] : 0;
      }
#pragma unroll
      for (int r = 0; r < HALF; ++r) {
        const int i = lane + 32 * (r0 + r);
        if (r0 + r < NPL && i < Np) {
          f0[i] = q[gi[r]];
          f1[i] = q[Gs + gi[r]];
        }
      }
    }
  }
  __syncwarp();
  // modal coefficients of both fields: V^-1 along r, s and t (node order r fastest)
#pragma unroll 1
  for (int axis = 0; axis < 3; ++axis) {
    const int stride = axis == 0 ? 1 : (axis == 1 ? n : NL);
#pragma unroll 1
    for (int t = lane; t < 2 * NL; t += 32) {
      const int f = t / NL, L = t - f * NL;
      const int base = axis == 0 ? L * n : (axis == 1 ? (L % n) + NL * (L / n) : L);
      Real *row = sq[wid][f] + base;
      Real v[n];
#pragma unroll
      for (int k = 0; k < n; ++k) v[k] = row[k * stride];
      dense_vals<Real, n>(v, sVi);
#pragma unroll
      for (int k = 0; k < n; ++k) row[k * stride] = v[k];
    }
    __syncwarp();
  }
  // shell energies E_k = sum over max(k0, k1, k2) = k of the squared coefficients
  Real en[2][n];
#pragma unroll
  for (int k = 0; k < n; ++k) { en[0][k] = 0; en[1][k] = 0; }
  for (int i = lane; i < Np; i += 32) {
    const int i0 = i % n, i1 = (i / n) % n, i2 = i / NL;
    const int sh = max(i0, max(i1, i2));
    const Real q0 = f0[i], q1 = f1[i];
#pragma unroll
    for (int k = 0; k < n; ++k)
      if (k == sh) { en[0][k] += q0 * q0; en[1][k] += q1 * q1; }
  }
  Real mine = 0;                                      // lane k < nin: energy k
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const Real sum = warp_sum(en[f][k]);
      if (lane == f * n + k) mine = sum;
    }
  if (lane < nin) {
    const Real x = log10(mine + Real(1e-30));
    X[(size_t)e * nin + lane] = x;
    if (c.feat_out) c.feat_out[(size_t)e * nin + lane] = (float)x;
  }
}

// The network over kMlpEB elements per CTA (weights staged once in shared memory, every thread
// computing independent outputs): scaled inputs s = 2 (x - lo)/(hi - lo) - 1, h1 = tanh(W1 s + b1),
// h2 = tanh(W2 h1 + b2), o = W3 h2 + b3 (BF16 weights, Real arithmetic), then the element's
// transfer function: the paper's quadratic filter at (gamma, kc) = (0.5 sigmoid(o0),
// 2 + (N-3) sigmoid(o1)), or the fixed filter when a feature leaves [lo, hi] or the drift
// fallback is on.  sigma_out [E][n].
constexpr int kMlpThreads = 256;
template <typename Real>
constexpr int mlp_elements_per_cta() { return 16; }
template <typename Real, int n>
__global__ void __launch_bounds__(kMlpThreads) mlp_sigma_kernel(const int E, const LearnedIn<Real, n> c, const Real *X) {
  constexpr int H = kHidden, nin = 2 * n, EB = mlp_elements_per_cta<Real>(), T = kMlpThreads;
  __shared__ float w1[H][nin], w2[H][H + 1], w3[2][H], b1[H], b2[H], b3[2];
  __shared__ Real sx[EB][nin], h1[EB][H], h2[EB][H], so[EB][2];
  __shared__ int inr[EB];
  const int tid = threadIdx.x, e0 = blockIdx.x * EB;
  const __nv_bfloat16 *W1 = c.W, *B1 = W1 + H * nin, *W2 = B1 + H, *B2 = W2 + H * H, *W3 = B2 + H, *B3 = W3 + 2 * H;
  for (int k = tid; k < H * nin; k += T) w1[k / nin][k % nin] = __bfloat162float(W1[k]);
  for (int k = tid; k < H * H; k += T) w2[k / H][k % H] = __bfloat162float(W2[k]);
  for (int k = tid; k < 2 * H; k += T) w3[k / H][k % H] = __bfloat162float(W3[k]);
  for (int k = tid; k < H; k += T) { b1[k] = __bfloat162float(B1[k]); b2[k] = __bfloat162float(B2[k]); }
  if (tid < 2) b3[tid] = __bfloat162float(B3[tid]);
  if (tid < EB) inr[tid] = 1;
  __syncthreads();
  for (int k = tid; k < EB * nin; k += T) {
    const int el = k / nin, i = k - el * nin, e = e0 + el;
    Real sv = 0;
    if (e < E) {
      const Real x = X[(size_t)e * nin + i], lo = c.lo[i], hi = c.hi[i];
      if (!(x >= lo && x <= hi)) atomicAnd(&inr[el], 0);
      sv = Real(2) * (x - lo) / (hi - lo) - Real(1);
    }
    sx[el][i] = sv;
  }
  __syncthreads();
  for (int k = tid; k < EB * H; k += T) {
    const int el = k / H, o = k - el * H;
    Real z = (Real)b1[o];
#pragma unroll
    for (int i = 0; i < nin; ++i) z += (Real)w1[o][i] * sx[el][i];
    h1[el][o] = tanh(z);
  }
  __syncthreads();
  for (int k = tid; k < EB * H; k += T) {
    const int el = k / H, o = k - el * H;
    Real z = (Real)b2[o];
#pragma unroll 8
    for (int i = 0; i < H; ++i) z += (Real)w2[o][i] * h1[el][i];
    h2[el][o] = tanh(z);
  }
  __syncthreads();
  if (tid < 2 * EB) {
    const int el = tid >> 1, o = tid & 1;
    Real z = (Real)b3[o];
#pragma unroll 8
    for (int i = 0; i < H; ++i) z += (Real)w3[o][i] * h2[el][i];
    so[el][o] = z;
  }
  __syncthreads();
  for (int k = tid; k < EB * n; k += T) {
    const int el = k / n, j = k - el * n, e = e0 + el;
    if (e >= E) continue;
    const bool use_net = inr[el] && !(c.flag && *c.flag);
    Real sig = c.fixed_sigma[j];
    if (use_net) {
      const Real gam = Real(0.5) / (Real(1) + exp(-so[el][0]));
      const Real kc = Real(2) + Real(n - 4) / (Real(1) + exp(-so[el][1]));
      sig = Real(1);
      if (j > kc) {
        const Real r = (Real(j) - kc) / (Real(n - 1) - kc);
        sig = Real(1) - gam * r * r;
      }
    } else if (j == 0 && c.n_fallback) {
      atomicAdd(c.n_fallback, 1);
    }
    c.sigma_out[(size_t)e * n + j] = sig;
  }
}

// mass-weighted assembly of the learned control's filtered copies at shared nodes,
// then the collision there
template <typename Real, int LAT>
__global__ void __launch_bounds__(256) dss_collide_kernel(const KParams<Real> p) {
  constexpr int Q = LT<LAT>::v.Q;
  const size_t EN = (size_t)p.E * p.Nb;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < p.Gb; u += gridDim.x * blockDim.x) {
    const int c0 = p.bnode_off[u], c1 = p.bnode_off[u + 1];
    const size_t gid = p.bnode_g[u];
    const Real minv = p.bnode_minv[u];
    // populations in two halves, two copies per iteration (loads in flight together), added in
    // ascending copy order
    constexpr int QH = (Q + 1) / 2;
    Real s[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) s[a] = 0;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int a0 = hh * QH;
      int k = c0;
      for (; k + 1 < c1; k += 2) {
        const Real *t0 = p.T + p.bnode_slot[k] + (size_t)a0 * EN, *t1 = p.T + p.bnode_slot[k + 1] + (size_t)a0 * EN;
        Real v0[QH], v1[QH];
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) { v0[a] = t0[a * EN]; v1[a] = t1[a * EN]; }
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) { s[a0 + a] += v0[a]; s[a0 + a] += v1[a]; }
      }
      if (k < c1) {
        const Real *t0 = p.T + p.bnode_slot[k] + (size_t)a0 * EN;
#pragma unroll
        for (int a = 0; a < QH; ++a)
          if (a0 + a < Q) s[a0 + a] += t0[a * EN];
      }
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) s[a] *= minv;
    Real gacc[3];
    node_accel(p, gid, gacc);
    const Real rho = bgk_collide<Real, LAT>(s, p.rho0, p.omega, p.dt, p.half_dt, gacc, p.has_force != 0);
#pragma unroll
    for (int a = 0; a < Q; ++a) p.f0out[(size_t)a * p.Gs + gid] = s[a];
    if (p.has_force) p.rho[gid] = rho;
  }
}

// collision on unique nodes (no pending filter)
template <typename Real, int LAT>
__global__ void __launch_bounds__(256) collide_nodes_kernel(const KParams<Real> p) {
  constexpr int Q = LT<LAT>::v.Q;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (size_t)p.G; g += (size_t)gridDim.x * blockDim.x) {
    Real s[Q], gacc[3];
#pragma unroll
    for (int a = 0; a < Q; ++a) s[a] = p.fin[(size_t)a * p.Gs + g];
    node_accel(p, g, gacc);
    const Real rho = bgk_collide<Real, LAT>(s, p.rho0, p.omega, p.dt, p.half_dt, gacc, p.has_force != 0);
#pragma unroll
    for (int a = 0; a < Q; ++a) p.f0out[(size_t)a * p.Gs + g] = s[a];
    if (p.has_force) p.rho[g] = rho;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename Real, int n>
FastMats<Real, n> make_fast_mats(const SplitHost &h) {
  FastMats<Real, n> m{};
  for (int k = 0; k < n * n; ++k) { m.D[k] = (Real)h.D[k]; m.U[k] = (Real)h.U[k]; m.W[k] = (Real)h.W[k]; }
  for (int k = 0; k < n; ++k) m.w[k] = (Real)h.w[k];
  m.r = h.r;
  fill_even_odd(m, h.D);
  return m;
}

// sets the kernel's dynamic shared-memory limit once per device (per instantiation)
#define SLB_SET_SMEM_ONCE(kernel, smem)                                                          \
  do {                                                                                           \
    static thread_local int attr_dev_ = -1;                                                      \
    static thread_local size_t attr_smem_ = 0;                                                   \
    int dev_ = 0;                                                                                \
    cudaGetDevice(&dev_);                                                                        \
    if (attr_dev_ != dev_ || attr_smem_ < (smem)) {                                              \
      cudaError_t err_ = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem)); \
      if (err_ != cudaSuccess) return err_;                                                      \
      attr_dev_ = dev_;                                                                          \
      attr_smem_ = (smem);                                                                       \
    }                                                                                            \
  } while (0)

template <typename Real, int LAT, int n, bool AFFINE, int PBW = 0>
cudaError_t launch_split_t(const KParams<Real> &p, const SplitHost &h, cudaStream_t s) {
  using S = SplitShape<LAT, n, PBW>;
  const size_t smem = split_smem_bytes<Real, LAT, n, AFFINE, PBW>(p.wall_max);
  auto k = stage_split_kernel<Real, LAT, n, AFFINE, PBW>;
  SLB_SET_SMEM_ONCE(k, smem);
  k<<<p.E * S::NG, S::THREADS, smem, s>>>(p, make_fast_mats<Real, n>(h));
  return cudaGetLastError();
}

template <typename Real, int LAT, int n, bool AFFINE, int MODE>
cudaError_t launch_prologue_t(const KParams<Real> &p, const SplitHost &h, const LearnedPtrs<Real> &lp, cudaStream_t s) {
  LearnedIn<Real, n> c{};
  if (MODE == PRO_LEARNED) {
    for (int k = 0; k < n * n; ++k) { c.Vm[k] = (Real)h.Vm[k]; c.Vinv[k] = (Real)h.Vinv[k]; }
    for (int k = 0; k < n; ++k) c.fixed_sigma[k] = (Real)h.fixed_sigma[k];
    c.W = lp.W; c.lo = lp.lo; c.hi = lp.hi; c.flag = lp.flag; c.acc = lp.acc; c.sigma_out = lp.sigma_out;
    c.feat_out = lp.feat_out; c.n_fallback = lp.n_fallback; c.outputs = lp.outputs;
  }
  const size_t smem = prologue_smem_bytes<Real, LAT, n, AFFINE, MODE>();
  auto k = prologue_kernel<Real, LAT, n, AFFINE, MODE>;
  SLB_SET_SMEM_ONCE(k, smem);
  k<<<p.E, kProThreads, smem, s>>>(p, make_fast_mats<Real, n>(h), c);
  return cudaGetLastError();
}

// learned control of the split form: node features (+ drift integrals), element features X
// [E][2n], then the network over all elements; q: device buffer [2][Gs]
template <typename Real, int LAT, int n>
cudaError_t launch_split_control_t(const KParams<Real> &p, const SplitHost &h, const LearnedPtrs<Real> &lp, Real *q,
                                   Real *X, const double *mass, cudaStream_t s) {
  LearnedIn<Real, n> c{};
  for (int k = 0; k < n * n; ++k) { c.Vm[k] = (Real)h.Vm[k]; c.Vinv[k] = (Real)h.Vinv[k]; }
  for (int k = 0; k < n; ++k) c.fixed_sigma[k] = (Real)h.fixed_sigma[k];
  c.W = lp.W; c.lo = lp.lo; c.hi = lp.hi; c.flag = lp.flag; c.acc = lp.acc; c.sigma_out = lp.sigma_out;
  c.feat_out = lp.feat_out; c.n_fallback = lp.n_fallback; c.outputs = lp.outputs;
  const int blocks = (int)std::min<size_t>(((size_t)p.G + 255) / 256, 152 * 8);
  node_features_kernel<Real, LAT><<<blocks, 256, 0, s>>>(p, q, mass, lp.acc);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  element_features_kernel<Real, n><<<(p.E + kCtlWarps - 1) / kCtlWarps, 32 * kCtlWarps, 0, s>>>(p, c, q, X);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  constexpr int EB = mlp_elements_per_cta<Real>();
  mlp_sigma_kernel<Real, n><<<(p.E + EB - 1) / EB, kMlpThreads, 0, s>>>(p.E, c, X);
  return cudaGetLastError();
}

template <typename Real, int LAT>
cudaError_t launch_dss_collide_t(const KParams<Real> &p, cudaStream_t s) {
  if (p.Gb == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (int)std::min<size_t>(((size_t)p.Gb + threads - 1) / threads, 152 * 32);
  dss_collide_kernel<Real, LAT><<<blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename Real, int LAT>
cudaError_t launch_collide_nodes_t(const KParams<Real> &p, cudaStream_t s) {
  const int threads = 256;
  const int blocks = (int)std::min<size_t>(((size_t)p.G + threads - 1) / threads, 152 * 32);
  collide_nodes_kernel<Real, LAT><<<blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace slb
