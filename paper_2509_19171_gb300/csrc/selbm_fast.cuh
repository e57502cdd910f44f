// Register-blocked stage kernel for compile-time order N and lattice.
//
// One CTA per element; the element's Q x (N+1)^d populations are gathered
// into shared memory once.  Each thread owns one (population, r-line) task:
// the r-line's N+1 values sit in registers, the r-derivative is formed from
// them with D_hat in the kernel-parameter constant bank, and the s- and
// t-derivatives accumulate whole neighbouring r-lines read from shared memory
// (vector loads) scaled by one entry of D_hat each.  The Runge-Kutta weight
// -B dt and the element metrics are folded into the per-population
// coefficients, so an element-interior output costs one FMA per derivative
// term plus two for the stage combination.
//
// Tile layout (FP32, N = 7, 3D): r-line (i1, i2) is stored in slot i1 ^ (i2 & 3)
// of its t-plane and its two 16-byte halves are swapped when bit 2 of i1 is
// set, so that the r-line reads of the s-derivative (four planes per warp), of
// the t-derivative (eight lines per warp), the write-back of results and the
// per-node accesses all hit distinct shared-memory banks.
#pragma once
#include "selbm_kernels.cuh"
#include "selbm_lattice.cuh"
#include "selbm_setup.h"

namespace slb {

// dense D_hat (r-derivative, uniform indices) and the low-rank filter
// F = I + U W (U: n x r, W: r x n), plus GLL weights; passed by value
template <typename Real, int n>
struct FastMats {
  Real D[n * n];
  Real U[n * n];
  Real W[n * n];
  Real w[n];
  // even-odd form of D_hat for even n (see deriv_line): pairs (P_jk, M_jk), j, k < n/2
  Real PM[(n / 2) * (n / 2) * 2 + 2];
  int r;
};

// The GLL nodes are symmetric about 0, so D_hat[n-1-j][n-1-k] = -D_hat[j][k].  With
// P_jk = (D_jk + D_j,n-1-k) / 2 and M_jk = (D_jk - D_j,n-1-k) / 2 (j, k < n/2, formed in FP64)
// the product d = D_hat v of an even-length line is d_j = P e + M o, d_{n-1-j} = M o - P e with
// e_k = v_k + v_{n-1-k}, o_k = v_k - v_{n-1-k}: n^2/2 multiply-adds instead of n^2.
template <typename Real, int n>
void fill_even_odd(FastMats<Real, n> &m, const double *D) {
  constexpr int H = n / 2;
  for (int j = 0; j < H; ++j)
    for (int k = 0; k < H; ++k) {
      m.PM[(j * H + k) * 2] = (Real)(0.5 * (D[j * n + k] + D[j * n + n - 1 - k]));
      m.PM[(j * H + k) * 2 + 1] = (Real)(0.5 * (D[j * n + k] - D[j * n + n - 1 - k]));
    }
}

// d = D_hat v along one line: the even-odd form for even n (FP32: the P and M sums of an output
// pair as one packed FMA chain), the dense product for odd n
template <typename Real, int n>
__device__ __forceinline__ void deriv_line(const FastMats<Real, n> &m, const Real (&v)[n], Real (&d)[n]) {
  if constexpr (n % 2 == 0) {
    constexpr int H = n / 2;
    if constexpr (sizeof(Real) == 4) {
      float2 eo[H];
#pragma unroll
      for (int k = 0; k < H; ++k) eo[k] = make_float2(v[k] + v[n - 1 - k], v[k] - v[n - 1 - k]);
#pragma unroll
      for (int j = 0; j < H; ++j) {
        float2 acc = __fmul2_rn(make_float2(m.PM[j * H * 2], m.PM[j * H * 2 + 1]), eo[0]);
#pragma unroll
        for (int k = 1; k < H; ++k)
          acc = __ffma2_rn(make_float2(m.PM[(j * H + k) * 2], m.PM[(j * H + k) * 2 + 1]), eo[k], acc);
        d[j] = acc.x + acc.y;
        d[n - 1 - j] = acc.y - acc.x;
      }
    } else {
      Real ev[H], od[H];
#pragma unroll
      for (int k = 0; k < H; ++k) { ev[k] = v[k] + v[n - 1 - k]; od[k] = v[k] - v[n - 1 - k]; }
#pragma unroll
      for (int j = 0; j < H; ++j) {
        Real sp = m.PM[j * H * 2] * ev[0], sm = m.PM[j * H * 2 + 1] * od[0];
#pragma unroll
        for (int k = 1; k < H; ++k) {
          sp += m.PM[(j * H + k) * 2] * ev[k];
          sm += m.PM[(j * H + k) * 2 + 1] * od[k];
        }
        d[j] = sp + sm;
        d[n - 1 - j] = sm - sp;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j) {
      Real s = 0;
#pragma unroll
      for (int k = 0; k < n; ++k) s += m.D[j * n + k] * v[k];
      d[j] = s;
    }
  }
}

template <typename Real, int n, int DIM>
struct Tile {
  static constexpr bool SW = sizeof(Real) == 4 && n == 8 && DIM == 3;
  static constexpr int PL = n * n;                          // t-plane stride
  static constexpr int PS = DIM == 3 ? n * PL : n * n;      // population stride
  // r-line (i1, i2) sits in slot i1 ^ (i2 & 3) of its plane; its two 16-byte halves
  // are swapped when bit 2 of i1 is set
  __device__ __forceinline__ static int line(int i1, int i2) { return i2 * PL + (SW ? (i1 ^ (i2 & 3)) : i1) * n; }
  __device__ __forceinline__ static int sw(int i1) { return SW ? (((i1 >> 2) & 1) << 2) : 0; }
  __device__ __forceinline__ static int at(int i0, int i1, int i2) { return line(i1, i2) + (i0 ^ sw(i1)); }
  __device__ __forceinline__ static int node(int i) {
    const int i0 = i % n, i1 = (i / n) % n, i2 = DIM == 3 ? i / (n * n) : 0;
    return at(i0, i1, i2);
  }
};

// out = v + U (W v) on n values; U (n x r) and W (r x n) in shared memory, row stride n
template <typename Real, int n>
__device__ __forceinline__ void filter_vals(Real (&v)[n], const Real *U, const Real *W, int r) {
  Real o[n];
#pragma unroll
  for (int j = 0; j < n; ++j) o[j] = v[j];
#pragma unroll
  for (int q = 0; q < n; ++q) {
    if (q < r) {
      Real s = 0;
#pragma unroll
      for (int k = 0; k < n; ++k) s += W[q * n + k] * v[k];
#pragma unroll
      for (int j = 0; j < n; ++j) o[j] += U[j * n + q] * s;
    }
  }
#pragma unroll
  for (int j = 0; j < n; ++j) v[j] = o[j];
}

// the n values of r-line starting at `src` whose halves are swapped when swz = 4
template <typename Real, int n>
__device__ __forceinline__ void load_line(const Real *src, int swz, Real (&v)[n]) {
  if constexpr (sizeof(Real) == 4 && n % 4 == 0) {
#pragma unroll
    for (int c = 0; c < n; c += 4) {
      const float4 q = *reinterpret_cast<const float4 *>(src + (c ^ swz));
      v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
    }
  } else if constexpr (sizeof(Real) == 8 && n % 2 == 0) {
#pragma unroll
    for (int j = 0; j < n; j += 2) {
      const double2 q = *reinterpret_cast<const double2 *>(src + j);
      v[j] = q.x; v[j + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j) v[j] = src[j];
  }
}

template <typename Real, int n>
__device__ __forceinline__ void store_line(Real *dst, int swz, const Real (&v)[n]) {
  if constexpr (sizeof(Real) == 4 && n % 4 == 0) {
#pragma unroll
    for (int c = 0; c < n; c += 4)
      *reinterpret_cast<float4 *>(dst + (c ^ swz)) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
  } else if constexpr (sizeof(Real) == 8 && n % 2 == 0) {
#pragma unroll
    for (int j = 0; j < n; j += 2) *reinterpret_cast<double2 *>(dst + j) = make_double2(v[j], v[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j) dst[j] = v[j];
  }
}

template <int LAT, int n>
struct FastShape {
  static constexpr int Q = LT<LAT>::v.Q, DIM = LT<LAT>::v.D;
  static constexpr int Np = DIM == 3 ? n * n * n : n * n;
  static constexpr int NL = Np / n;
  static constexpr int THREADS = NL * ((DIM == 3 ? 256 : 128) / NL);   // whole populations per round
  static constexpr int GEO = DIM * DIM + 1;
  static constexpr int NINT = DIM == 3 ? (n - 2) * (n - 2) * (n - 2) : (n - 2) * (n - 2);
};

template <typename Real, int LAT, int n, bool AFFINE>
constexpr size_t fast_smem_bytes(int wall_max) {
  using S = FastShape<LAT, n>;
  using TI = Tile<Real, n, S::DIM>;
  size_t reals = (size_t)S::Q * TI::PS + 3 * n * n + S::Q * S::DIM + S::Q + n;
  if (!AFFINE) reals += (size_t)S::Np * S::GEO;
  reals += (size_t)S::Q * wall_max;
  return reals * sizeof(Real);
}

template <typename Real, int LAT, int n, bool AFFINE>
__global__ void __launch_bounds__(FastShape<LAT, n>::THREADS, (FastShape<LAT, n>::DIM == 3 ? (sizeof(Real) == 4 ? 4 : 2) : 8))
stage_fast_kernel(const KParams<Real> p, const FastMats<Real, n> m) {
  using S = FastShape<LAT, n>;
  constexpr int Q = S::Q, DIM = S::DIM, Np = S::Np, NL = S::NL, T = S::THREADS, GEO = S::GEO, NINT = S::NINT;
  using TI = Tile<Real, n, DIM>;
  constexpr int PS = TI::PS;
  constexpr VelTab V = LT<LAT>::v;
  constexpr int KU = sizeof(Real) == 4 ? n : 2;    // s/t-line loop unroll: partial for FP64 (registers)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sf = reinterpret_cast<Real *>(smem_raw);   // [Q][PS] tile
  Real *sD = sf + Q * PS;                           // [n][n]
  Real *sU = sD + n * n;                            // [n][n]    filter F = I + U W (low rank)
  Real *sW = sU + n * n;                            // [n][n]
  Real *scoef = sW + n * n;                         // [Q][DIM]  (affine: -B dt sum_k e_k dr_l/dx_k)
  Real *sfc = scoef + Q * DIM;                      // [Q]       B dt F*_a / rho
  Real *sw = sfc + Q;                               // [n]       GLL weights
  Real *sgeo = sw + n;                              // [Np][GEO] (curved: -B dt dr_l/dx_k, wJ)
  Real *wbuf = sgeo + (AFFINE ? 0 : Np * GEO);      // [wall nodes][Q]
  const int e = blockIdx.x, tid = threadIdx.x;
  const Real Bdt = p.B * p.dt;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t G = p.G;
  const size_t GS = p.Gs;                         // population stride of the state

  // ---- per-element constants
  __shared__ int s_r;
  for (int k = tid; k < n * n; k += T) sD[k] = m.D[k];
  if (p.stage == 1 && p.apply_filter) {
    for (int k = tid; k < n * n; k += T) { sU[k] = m.U[k]; sW[k] = m.W[k]; }
    if (tid == 0) s_r = m.r;
  }
  if (tid < n) sw[tid] = m.w[tid];
  if (tid < Q) {
    Real ge = 0;
    static_for<0, Q>([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      if (a == tid) {
        if (AFFINE) {
#pragma unroll
          for (int l = 0; l < DIM; ++l) {
            Real c = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k)
              if (V.e[a][k] != 0) c += (V.e[a][k] > 0 ? Real(1) : Real(-1)) * p.el_drdx[((size_t)e * DIM + l) * DIM + k];
            scoef[a * DIM + l] = -Bdt * c;
          }
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (V.e[a][k] != 0) ge += (V.e[a][k] > 0 ? Real(1) : Real(-1)) * p.g[k];
        sfc[a] = Bdt * Real(V.t[a]) * Real(3) * ge;
      }
    });
  }
  // ---- gather the element tile (and per-node metrics on curved elements)
  {
    const Real *__restrict__ fin = p.fin;
    for (int i = tid; i < Np; i += T) {
      const size_t g = l2g[i];
      const int ti = TI::node(i);
#pragma unroll
      for (int a = 0; a < Q; ++a) sf[a * PS + ti] = fin[(size_t)a * GS + g];
      if (!AFFINE) {
        const Real *gm = p.drdx + ((size_t)e * Np + i) * DIM * DIM;
#pragma unroll
        for (int c = 0; c < DIM * DIM; ++c) sgeo[i * GEO + c] = -Bdt * gm[c];
        sgeo[i * GEO + DIM * DIM] = p.wJ[(size_t)e * Np + i];
      }
    }
  }
  __syncthreads();

  if (p.stage == 1) {
    // ---- explicit filter of the previous step (Sec. 2.4), one 1D pass per axis
    if (p.apply_filter) {
      for (int t = tid; t < Q * NL; t += T) {          // r-lines
        const int a = t / NL, L = t - a * NL;
        const int i1 = DIM == 3 ? L % n : L, i2 = DIM == 3 ? L / n : 0;
        Real v[n];
        Real *base = sf + a * PS + TI::line(i1, i2);
        load_line<Real, n>(base, TI::sw(i1), v);
        filter_vals<Real, n>(v, sU, sW, s_r);
        store_line<Real, n>(base, TI::sw(i1), v);
      }
      __syncthreads();
      for (int t = tid; t < Q * NL; t += T) {          // s-lines: (a, i2, i0), i0 fastest
        const int a = t / NL, r = t - a * NL, i0 = r % n, i2 = DIM == 3 ? r / n : 0;
        Real v[n];
#pragma unroll
        for (int k = 0; k < n; ++k) v[k] = sf[a * PS + TI::at(i0, k, i2)];
        filter_vals<Real, n>(v, sU, sW, s_r);
#pragma unroll
        for (int k = 0; k < n; ++k) sf[a * PS + TI::at(i0, k, i2)] = v[k];
      }
      if (DIM == 3) {
        __syncthreads();
        for (int t = tid; t < Q * NL; t += T) {        // t-lines: (a, i1, i0), i0 fastest
          const int a = t / NL, r = t - a * NL, i0 = r % n, i1 = r / n;
          Real v[n];
#pragma unroll
          for (int k = 0; k < n; ++k) v[k] = sf[a * PS + TI::at(i0, i1, k)];
          filter_vals<Real, n>(v, sU, sW, s_r);
#pragma unroll
          for (int k = 0; k < n; ++k) sf[a * PS + TI::at(i0, i1, k)] = v[k];
        }
      }
      __syncthreads();
    }
    // ---- BGK collision with F** at every node (Sec. 2.1), deviation form g = f_bar - t rho0
    for (int i = tid; i < Np; i += T) {
      const int ti = TI::node(i);
      // FP32: keep the node's populations in registers; FP64: re-read them from
      // shared memory (register pressure, and the FP64 path is ALU-bound anyway)
      constexpr int QR = sizeof(Real) == 4 ? Q : 1;
      Real fr[QR];
      if constexpr (sizeof(Real) == 4) {
#pragma unroll
        for (int a = 0; a < Q; ++a) fr[a] = sf[a * PS + ti];
      }
      auto f = [&](int a) -> Real { if constexpr (sizeof(Real) == 4) return fr[a]; else return sf[a * PS + ti]; };
      Real drho = 0, j[3] = {0, 0, 0};
      static_for<0, Q>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        const Real fa = f(a);
        drho += fa;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          if (V.e[a][k] > 0) j[k] += fa;
          else if (V.e[a][k] < 0) j[k] -= fa;
        }
      });
      const Real rho = p.rho0 + drho;
      const Real inv = Real(1) / rho;
      const size_t gid = l2g[i];
      Real ga[3];
      node_accel(p, gid, ga);
      Real u[3] = {0, 0, 0}, F[3] = {0, 0, 0}, uu = 0, uF = 0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        u[k] = j[k] * inv;
        uu += u[k] * u[k];
        if (p.has_force) { F[k] = rho * ga[k]; uF += u[k] * F[k]; }
      }
      const bool own = p.owner[(size_t)e * Np + i] != 0;
      const Real base = Real(1.5) * uu;
      static_for<0, Q>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        Real eu = 0, eF = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          if (V.e[a][k] > 0) { eu += u[k]; eF += F[k]; }
          else if (V.e[a][k] < 0) { eu -= u[k]; eF -= F[k]; }
        }
        const Real t = Real(V.t[a]);
        Real feq = t * (drho + rho * (Real(3) * eu + Real(4.5) * eu * eu - base));
        Real Fss = 0;
        if (p.has_force) {
          Fss = t * (Real(9) * eu * eF - Real(3) * uF);
          feq -= p.half_dt * Fss;
        }
        const Real fa = f(a);
        const Real out = fa - p.omega * (fa - feq) + p.dt * Fss;
        sf[a * PS + ti] = out;
        if (own) p.f0out[(size_t)a * GS + gid] = out;
      });
      if (own && p.has_force) p.rho[gid] = rho;
    }
    __syncthreads();
  }

  // ---- flux bounce-back terms of this element's wall nodes (Sec. 2.2.1), from the tile
  //      before it is overwritten; kept in wbuf[k][a] (scaled by B dt like the rest of T)
  const int w0 = p.wall_off[e], nw = p.wall_off[e + 1] - w0;
  for (int idx = tid; idx < Q * nw; idx += T) {
    const int a = idx % Q, k = idx / Q;
    const WallPt<Real> &wp = p.walls[w0 + k];
    const int ti = TI::node(wp.i);
    Real sum = 0;
    static_for<0, Q>([&](auto ac) {
      constexpr int aa = decltype(ac)::value;
      if (aa == a) {
        constexpr int oa = V.opp[aa];
        for (int f = 0; f < wp.nf; ++f) {
          Real ne = 0, eu = 0;
          const Real *ub = p.wall_u + 3 * (wp.wid[f] - 1);
#pragma unroll
          for (int k2 = 0; k2 < DIM; ++k2) {
            if (V.e[aa][k2] > 0) { ne += wp.n[f][k2]; eu += ub[k2]; }
            else if (V.e[aa][k2] < 0) { ne -= wp.n[f][k2]; eu -= ub[k2]; }
          }
          if (ne < Real(0)) {
            const Real jump = sf[aa * PS + ti] - sf[oa * PS + ti] - Real(2) * Real(V.t[aa]) * p.rho0 * eu * Real(3);
            sum += wp.wsJs[f] * ne * jump;
          }
        }
      }
    });
    wbuf[k * Q + a] = Bdt * sum;
  }

  // ---- streaming right-hand side and stage combination, in rounds of whole populations:
  //      a round's tasks read only their own populations' lines, so after one barrier
  //      their results can replace those populations in the tile
  const Real Je = AFFINE ? p.el_J[e] : Real(0);
  constexpr int ROUNDS = (Q * NL + T - 1) / T;
  // T is a multiple of NL, so this thread's r-line (i1, i2) is the same in every round:
  // the offsets of the s-lines (k, i2) and t-lines (i1, k) it reads are fixed once here
  // (for the swizzled tile they depend on k only through k & 3, plus an immediate)
  const int L = tid % NL;
  const int i1 = DIM == 3 ? L % n : L, i2 = DIM == 3 ? L / n : 0;
  int yq[4], zq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    yq[q] = TI::SW ? i2 * TI::PL + ((q ^ (i2 & 3)) << 3) : i2 * TI::PL;
    zq[q] = TI::SW ? ((i1 ^ q) << 3) : i1 * n;
  }
  auto yline = [&](int k) -> int { return TI::SW ? yq[k & 3] + ((k & 4) << 3) : yq[0] + k * n; };
  auto zline = [&](int k) -> int { return TI::SW ? k * TI::PL + zq[k & 3] : k * TI::PL + zq[0]; };
  const int zswz = TI::sw(i1);
  const Real *sDi1 = sD + i1 * n, *sDi2 = sD + i2 * n;
  const Real wl = DIM == 3 ? sw[i1] * sw[i2] : sw[i1];
  const Real Jwl = Je * wl;
  const bool edge_line = i1 == 0 || i1 == n - 1 || (DIM == 3 && (i2 == 0 || i2 == n - 1));
  const int own = TI::line(i1, i2), own_swz = TI::sw(i1);
  for (int rd = 0; rd < ROUNDS; ++rd) {
    const int t = rd * T + tid;
    const bool active = t < Q * NL;
    const int a = active ? t / NL : 0;
    Real res[n];
    if (active) {
      const Real *fa = sf + a * PS;
      Real v[n];
      load_line<Real, n>(fa + own, own_swz, v);
      Real adv[n];
#pragma unroll
      for (int j = 0; j < n; ++j) adv[j] = 0;
      if (AFFINE) {
        const Real c0 = scoef[a * DIM + 0], c1 = scoef[a * DIM + 1];
        const Real c2 = DIM == 3 ? scoef[a * DIM + 2] : Real(0);
        if (c0 != Real(0)) {
          Real d[n];
          deriv_line<Real, n>(m, v, d);
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] = c0 * d[j];
        }
        if (c1 != Real(0)) {
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            const Real s = c1 * sDi1[k];
            Real w[n];
            load_line<Real, n>(fa + yline(k), TI::sw(k), w);
#pragma unroll
            for (int j = 0; j < n; ++j) adv[j] += s * w[j];
          }
        }
        if (DIM == 3 && c2 != Real(0)) {
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            const Real s = c2 * sDi2[k];
            Real w[n];
            load_line<Real, n>(fa + zline(k), zswz, w);
#pragma unroll
            for (int j = 0; j < n; ++j) adv[j] += s * w[j];
          }
        }
      } else {
        // curved elements: adv = sum_l c_l d_l with c_l = sum_k e_k (-B dt dr_l/dx_k) per node
        int ek[3] = {0, 0, 0};
        static_for<0, Q>([&](auto ac) {
          constexpr int aa = decltype(ac)::value;
          if (aa == a) { ek[0] = V.e[aa][0]; ek[1] = V.e[aa][1]; ek[2] = V.e[aa][2]; }
        });
        auto coef = [&](int j, int l) -> Real {
          const Real *gm = sgeo + (L * n + j) * GEO + l * DIM;
          Real c = 0;
#pragma unroll
          for (int k = 0; k < DIM; ++k)
            if (ek[k] != 0) c += ek[k] > 0 ? gm[k] : -gm[k];
          return c;
        };
        {
          Real d[n];
          deriv_line<Real, n>(m, v, d);
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] = coef(j, 0) * d[j];
        }
        {
          Real d[n];
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = 0;
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            const Real s = sDi1[k];
            Real w[n];
            load_line<Real, n>(fa + yline(k), TI::sw(k), w);
#pragma unroll
            for (int j = 0; j < n; ++j) d[j] += s * w[j];
          }
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] += coef(j, 1) * d[j];
        }
        if (DIM == 3) {
          Real d[n];
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = 0;
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            const Real s = sDi2[k];
            Real w[n];
            load_line<Real, n>(fa + zline(k), zswz, w);
#pragma unroll
            for (int j = 0; j < n; ++j) d[j] += s * w[j];
          }
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] += coef(j, 2) * d[j];
        }
      }
      // element-interior nodes: B f^{s-1} + (-B dt) e.grad f  (A f^0 is added on output);
      // element-boundary nodes: weighted share wJ (-B dt) e.grad f for the assembly
#pragma unroll
      for (int j = 0; j < n; ++j) {
        const bool bnd = edge_line || j == 0 || j == n - 1;
        if (!bnd) {
          res[j] = (p.stage == 1 ? v[j] : p.B * v[j]) + adv[j];
        } else {
          const Real wJ = AFFINE ? Jwl * m.w[j] : sgeo[(L * n + j) * GEO + DIM * DIM];
          res[j] = wJ * adv[j];
        }
      }
    }
    __syncthreads();
    if (active) store_line<Real, n>(sf + a * PS + own, own_swz, res);
  }
  __syncthreads();
  // ---- outputs, one thread per node and all populations in flight (coalesced across
  //      the warp for each population): element-interior nodes finish (+ A f^0, + B dt F*),
  //      element-boundary nodes write their share to the trace T[a][e*Nb + b]
  {
    const Real *__restrict__ f0 = p.f0;
    const Real *__restrict__ rho = p.rho;
    Real *__restrict__ fout = p.fout;
    Real *__restrict__ Tr = p.T;
    const size_t EN = (size_t)p.E * p.Nb;
    for (int i = tid; i < Np; i += T) {
      const int ti = TI::node(i);
      const int b = p.bslot[i];
      if (b < 0) {
        const size_t gid = l2g[i];
        const Real rg = p.has_force ? rho[gid] : Real(0);
        const Real *f0p = f0 + gid;
        Real *fo = fout + gid;
        // B dt F*_a / rho, with the per-node acceleration field: + B dt 3 t_a e_a . (A S_g)
        Real sx[3] = {0, 0, 0};
        const bool field = p.fS != nullptr;
        if (field) {
          const Real A = *p.famp;
#pragma unroll
          for (int k = 0; k < 3; ++k) sx[k] = A * p.fS[(size_t)k * G + gid];
        }
        auto force = [&](int a) -> Real {
          if (!field) return sfc[a] * rg;
          Real es = 0;
#pragma unroll
          for (int k = 0; k < DIM; ++k) es += Real(V.e[a][k]) * sx[k];
          return (sfc[a] + p.B * p.dt * Real(V.t[a]) * Real(3) * es) * rg;
        };
        if (p.stage != 1) {
#pragma unroll
          for (int a = 0; a < Q; ++a) {
            Real out = sf[a * PS + ti] + p.A * f0p[(size_t)a * GS];
            if (p.has_force) out += force(a);
            fo[(size_t)a * GS] = out;
          }
        } else {
#pragma unroll
          for (int a = 0; a < Q; ++a) {
            Real out = sf[a * PS + ti];
            if (p.has_force) out += force(a);
            fo[(size_t)a * GS] = out;
          }
        }
      } else {
        Real *tp = Tr + (size_t)e * p.Nb + b;
#pragma unroll
        for (int a = 0; a < Q; ++a) tp[a * EN] = sf[a * PS + ti];
      }
    }
  }
  if (nw > 0) {
    __syncthreads();
    const size_t EN = (size_t)p.E * p.Nb;
    for (int idx = tid; idx < Q * nw; idx += T) {
      const int a = idx % Q, k = idx / Q;
      p.T[a * EN + (size_t)e * p.Nb + p.walls[w0 + k].b] += wbuf[k * Q + a];
    }
  }
}

// host-side launcher for one (Real, LAT, n, AFFINE)
template <typename Real, int LAT, int n, bool AFFINE>
cudaError_t launch_fast_t(const KParams<Real> &p, const double *D, const double *U, const double *W, int r,
                          const double *w, cudaStream_t s) {
  FastMats<Real, n> m{};
  for (int k = 0; k < n * n; ++k) { m.D[k] = (Real)D[k]; m.U[k] = (Real)U[k]; m.W[k] = (Real)W[k]; }
  for (int k = 0; k < n; ++k) m.w[k] = (Real)w[k];
  m.r = r;
  fill_even_odd(m, D);
  const size_t smem = fast_smem_bytes<Real, LAT, n, AFFINE>(p.wall_max);
  auto k = stage_fast_kernel<Real, LAT, n, AFFINE>;
  static thread_local int attr_dev = -1;
  static thread_local size_t attr_smem = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev || attr_smem < smem) {
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_dev = dev;
    attr_smem = smem;
  }
  k<<<p.E, FastShape<LAT, n>::THREADS, smem, s>>>(p, m);
  return cudaGetLastError();
}

}  // namespace slb
