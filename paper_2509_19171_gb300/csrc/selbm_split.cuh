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
// With the learned control, copies of a shared node are filtered by different
// element filters; the prologue writes their weighted shares wJ f to the trace and
// dss_collide_kernel forms the mass-weighted average and collides it.
#pragma once
#include <cuda_bf16.h>

#include <algorithm>

#include "selbm_collide.cuh"
#include "selbm_fast.cuh"

namespace slb {

// asynchronous global -> shared copy of one value (cp.async, 4 or 8 bytes)
template <typename Real>
__device__ __forceinline__ void cp_async(Real *dst, const Real *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(Real) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int LAT, int n>
struct SplitShape {
  static constexpr int Q = LT<LAT>::v.Q;
  static constexpr int Np = n * n * n, NL = n * n;
  static constexpr int LPR = 256 / NL < 1 ? 1 : 256 / NL;         // populations per round of tasks
  static constexpr int THREADS = LPR * NL;                        // one (population, r-line) task per round
  static constexpr int ROUNDS = 2;
  static constexpr int PB = ROUNDS * LPR;                         // populations per work item
  static constexpr int NG = (Q + PB - 1) / PB;                    // work items per element
  static constexpr int NPT = (Np + THREADS - 1) / THREADS;        // nodes per thread when gathering
};

template <typename Real, int LAT, int n, bool AFFINE>
constexpr size_t split_smem_bytes(int wall_max) {
  using S = SplitShape<LAT, n>;
  using TI = Tile<Real, n, 3>;
  size_t reals = 2 * (size_t)S::PB * TI::PS + n * n + S::PB * 3 + 2 * S::PB + n;
  if (!AFFINE) reals += (size_t)S::Np * 10;
  reals += (size_t)S::PB * wall_max;
  return reals * sizeof(Real);
}

// bit a of pos_mask(k) (neg_mask(k)) is set when population a has e_k = +1 (-1)
constexpr uint32_t vel_mask(const VelTab &v, int k, int sgn) {
  uint32_t m = 0;
  for (int a = 0; a < v.Q; ++a)
    if (v.e[a][k] == sgn) m |= 1u << a;
  return m;
}
template <typename Real>
__device__ __forceinline__ Real mask_sign(uint32_t pos, uint32_t neg, int a) {
  return Real((int)((pos >> a) & 1u) - (int)((neg >> a) & 1u));
}

// acc[j] += s * w[j], j < n (packed FP32 pairs where the type allows)
template <typename Real, int n>
__device__ __forceinline__ void axpy_line(Real (&acc)[n], Real s, const Real (&w)[n]) {
  if constexpr (sizeof(Real) == 4 && n % 2 == 0) {
    const float2 ss = make_float2(s, s);
#pragma unroll
    for (int j = 0; j < n; j += 2) {
      const float2 r = __ffma2_rn(ss, make_float2(w[j], w[j + 1]), make_float2(acc[j], acc[j + 1]));
      acc[j] = r.x;
      acc[j + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j) acc[j] += s * w[j];
  }
}

// asynchronous copy of one value to a shared-memory byte address
template <typename Real>
__device__ __forceinline__ void cp_async_s(unsigned dst, const Real *src) {
  if constexpr (sizeof(Real) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}

// ---------------------------------------------------------------------------
// one Runge-Kutta stage for PB populations of one element
// ---------------------------------------------------------------------------
template <typename Real, int LAT, int n, bool AFFINE>
__global__ void __launch_bounds__(SplitShape<LAT, n>::THREADS, (sizeof(Real) == 4 ? (AFFINE ? 5 : 4) : 2))
stage_split_kernel(const KParams<Real> p, const FastMats<Real, n> m) {
  using S = SplitShape<LAT, n>;
  constexpr int Q = S::Q, DIM = 3, Np = S::Np, NL = S::NL, T = S::THREADS, PB = S::PB, NG = S::NG;
  constexpr int NPT = S::NPT, LPR = S::LPR, ROUNDS = S::ROUNDS;
  using TI = Tile<Real, n, DIM>;
  constexpr int PS = TI::PS;
  constexpr VelTab V = LT<LAT>::v;
  constexpr uint32_t POS[3] = {vel_mask(V, 0, 1), vel_mask(V, 1, 1), vel_mask(V, 2, 1)};
  constexpr uint32_t NEG[3] = {vel_mask(V, 0, -1), vel_mask(V, 1, -1), vel_mask(V, 2, -1)};
  constexpr int KU = sizeof(Real) == 4 ? n : 2;
  constexpr unsigned RS = sizeof(Real);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sf = reinterpret_cast<Real *>(smem_raw);   // [PB][PS] f^{s-1} of the group
  Real *so = sf + PB * PS;                          // [PB][PS] f^0 in, stage result out
  Real *sD = so + PB * PS;                          // [n][n]
  Real *cf = sD + n * n;                            // [PB][DIM] (affine: -B dt sum_k e_k dr_l/dx_k)
  Real *fc = cf + PB * DIM;                         // [2][PB]   B dt F*_a / rho; B dt 3 t_a
  Real *sw = fc + 2 * PB;                           // [n]
  Real *sg = sw + n;                                // curved: dr_l/dx_k [Np][9], wJ [Np]
  Real *wbuf = sg + (AFFINE ? 0 : Np * 10);         // [wall nodes][PB]
  const int e = blockIdx.x / NG, a0 = (blockIdx.x - e * NG) * PB;
  const int na = Q - a0 < PB ? Q - a0 : PB;
  const bool full = na == PB;
  const int tid = threadIdx.x;
  const Real Bdt = p.B * p.dt;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t G = p.G;
  const bool use_f0 = p.stage != 1;

  // ---- gather f^{s-1} of the group (and f^0 of element-interior nodes) with asynchronous
  //      copies: no register staging, all of them in flight at once
  {
    const unsigned s_f = (unsigned)__cvta_generic_to_shared(sf), s_o = (unsigned)__cvta_generic_to_shared(so);
    const Real *fin = p.fin + (size_t)a0 * G;
    const Real *f0 = p.f0 + (size_t)a0 * G;
#pragma unroll
    for (int r = 0; r < NPT; ++r) {
      const int i = tid + r * T;
      if (i < Np) {
        const int g = l2g[i];
        const bool f0n = use_f0 && p.bslot[i] < 0;
        const unsigned ti = TI::node(i) * RS;
        const Real *src = fin + g, *src0 = f0 + g;
        if (full) {
#pragma unroll
          for (int pl = 0; pl < PB; ++pl) cp_async_s<Real>(s_f + ti + pl * PS * RS, src + pl * G);
          if (f0n) {
#pragma unroll
            for (int pl = 0; pl < PB; ++pl) cp_async_s<Real>(s_o + ti + pl * PS * RS, src0 + pl * G);
          }
        } else {
#pragma unroll
          for (int pl = 0; pl < PB; ++pl) {
            if (pl < na) {
              cp_async_s<Real>(s_f + ti + pl * PS * RS, src + pl * G);
              if (f0n) cp_async_s<Real>(s_o + ti + pl * PS * RS, src0 + pl * G);
            }
          }
        }
      }
    }
    if (!AFFINE) {
      const unsigned s_g = (unsigned)__cvta_generic_to_shared(sg);
      const Real *gm = p.drdx + (size_t)e * Np * 9;
      for (int c = tid; c < Np * 9; c += T) cp_async_s<Real>(s_g + c * RS, gm + c);
      const Real *wj = p.wJ + (size_t)e * Np;
      for (int c = tid; c < Np; c += T) cp_async_s<Real>(s_g + (Np * 9 + c) * RS, wj + c);
    }
  }
  // ---- per-element constants while the copies are in flight
  for (int k = tid; k < n * n; k += T) sD[k] = m.D[k];
  if (tid < n) sw[tid] = m.w[tid];
  if (AFFINE && tid < PB * DIM) {
    const int pl = tid / DIM, l = tid - pl * DIM;
    const int a = a0 + pl;
    Real c = 0;
    if (a < Q) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) c += mask_sign<Real>(POS[k], NEG[k], a) * p.el_drdx[((size_t)e * DIM + l) * DIM + k];
    }
    cf[tid] = -Bdt * c;
  }
  if (p.has_force && tid < na) {
    const int a = a0 + tid;
    Real ge = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) ge += mask_sign<Real>(POS[k], NEG[k], a) * p.g[k];
    Real ta = 0;
    static_for<0, Q>([&](auto ac) {
      constexpr int aa = decltype(ac)::value;
      if (aa == a) ta = Real(V.t[aa]);
    });
    fc[tid] = Bdt * ta * Real(3) * ge;
    fc[PB + tid] = Bdt * ta * Real(3);
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- flux bounce-back terms of the group's populations at this element's wall nodes
  //      (Sec. 2.2.1); the opposite population comes from the unique-node array
  const int w0 = p.wall_off[e], nw = p.wall_off[e + 1] - w0;
  for (int idx = tid; idx < na * nw; idx += T) {
    const int k = idx / na, pl = idx - k * na;
    const int a = a0 + pl;
    const WallPt<Real> &wp = p.walls[w0 + k];
    const int ti = TI::node(wp.i);
    const size_t g = l2g[wp.i];
    Real sum = 0;
    static_for<0, Q>([&](auto ac) {
      constexpr int aa = decltype(ac)::value;
      if (aa == a) {
        constexpr int oa = V.opp[aa];
        const Real fo = p.fin[(size_t)oa * G + g];
        for (int f = 0; f < wp.nf; ++f) {
          Real ne = 0, eu = 0;
          const Real *ub = p.wall_u + 3 * (wp.wid[f] - 1);
#pragma unroll
          for (int k2 = 0; k2 < DIM; ++k2) {
            if (V.e[aa][k2] > 0) { ne += wp.n[f][k2]; eu += ub[k2]; }
            else if (V.e[aa][k2] < 0) { ne -= wp.n[f][k2]; eu -= ub[k2]; }
          }
          if (ne < Real(0)) {
            const Real jump = sf[pl * PS + ti] - fo - Real(2) * Real(V.t[aa]) * p.rho0 * eu * Real(3);
            sum += wp.wsJs[f] * ne * jump;
          }
        }
      }
    });
    wbuf[k * PB + pl] = Bdt * sum;
  }

  // ---- (population, r-line) tasks, ROUNDS per thread with the same r-line (i1, i2);
  //      a task reads f^{s-1} lines from sf and replaces its own line of so (f^0 in,
  //      result out), which no other task touches
  if constexpr (AFFINE && TI::SW) {
    // swizzled FP32 tile (N = 7): one warp per population, one axis per pass.  A pass
    // takes two adjacent lines along its axis into registers (8-byte loads, conflict-free
    // on the swizzled tile), applies D and adds c_l (D f) into the population's slice of so,
    // whose element-interior nodes start as A f^0; the r-pass adds the r-derivative and
    // finishes the stage combination.  Every tile value is read once per axis.
    const int pl = tid >> 5, lane = tid & 31;
    const int x = lane & 7, y = lane >> 3;                    // lines (x, y) and (x, y + 4)
    if (pl < na) {
      const Real *fa = sf + pl * PS;
      Real *oa = so + pl * PS;
      const Real c0 = cf[pl * DIM + 0], c1 = cf[pl * DIM + 1], c2 = cf[pl * DIM + 2];
      // s-pass (AX = 1) and t-pass (AX = 2): the lines along the axis at r-index xp, xp + 1
      // and o (the remaining index), one pair per lane
      // acc: so holds earlier passes' sums (add to it); otherwise so starts as A f^0 on
      // element-interior nodes (stages 2, 3) and 0 elsewhere.  Selects, not branches.
      auto pass = [&](auto ax, auto acc_c, Real c) {
        constexpr int AX = decltype(ax)::value;
        constexpr bool acc = decltype(acc_c)::value;
        const int xp = 2 * (lane & 3), o = lane >> 2;          // lines (xp, o) and (xp + 1, o)
        const bool oin = o > 0 && o < n - 1;
        const Real A = use_f0 ? p.A : Real(0);
        const bool k0 = acc || (use_f0 && oin && xp > 0), k1 = acc || (use_f0 && oin && xp + 1 < n - 1);
        const Real a0 = acc ? Real(1) : A;
        float2 d[n];
#pragma unroll
        for (int j = 0; j < n; ++j) d[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const float2 vk = *reinterpret_cast<const float2 *>(fa + (AX == 1 ? TI::at(xp, k, o) : TI::at(xp, o, k)));
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = __ffma2_rn(make_float2(m.D[j * n + k], m.D[j * n + k]), vk, d[j]);
        }
        const float2 cc = make_float2(c, c);
#pragma unroll
        for (int j = 0; j < n; ++j) {
          float2 *dst = reinterpret_cast<float2 *>(oa + (AX == 1 ? TI::at(xp, j, o) : TI::at(xp, o, j)));
          const float2 old = *dst;
          float2 r = __fmul2_rn(cc, d[j]);
          const bool jin = acc || (j > 0 && j < n - 1);
          r.x = (k0 && jin) ? fmaf(a0, old.x, r.x) : r.x;
          r.y = (k1 && jin) ? fmaf(a0, old.y, r.y) : r.y;
          *dst = r;
        }
        __syncwarp();
      };
      if (c1 != Real(0)) pass(std::integral_constant<int, 1>{}, std::false_type{}, c1);
      if (c2 != Real(0)) {
        if (c1 != Real(0)) pass(std::integral_constant<int, 2>{}, std::true_type{}, c2);
        else pass(std::integral_constant<int, 2>{}, std::false_type{}, c2);
      }
      const bool fresh = c1 == Real(0) && c2 == Real(0);     // so holds f^0 or nothing yet
      // r-pass and stage combination, lines (x, y) and (x, y + 4)
      const Real Jwx = p.el_J[e] * sw[x];
      const int swz = TI::sw(x);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int o = y + 4 * h;
        const bool lin = x > 0 && x < n - 1 && o > 0 && o < n - 1;
        const int own = TI::line(x, o);
        Real v[n], acc[n];
        load_line<Real, n>(fa + own, swz, v);
        if (!fresh) {
          load_line<Real, n>(oa + own, swz, acc);
        } else if (use_f0 && lin) {
          load_line<Real, n>(oa + own, swz, acc);
          acc[0] = 0;
          acc[n - 1] = 0;
#pragma unroll
          for (int j = 1; j < n - 1; ++j) acc[j] *= p.A;
        } else {
#pragma unroll
          for (int j = 0; j < n; ++j) acc[j] = 0;
        }
        if (c0 != Real(0)) {
#pragma unroll
          for (int j = 0; j < n; ++j) {
            Real d = 0;
#pragma unroll
            for (int k = 0; k < n; ++k) d += m.D[j * n + k] * v[k];
            acc[j] += c0 * d;
          }
        }
        const Real Jwl = Jwx * sw[o];
        Real res[n];
        if (!lin) {
#pragma unroll
          for (int j = 0; j < n; ++j) res[j] = Jwl * m.w[j] * acc[j];
        } else {
          res[0] = Jwl * m.w[0] * acc[0];
          res[n - 1] = Jwl * m.w[n - 1] * acc[n - 1];
#pragma unroll
          for (int j = 1; j < n - 1; ++j) res[j] = p.B * v[j] + acc[j];
        }
        store_line<Real, n>(oa + own, swz, res);
      }
    }
  } else
  {
    const int L = tid % NL;
    const int i1 = L % n, i2 = L / n;
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
    const Real *swj = sg + Np * 9;
    const Real Jwl = AFFINE ? p.el_J[e] * sw[i1] * sw[i2] : Real(0);
    const bool edge_line = i1 == 0 || i1 == n - 1 || i2 == 0 || i2 == n - 1;
    const int own = TI::line(i1, i2), own_swz = TI::sw(i1);
#pragma unroll 1
    for (int rd = 0; rd < ROUNDS; ++rd) {
      const int pl = tid / NL + rd * LPR;
      if (pl >= na) break;
      const Real *fa = sf + pl * PS;
      // t-line k of this task: halves at zlo[k & 3] + k PL and zhi[k & 3] + k PL
      const Real *zlo[4], *zhi[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        zlo[q] = TI::SW ? fa + zq[q] + zswz : fa;
        zhi[q] = TI::SW ? fa + zq[q] + (4 ^ zswz) : fa;
      }
      auto load_t = [&](int k, Real (&w)[n]) {
        if constexpr (TI::SW) {
          const float4 a = *reinterpret_cast<const float4 *>(zlo[k & 3] + k * TI::PL);
          const float4 b = *reinterpret_cast<const float4 *>(zhi[k & 3] + k * TI::PL);
          w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
          w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
          load_line<Real, n>(fa + zline(k), zswz, w);
        }
      };
      Real v[n];
      load_line<Real, n>(fa + own, own_swz, v);
      Real adv[n];
#pragma unroll
      for (int j = 0; j < n; ++j) adv[j] = 0;
      if (AFFINE) {
        const Real c0 = cf[pl * DIM + 0], c1 = cf[pl * DIM + 1], c2 = cf[pl * DIM + 2];
        if (c0 != Real(0)) {
#pragma unroll
          for (int j = 0; j < n; ++j) {
            Real d = 0;
#pragma unroll
            for (int k = 0; k < n; ++k) d += m.D[j * n + k] * v[k];
            adv[j] = c0 * d;
          }
        }
        if (c1 != Real(0)) {
          Real dr[n];
          if (KU == n) load_line<Real, n>(sDi1, 0, dr);
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            Real w[n];
            load_line<Real, n>(fa + yline(k), TI::sw(k), w);
            axpy_line<Real, n>(adv, c1 * (KU == n ? dr[k] : sDi1[k]), w);
          }
        }
        if (c2 != Real(0)) {
          Real dr[n];
          if (KU == n) load_line<Real, n>(sDi2, 0, dr);
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            Real w[n];
            load_t(k, w);
            axpy_line<Real, n>(adv, c2 * (KU == n ? dr[k] : sDi2[k]), w);
          }
        }
      } else {
        // curved elements: adv = -B dt sum_l c_l d_l with c_l = sum_k e_k dr_l/dx_k per node
        const int a = a0 + pl;
        const Real ek[3] = {mask_sign<Real>(POS[0], NEG[0], a), mask_sign<Real>(POS[1], NEG[1], a),
                            mask_sign<Real>(POS[2], NEG[2], a)};
        auto coef = [&](int j, int l) -> Real {
          const Real *gm = sg + (L * n + j) * 9 + l * DIM;
          return -Bdt * (ek[0] * gm[0] + ek[1] * gm[1] + ek[2] * gm[2]);
        };
#pragma unroll
        for (int j = 0; j < n; ++j) {
          Real d = 0;
#pragma unroll
          for (int k = 0; k < n; ++k) d += m.D[j * n + k] * v[k];
          adv[j] = coef(j, 0) * d;
        }
        {
          Real d[n], dr[n];
          if (KU == n) load_line<Real, n>(sDi1, 0, dr);
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = 0;
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            Real w[n];
            load_line<Real, n>(fa + yline(k), TI::sw(k), w);
            axpy_line<Real, n>(d, KU == n ? dr[k] : sDi1[k], w);
          }
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] += coef(j, 1) * d[j];
        }
        {
          Real d[n], dr[n];
          if (KU == n) load_line<Real, n>(sDi2, 0, dr);
#pragma unroll
          for (int j = 0; j < n; ++j) d[j] = 0;
#pragma unroll KU
          for (int k = 0; k < n; ++k) {
            Real w[n];
            load_t(k, w);
            axpy_line<Real, n>(d, KU == n ? dr[k] : sDi2[k], w);
          }
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] += coef(j, 2) * d[j];
        }
      }
      // element-interior nodes: A f^0 + B f^{s-1} + (-B dt) e.grad f (B dt F* added on
      // output); element-boundary nodes: weighted share wJ (-B dt) e.grad f
      Real *ob = so + pl * PS + own;
      auto wJ = [&](int j) -> Real { return AFFINE ? Jwl * m.w[j] : swj[L * n + j]; };
      Real res[n];
      if (edge_line) {
#pragma unroll
        for (int j = 0; j < n; ++j) res[j] = wJ(j) * adv[j];
      } else {
        res[0] = wJ(0) * adv[0];
        res[n - 1] = wJ(n - 1) * adv[n - 1];
        if (use_f0) {
          Real f0l[n];
          load_line<Real, n>(ob, own_swz, f0l);
#pragma unroll
          for (int j = 1; j < n - 1; ++j) res[j] = p.B * v[j] + adv[j] + p.A * f0l[j];
        } else {
#pragma unroll
          for (int j = 1; j < n - 1; ++j) res[j] = p.B * v[j] + adv[j];
        }
      }
      store_line<Real, n>(ob, own_swz, res);
    }
  }
  __syncthreads();
  if (nw > 0) {
    // wall terms join the weighted shares of their boundary nodes
    for (int idx = tid; idx < na * nw; idx += T) {
      const int k = idx / na, pl = idx - k * na;
      so[pl * PS + TI::node(p.walls[w0 + k].i)] += wbuf[k * PB + pl];
    }
    __syncthreads();
  }

  // ---- outputs, one node per thread with the group's populations (coalesced across the
  //      warp for each population)
  {
    const size_t EN = (size_t)p.E * p.Nb;
#pragma unroll
    for (int r = 0; r < NPT; ++r) {
      const int i = tid + r * T;
      if (i < Np) {
        const Real *sv = so + TI::node(i);
        const int b = p.bslot[i];
        if (b < 0) {
          const int g = l2g[i];
          Real *fo = p.fout + (size_t)a0 * G + g;
          if (p.has_force && !p.fS) {
            const Real rg = p.rho[g];
#pragma unroll
            for (int pl = 0; pl < PB; ++pl)
              if (pl < na) fo[pl * G] = sv[pl * PS] + fc[pl] * rg;
          } else if (p.has_force) {
            const Real rg = p.rho[g];
            const Real A = *p.famp;                 // A(t) S_g of the per-node field
            const Real sx[3] = {A * p.fS[g], A * p.fS[G + g], A * p.fS[2 * G + g]};
#pragma unroll
            for (int pl = 0; pl < PB; ++pl)
              if (pl < na) {
                const int a = a0 + pl;
                const Real es = mask_sign<Real>(POS[0], NEG[0], a) * sx[0] + mask_sign<Real>(POS[1], NEG[1], a) * sx[1] +
                                mask_sign<Real>(POS[2], NEG[2], a) * sx[2];
                fo[pl * G] = sv[pl * PS] + (fc[pl] + fc[PB + pl] * es) * rg;
              }
          } else if (full) {
#pragma unroll
            for (int pl = 0; pl < PB; ++pl) fo[pl * G] = sv[pl * PS];
          } else {
#pragma unroll
            for (int pl = 0; pl < PB; ++pl)
              if (pl < na) fo[pl * G] = sv[pl * PS];
          }
        } else {
          Real *tp = p.T + (size_t)a0 * EN + (size_t)e * p.Nb + b;
          if (full) {
#pragma unroll
            for (int pl = 0; pl < PB; ++pl) tp[pl * EN] = sv[pl * PS];
          } else {
#pragma unroll
            for (int pl = 0; pl < PB; ++pl)
              if (pl < na) tp[pl * EN] = sv[pl * PS];
          }
        }
      }
    }
  }
}

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
  if (MODE == PRO_LEARNED)
    reals += 2 * (size_t)TI::PS + n * n + n + 2 * n + 2 * kHidden + 2 + (kProThreads / 32) * 2 * n;
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
__global__ void __launch_bounds__(kProThreads, sizeof(Real) == 4 ? (MODE == PRO_LEARNED ? 3 : 4) : 1)
prologue_kernel(const KParams<Real> p, const FastMats<Real, n> m, const LearnedIn<Real, n> c) {
  constexpr int Q = LT<LAT>::v.Q, DIM = 3, Np = n * n * n, T = kProThreads, NW = T / 32, H = kHidden, nin = 2 * n;
  using TI = Tile<Real, n, DIM>;
  constexpr int PS = TI::PS;
  constexpr VelTab V = LT<LAT>::v;
  constexpr bool LEARNED = MODE == PRO_LEARNED;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *sf = reinterpret_cast<Real *>(smem_raw);   // [Q][PS]
  Real *sM0 = sf + Q * PS;                          // learned: [n][n] F_e or U_e^T
  Real *sM1 = sM0 + n * n;                          // learned: [n][n] V^-1
  Real *sq = sM1 + n * n;                           // learned: [2][PS] rho - rho0, |u| -> modal
  Real *sVm = sq + 2 * PS;                          // [n][n]
  Real *ssig = sVm + n * n;                         // [n]
  Real *sx = ssig + n;                              // [2n]
  Real *h1 = sx + nin;                              // [64]
  Real *h2 = h1 + H;                                // [64]
  Real *so = h2 + H;                                // [2]
  Real *spart = so + 2;                             // [NW][2n]
  __shared__ double dred[NW][2];
  __shared__ int s_r, in_range, s_mode[n];
  const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t G = p.G;
  auto weight = [&](int i) -> Real {
    if (AFFINE) {
      const int i0 = i % n, i1 = (i / n) % n, i2 = i / (n * n);
      return p.el_J[e] * p.gllw[i0] * p.gllw[i1] * p.gllw[i2];
    }
    return p.wJ[(size_t)e * Np + i];
  };
  if (LEARNED) {
    for (int k = tid; k < n * n; k += T) { sM1[k] = c.Vinv[k]; sVm[k] = c.Vm[k]; }
    if (tid == 0) in_range = 1;
  }
  // ---- gather with asynchronous copies (all Q populations of the thread's nodes in
  //      flight at once); the learned control then takes rho - rho0 and |u| at every node
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
  double pm = 0.0, pk = 0.0;
  if (LEARNED) {
    for (int i = tid; i < Np; i += T) {        // the nodes this thread copied
      const int ti = TI::node(i);
      Real drho = 0, j[3] = {0, 0, 0};
      static_for<0, Q>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        const Real v = sf[a * PS + ti];
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
      sq[ti] = drho;
      sq[PS + ti] = sqrt(uu);
      if (c.acc) {
        const double wq = (double)weight(i);
        pm += wq * (double)rho;
        pk += 0.5 * (double)p.rho0 * wq * (double)uu;
      }
    }
  }
  if (LEARNED && c.acc) {
    pm = warp_sum(pm);
    pk = warp_sum(pk);
    if (lane == 0) { dred[wid][0] = pm; dred[wid][1] = pk; }
  }
  __syncthreads();

  if (LEARNED) {
    if (c.acc && tid == 0) {
      double sm = 0.0, sk = 0.0;
      for (int w = 0; w < NW; ++w) { sm += dred[w][0]; sk += dred[w][1]; }
      atomicAdd(&c.acc[0], sm);
      atomicAdd(&c.acc[1], sk);
    }
    // modal coefficients of both fields: V^-1 along every axis
    tile_pass3<Real, n, 2, T>(sq, tid, [&](Real (&v)[n]) { dense_vals<Real, n>(v, sM1); });
    // shell energies E_k = sum over max(k0, k1, k2) = k of the squared coefficients
    Real en[2][n];
#pragma unroll
    for (int k = 0; k < n; ++k) { en[0][k] = 0; en[1][k] = 0; }
    for (int i = tid; i < Np; i += T) {
      const int i0 = i % n, i1 = (i / n) % n, i2 = i / (n * n);
      const int sh = max(i0, max(i1, i2));
      const int ti = TI::node(i);
      const Real q0 = sq[ti], q1 = sq[PS + ti];
#pragma unroll
      for (int k = 0; k < n; ++k)
        if (k == sh) { en[0][k] += q0 * q0; en[1][k] += q1 * q1; }
    }
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const Real s = warp_sum(en[f][k]);
        if (lane == 0) spart[wid * nin + f * n + k] = s;
      }
    __syncthreads();
    if (tid < nin) {
      Real s = 0;
      for (int w = 0; w < NW; ++w) s += spart[w * nin + tid];
      const Real x = log10(s + Real(1e-30));
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
      const __nv_bfloat16 *W1 = c.W, *b1 = W1 + H * nin, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + 2 * H;
      for (int o = wid; o < H; o += NW) {
        Real z = lane < nin ? (Real)__bfloat162float(W1[o * nin + lane]) * sx[lane] : Real(0);
        z = warp_sum(z);
        if (lane == 0) h1[o] = tanh((Real)__bfloat162float(b1[o]) + z);
      }
      __syncthreads();
      for (int o = wid; o < H; o += NW) {
        const __nv_bfloat162 w2 = reinterpret_cast<const __nv_bfloat162 *>(W2 + o * H)[lane];
        Real z = (Real)__low2float(w2) * h1[2 * lane] + (Real)__high2float(w2) * h1[2 * lane + 1];
        z = warp_sum(z);
        if (lane == 0) h2[o] = tanh((Real)__bfloat162float(b2[o]) + z);
      }
      __syncthreads();
      if (wid < 2) {
        const __nv_bfloat162 w3 = reinterpret_cast<const __nv_bfloat162 *>(W3 + wid * H)[lane];
        Real z = (Real)__low2float(w3) * h2[2 * lane] + (Real)__high2float(w3) * h2[2 * lane + 1];
        z = warp_sum(z);
        if (lane == 0) so[wid] = (Real)__bfloat162float(b3[wid]) + z;
      }
      __syncthreads();
    } else if (tid == 0 && c.n_fallback) {
      atomicAdd(c.n_fallback, 1);
    }
    if (tid < n) {
      Real sig = c.fixed_sigma[tid];
      if (use_net) {
        const Real gam = Real(0.5) / (Real(1) + exp(-so[0]));
        const Real kc = Real(2) + Real(n - 4) / (Real(1) + exp(-so[1]));
        sig = Real(1);
        if (tid > kc) {
          const Real r = (Real(tid) - kc) / (Real(n - 1) - kc);
          sig = Real(1) - gam * r * r;
        }
      }
      ssig[tid] = sig;
      if (c.sigma_out) c.sigma_out[(size_t)e * n + tid] = sig;
    }
    if (!c.outputs) return;
    __syncthreads();
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
    Real *sW = sq;                                     // the modal fields are no longer needed
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
      tile_pass3<Real, n, Q, T>(sf, tid, [&](Real (&v)[n]) { filter_rows<Real, n>(v, sM0, sW, r); });
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
    Real s[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) s[a] = 0;
    for (int k = c0; k < c1; ++k) {
      const Real *tc = p.T + p.bnode_slot[k];
#pragma unroll
      for (int a = 0; a < Q; ++a) s[a] += tc[a * EN];
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) s[a] *= minv;
    Real gacc[3];
    node_accel(p, gid, gacc);
    const Real rho = bgk_collide<Real, LAT>(s, p.rho0, p.omega, p.dt, p.half_dt, gacc, p.has_force != 0);
#pragma unroll
    for (int a = 0; a < Q; ++a) p.f0out[(size_t)a * p.G + gid] = s[a];
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
    for (int a = 0; a < Q; ++a) s[a] = p.fin[(size_t)a * p.G + g];
    node_accel(p, g, gacc);
    const Real rho = bgk_collide<Real, LAT>(s, p.rho0, p.omega, p.dt, p.half_dt, gacc, p.has_force != 0);
#pragma unroll
    for (int a = 0; a < Q; ++a) p.f0out[(size_t)a * p.G + g] = s[a];
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

template <typename Real, int LAT, int n, bool AFFINE>
cudaError_t launch_split_t(const KParams<Real> &p, const SplitHost &h, cudaStream_t s) {
  using S = SplitShape<LAT, n>;
  const size_t smem = split_smem_bytes<Real, LAT, n, AFFINE>(p.wall_max);
  auto k = stage_split_kernel<Real, LAT, n, AFFINE>;
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
