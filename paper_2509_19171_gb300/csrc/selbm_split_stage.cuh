// Advection stage of the population-split step for hexahedral meshes: one CTA per
// (element, group of PB populations) gathers the group's f^{s-1} tile (and f^0 of
// element-interior nodes), forms -B dt e.grad f by sum factorisation with the flux
// bounce-back wall terms (Sec. 2.2, 2.2.1), and writes the stage combination of
// element-interior nodes to f^s and the weighted boundary shares to the assembly trace.
#pragma once
#include <cuda_runtime.h>

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

template <int LAT, int n, int PBW = 0>
struct SplitShape {
  static constexpr int Q = LT<LAT>::v.Q;
  static constexpr int Np = n * n * n, NL = n * n;
  static constexpr int LPR = 256 / NL < 1 ? 1 : 256 / NL;         // populations per round of tasks
  // PBW > 0 (swizzled FP32 tile, one warp per population): PBW populations per work item
  static constexpr int THREADS = PBW > 0 ? 32 * PBW : LPR * NL;   // one (population, r-line) task per round
  static constexpr int ROUNDS = 2;
  static constexpr int PB = PBW > 0 ? PBW : ROUNDS * LPR;         // populations per work item
  static constexpr int NG = (Q + PB - 1) / PB;                    // work items per element
  static constexpr int NPT = (Np + THREADS - 1) / THREADS;        // nodes per thread when gathering
};

// offset (in values) of the curved-element metric planes: 16-byte aligned, since the passes read
// them with 8- and 16-byte vector loads
template <typename Real, int LAT, int n, int PBW = 0>
constexpr size_t split_sg_offset() {
  using S = SplitShape<LAT, n, PBW>;
  using TI = Tile<Real, n, 3>;
  constexpr size_t V16 = 16 / sizeof(Real);
  return (2 * (size_t)S::PB * TI::PS + n * n + S::PB * 3 + 2 * S::PB + n + V16 - 1) / V16 * V16;
}

template <typename Real, int LAT, int n, bool AFFINE, int PBW = 0>
constexpr size_t split_smem_bytes(int wall_max) {
  using S = SplitShape<LAT, n, PBW>;
  size_t reals = split_sg_offset<Real, LAT, n, PBW>();
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
template <typename Real, int LAT, int n, bool AFFINE, int PBW = 0>
__global__ void __launch_bounds__(SplitShape<LAT, n, PBW>::THREADS, (sizeof(Real) == 4 ? (AFFINE ? (PBW > 9 ? 4 : 5) : (PBW > 0 ? 3 : 4)) : 2))
stage_split_kernel(const KParams<Real> p, const FastMats<Real, n> m) {
  using S = SplitShape<LAT, n, PBW>;
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
  Real *sg = sf + split_sg_offset<Real, LAT, n, PBW>();   // curved: dr_l/dx_k [Np][9], wJ [Np]
  static_assert(split_sg_offset<Real, LAT, n, PBW>() * sizeof(Real) % 16 == 0, "metric planes 16-byte aligned");
  Real *wbuf = sg + (AFFINE ? 0 : Np * 10);         // [wall nodes][PB]
  const int e = blockIdx.x / NG, a0 = (blockIdx.x - e * NG) * PB;
  const int na = Q - a0 < PB ? Q - a0 : PB;
  const bool full = na == PB;
  const int tid = threadIdx.x;
  const Real Bdt = p.B * p.dt;
  const int32_t *l2g = p.l2g + (size_t)e * Np;
  const size_t G = p.Gs;                            // population stride of the state
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
      const Real *wj = p.wJ + (size_t)e * Np;
      if constexpr (TI::SW) {
        // swizzled FP32 tile: metric component c of node i at c PS + node(i), wJ at 9 PS +
        // node(i), so that the passes read them like the tile
        for (int idx = tid; idx < Np * 9; idx += T) {
          const int i = idx / 9, c = idx - i * 9;
          cp_async_s<Real>(s_g + (c * PS + TI::node(i)) * RS, gm + idx);
        }
        for (int i = tid; i < Np; i += T) cp_async_s<Real>(s_g + (9 * PS + TI::node(i)) * RS, wj + i);
      } else {
        for (int c = tid; c < Np * 9; c += T) cp_async_s<Real>(s_g + c * RS, gm + c);
        for (int c = tid; c < Np; c += T) cp_async_s<Real>(s_g + (Np * 9 + c) * RS, wj + c);
      }
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
  if constexpr (TI::SW) {
    // swizzled FP32 tile (N = 7): one warp per population, one axis per pass.  A pass
    // takes two adjacent lines along its axis into registers (8-byte loads, conflict-free
    // on the swizzled tile), applies D and adds c_l (D f) into the population's slice of so,
    // whose element-interior nodes start as A f^0; the r-pass adds the r-derivative and
    // finishes the stage combination.  Every tile value is read once per axis.  On curved
    // elements c_l = -B dt sum_k e_k dr_l/dx_k is read per node from the metric planes.
    const int pl = tid >> 5, lane = tid & 31;
    const int x = lane & 7, y = lane >> 3;                    // lines (x, y) and (x, y + 4)
    if (pl < na) {
      const Real *fa = sf + pl * PS;
      Real *oa = so + pl * PS;
      Real c0 = 1, c1 = 1, c2 = 1;                            // curved: any non-zero marker
      Real eb[3] = {0, 0, 0};                                 // curved: -B dt e_k
      if constexpr (AFFINE) {
        c0 = cf[pl * DIM + 0];
        c1 = cf[pl * DIM + 1];
        c2 = cf[pl * DIM + 2];
      } else {
        const int a = a0 + pl;
#pragma unroll
        for (int k = 0; k < 3; ++k) eb[k] = -Bdt * mask_sign<Real>(POS[k], NEG[k], a);
      }
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
        // D_hat along the axis for both lines at once, in the even-odd form (see deriv_line)
        constexpr int H = n / 2;
        float2 ev[H], od[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const float2 lo = *reinterpret_cast<const float2 *>(fa + (AX == 1 ? TI::at(xp, k, o) : TI::at(xp, o, k)));
          const float2 hi =
              *reinterpret_cast<const float2 *>(fa + (AX == 1 ? TI::at(xp, n - 1 - k, o) : TI::at(xp, o, n - 1 - k)));
          ev[k] = __fadd2_rn(lo, hi);
          od[k] = __fadd2_rn(lo, make_float2(-hi.x, -hi.y));
        }
        float2 d[n];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const float P0 = m.PM[j * H * 2], M0 = m.PM[j * H * 2 + 1];
          float2 sp = __fmul2_rn(make_float2(P0, P0), ev[0]), sm = __fmul2_rn(make_float2(M0, M0), od[0]);
#pragma unroll
          for (int k = 1; k < H; ++k) {
            const float P = m.PM[(j * H + k) * 2], M = m.PM[(j * H + k) * 2 + 1];
            sp = __ffma2_rn(make_float2(P, P), ev[k], sp);
            sm = __ffma2_rn(make_float2(M, M), od[k], sm);
          }
          d[j] = __fadd2_rn(sp, sm);
          d[n - 1 - j] = __fadd2_rn(sm, make_float2(-sp.x, -sp.y));
        }
        const float2 cc = make_float2(c, c);
#pragma unroll
        for (int j = 0; j < n; ++j) {
          const int off = AX == 1 ? TI::at(xp, j, o) : TI::at(xp, o, j);
          float2 *dst = reinterpret_cast<float2 *>(oa + off);
          const float2 old = *dst;
          float2 r;
          if constexpr (AFFINE) {
            r = __fmul2_rn(cc, d[j]);
          } else {
            // per-node coefficients of the pair: metric planes dr_AX/dx_k
            float2 cn = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (eb[k] != Real(0))
                cn = __ffma2_rn(make_float2(eb[k], eb[k]), *reinterpret_cast<const float2 *>(sg + (AX * 3 + k) * PS + off), cn);
            r = __fmul2_rn(cn, d[j]);
          }
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
      const Real Jwx = AFFINE ? p.el_J[e] * sw[x] : Real(0);
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
        Real cr[n];                                           // r-coefficient per node
#pragma unroll
        for (int j = 0; j < n; ++j) cr[j] = c0;
        if constexpr (!AFFINE) {
#pragma unroll
          for (int j = 0; j < n; ++j) cr[j] = 0;
#pragma unroll
          for (int k = 0; k < 3; ++k)
            if (eb[k] != Real(0)) {
              Real mk[n];
              load_line<Real, n>(sg + k * PS + own, swz, mk);
#pragma unroll
              for (int j = 0; j < n; ++j) cr[j] += eb[k] * mk[j];
            }
        }
        if (c0 != Real(0)) {
          Real d[n];
          deriv_line<Real, n>(m, v, d);
#pragma unroll
          for (int j = 0; j < n; ++j) acc[j] += cr[j] * d[j];
        }
        Real wl[n];                                           // wJ of the line's nodes
        if constexpr (AFFINE) {
#pragma unroll
          for (int j = 0; j < n; ++j) wl[j] = Jwx * sw[o] * m.w[j];
        } else {
          load_line<Real, n>(sg + 9 * PS + own, swz, wl);
        }
        Real res[n];
        if (!lin) {
#pragma unroll
          for (int j = 0; j < n; ++j) res[j] = wl[j] * acc[j];
        } else {
          res[0] = wl[0] * acc[0];
          res[n - 1] = wl[n - 1] * acc[n - 1];
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
          Real d[n];
          deriv_line<Real, n>(m, v, d);
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] = c0 * d[j];
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
        {
          Real d[n];
          deriv_line<Real, n>(m, v, d);
#pragma unroll
          for (int j = 0; j < n; ++j) adv[j] = coef(j, 0) * d[j];
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
            const size_t GN = p.G;                   // the field is per node: [3][G]
            const Real sx[3] = {A * p.fS[g], A * p.fS[GN + g], A * p.fS[2 * GN + g]};
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

}  // namespace slb
