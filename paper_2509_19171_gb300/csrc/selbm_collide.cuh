// Node-local pieces shared by the element kernels: BGK collision with the split
// forcing in the deviation form, and a warp sum.
#pragma once
#include "selbm_lattice.cuh"

namespace slb {

// BGK collision with F** at one node (Sec. 2.1), deviation form: on entry g[a] holds
// f_bar_a - t_a rho0, on exit f*_a - t_a rho0.  Returns rho.
//   f_bar^eq = f^eq(rho, u) - dt/2 F**(u),   f* = f_bar - omega (f_bar - f_bar^eq) + dt F**,
//   F**_a = t_a (9 (e_a.u)(e_a.F) - 3 u.F),  F = rho g,  cs^2 = 1/3.
template <typename Real, int LAT>
__device__ __forceinline__ Real bgk_collide(Real (&g)[LT<LAT>::v.Q], Real rho0, Real omega, Real dt, Real half_dt,
                                            const Real (&gacc)[3], bool has_force) {
  constexpr VelTab V = LT<LAT>::v;
  constexpr int Q = V.Q, DIM = V.D;
  Real drho = 0, j[3] = {0, 0, 0};
  static_for<0, Q>([&](auto ac) {
    constexpr int a = decltype(ac)::value;
    const Real fa = g[a];
    drho += fa;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      if (V.e[a][k] > 0) j[k] += fa;
      else if (V.e[a][k] < 0) j[k] -= fa;
    }
  });
  const Real rho = rho0 + drho;
  const Real inv = Real(1) / rho;
  Real u[3] = {0, 0, 0}, F[3] = {0, 0, 0}, uu = 0, uF = 0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    u[k] = j[k] * inv;
    uu += u[k] * u[k];
    if (has_force) { F[k] = rho * gacc[k]; uF += u[k] * F[k]; }
  }
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
    if (has_force) {
      Fss = t * (Real(9) * eu * eF - Real(3) * uF);
      feq -= half_dt * Fss;
    }
    const Real fa = g[a];
    g[a] = fa - omega * (fa - feq) + dt * Fss;
  });
  return rho;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace slb
