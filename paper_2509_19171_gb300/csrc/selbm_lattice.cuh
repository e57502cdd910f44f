// Compile-time velocity sets (same ordering rule as slb::build_lattice: speed
// class, then ternary code ascending).  Used by the kernels so that velocity
// components are literal constants and multiplications by 0 / +-1 fold away.
#pragma once
#include <type_traits>

#include "../../include/selbm.h"

namespace slb {

struct VelTab {
  int e[27][3];
  double t[27];
  int opp[27];
  int Q;
  int D;
};

constexpr VelTab make_veltab(int lat) {
  VelTab v{};
  const int dim = lat == SELBM_D2Q9 ? 2 : 3;
  double wc[4] = {0, 0, 0, 0};
  if (lat == SELBM_D2Q9) { wc[0] = 4.0 / 9.0; wc[1] = 1.0 / 9.0; wc[2] = 1.0 / 36.0; }
  else if (lat == SELBM_D3Q19) { wc[0] = 1.0 / 3.0; wc[1] = 1.0 / 18.0; wc[2] = 1.0 / 36.0; }
  else { wc[0] = 8.0 / 27.0; wc[1] = 2.0 / 27.0; wc[2] = 1.0 / 54.0; wc[3] = 1.0 / 216.0; }
  const int ncode = dim == 2 ? 9 : 27;
  int q = 0;
  for (int cls = 0; cls <= dim; ++cls) {
    if (wc[cls] == 0.0) continue;
    for (int code = 0; code < ncode; ++code) {
      const int c0 = code % 3 - 1, c1 = (code / 3) % 3 - 1, c2 = dim == 3 ? code / 9 - 1 : 0;
      if (c0 * c0 + c1 * c1 + c2 * c2 != cls) continue;
      v.e[q][0] = c0; v.e[q][1] = c1; v.e[q][2] = c2;
      v.t[q] = wc[cls];
      ++q;
    }
  }
  v.Q = q;
  v.D = dim;
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b)
      if (v.e[b][0] == -v.e[a][0] && v.e[b][1] == -v.e[a][1] && v.e[b][2] == -v.e[a][2]) v.opp[a] = b;
  return v;
}

template <int LAT>
struct LT {
  static constexpr VelTab v = make_veltab(LAT);
};

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

}  // namespace slb
