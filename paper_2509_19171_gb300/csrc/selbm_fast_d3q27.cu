// Instantiations of the register-blocked stage kernel for D3Q27 (orders: 5 7).
#include "selbm_fast.cuh"

namespace slb {

template <typename Real>
bool launch_fast_d3q27(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 5: *err = affine ? launch_fast_t<Real, SELBM_D3Q27, 6, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D3Q27, 6, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
    case 7: *err = affine ? launch_fast_t<Real, SELBM_D3Q27, 8, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D3Q27, 8, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
  }
  return false;
}

template bool launch_fast_d3q27<float>(int, bool, const KParams<float> &, const FastHost &, cudaStream_t, cudaError_t *);
template bool launch_fast_d3q27<double>(int, bool, const KParams<double> &, const FastHost &, cudaStream_t, cudaError_t *);

}  // namespace slb
