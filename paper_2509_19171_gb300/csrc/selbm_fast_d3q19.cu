// Instantiations of the register-blocked stage kernel for D3Q19 (orders: 4 7).
#include "selbm_fast.cuh"

namespace slb {

template <typename Real>
bool launch_fast_d3q19(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 4: *err = affine ? launch_fast_t<Real, SELBM_D3Q19, 5, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D3Q19, 5, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
    case 7: *err = affine ? launch_fast_t<Real, SELBM_D3Q19, 8, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D3Q19, 8, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
  }
  return false;
}

template bool launch_fast_d3q19<float>(int, bool, const KParams<float> &, const FastHost &, cudaStream_t, cudaError_t *);
template bool launch_fast_d3q19<double>(int, bool, const KParams<double> &, const FastHost &, cudaStream_t, cudaError_t *);

}  // namespace slb
