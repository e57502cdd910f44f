// Instantiations of the register-blocked stage kernel for D2Q9 (orders: 4 8).
#include "selbm_fast.cuh"

namespace slb {

template <typename Real>
bool launch_fast_d2q9(int N, bool affine, const KParams<Real> &p, const FastHost &f, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 4: *err = affine ? launch_fast_t<Real, SELBM_D2Q9, 5, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D2Q9, 5, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
    case 8: *err = affine ? launch_fast_t<Real, SELBM_D2Q9, 9, true>(p, f.D, f.U, f.W, f.r, f.w, s) : launch_fast_t<Real, SELBM_D2Q9, 9, false>(p, f.D, f.U, f.W, f.r, f.w, s); return true;
  }
  return false;
}

template bool launch_fast_d2q9<float>(int, bool, const KParams<float> &, const FastHost &, cudaStream_t, cudaError_t *);
template bool launch_fast_d2q9<double>(int, bool, const KParams<double> &, const FastHost &, cudaStream_t, cudaError_t *);

}  // namespace slb
