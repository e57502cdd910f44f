// Instantiations of the per-element prologue (pending filter + collision) for
// D3Q27 (orders: 5 7).
#include "selbm_split.cuh"

namespace slb {

template <typename Real, int n>
static cudaError_t prologue_n(bool affine, int mode, const KParams<Real> &p, const SplitHost &h,
                              const LearnedPtrs<Real> &lp, cudaStream_t s) {
  if (mode == PRO_LEARNED)
    return affine ? launch_prologue_t<Real, SELBM_D3Q27, n, true, PRO_LEARNED>(p, h, lp, s)
                  : launch_prologue_t<Real, SELBM_D3Q27, n, false, PRO_LEARNED>(p, h, lp, s);
  return affine ? launch_prologue_t<Real, SELBM_D3Q27, n, true, PRO_FIXED>(p, h, lp, s)
                : launch_prologue_t<Real, SELBM_D3Q27, n, false, PRO_FIXED>(p, h, lp, s);
}

template <typename Real>
bool split_prologue_d3q27(int N, bool affine, int mode, const KParams<Real> &p, const SplitHost &h,
                         const LearnedPtrs<Real> &lp, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 5: *err = prologue_n<Real, 6>(affine, mode, p, h, lp, s); return true;
    case 7: *err = prologue_n<Real, 8>(affine, mode, p, h, lp, s); return true;
  }
  return false;
}

template bool split_prologue_d3q27<float>(int, bool, int, const KParams<float> &, const SplitHost &,
                                         const LearnedPtrs<float> &, cudaStream_t, cudaError_t *);
template bool split_prologue_d3q27<double>(int, bool, int, const KParams<double> &, const SplitHost &,
                                          const LearnedPtrs<double> &, cudaStream_t, cudaError_t *);

// learned control of the split form (node features, element network) -> lp.sigma_out
template <typename Real>
bool split_control_d3q27(int N, const KParams<Real> &p, const SplitHost &h, const LearnedPtrs<Real> &lp, Real *q,
                        Real *X, const double *mass, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 5: *err = launch_split_control_t<Real, SELBM_D3Q27, 6>(p, h, lp, q, X, mass, s); return true;
    case 7: *err = launch_split_control_t<Real, SELBM_D3Q27, 8>(p, h, lp, q, X, mass, s); return true;
  }
  return false;
}
template bool split_control_d3q27<float>(int, const KParams<float> &, const SplitHost &, const LearnedPtrs<float> &,
                                        float *, float *, const double *, cudaStream_t, cudaError_t *);
template bool split_control_d3q27<double>(int, const KParams<double> &, const SplitHost &, const LearnedPtrs<double> &,
                                         double *, double *, const double *, cudaStream_t, cudaError_t *);

}  // namespace slb
