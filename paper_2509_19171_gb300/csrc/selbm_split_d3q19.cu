// Instantiations of the population-split stage kernel and the node collision kernels
// for D3Q19 (orders: 4 7).
#include "selbm_split.cuh"

namespace slb {

template <typename Real>
bool split_stage_d3q19(int N, bool affine, const KParams<Real> &p, const SplitHost &h, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 4: *err = affine ? launch_split_t<Real, SELBM_D3Q19, 5, true>(p, h, s) : launch_split_t<Real, SELBM_D3Q19, 5, false>(p, h, s); return true;
    case 7:
      // FP32: 10 populations per work item, one warp each (no idle warps); on curved elements
      // two work items per element also halve the re-reads of the per-node metrics
      if constexpr (std::is_same<Real, float>::value) {
        *err = affine ? launch_split_t<Real, SELBM_D3Q19, 8, true, 10>(p, h, s)
                      : launch_split_t<Real, SELBM_D3Q19, 8, false, 10>(p, h, s);
        return true;
      }
      *err = affine ? launch_split_t<Real, SELBM_D3Q19, 8, true>(p, h, s) : launch_split_t<Real, SELBM_D3Q19, 8, false>(p, h, s);
      return true;
  }
  return false;
}

// which: 0 collision on unique nodes, 1 assembly of learned-filter shares + collision
template <typename Real>
cudaError_t split_collide_d3q19(int which, const KParams<Real> &p, cudaStream_t s) {
  return which == 0 ? launch_collide_nodes_t<Real, SELBM_D3Q19>(p, s) : launch_dss_collide_t<Real, SELBM_D3Q19>(p, s);
}

template bool split_stage_d3q19<float>(int, bool, const KParams<float> &, const SplitHost &, cudaStream_t, cudaError_t *);
template bool split_stage_d3q19<double>(int, bool, const KParams<double> &, const SplitHost &, cudaStream_t, cudaError_t *);
template cudaError_t split_collide_d3q19<float>(int, const KParams<float> &, cudaStream_t);
template cudaError_t split_collide_d3q19<double>(int, const KParams<double> &, cudaStream_t);

}  // namespace slb
