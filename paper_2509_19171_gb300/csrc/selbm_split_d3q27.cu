// Instantiations of the population-split stage kernel and the node collision kernels
// for D3Q27 (orders: 5 7).
#include "selbm_split.cuh"

namespace slb {

template <typename Real>
bool split_stage_d3q27(int N, bool affine, const KParams<Real> &p, const SplitHost &h, cudaStream_t s, cudaError_t *err) {
  switch (N) {
    case 5: *err = affine ? launch_split_t<Real, SELBM_D3Q27, 6, true>(p, h, s) : launch_split_t<Real, SELBM_D3Q27, 6, false>(p, h, s); return true;
    case 7:
      // FP32: 9 populations per work item, one warp each (no idle warps); on curved elements
      // three work items per element instead of four also cut the re-reads of the metrics
      if constexpr (std::is_same<Real, float>::value) {
        *err = affine ? launch_split_t<Real, SELBM_D3Q27, 8, true, 9>(p, h, s)
                      : launch_split_t<Real, SELBM_D3Q27, 8, false, 9>(p, h, s);
        return true;
      }
      *err = affine ? launch_split_t<Real, SELBM_D3Q27, 8, true>(p, h, s) : launch_split_t<Real, SELBM_D3Q27, 8, false>(p, h, s);
      return true;
  }
  return false;
}

// which: 0 collision on unique nodes, 1 assembly of learned-filter shares + collision
template <typename Real>
cudaError_t split_collide_d3q27(int which, const KParams<Real> &p, cudaStream_t s) {
  return which == 0 ? launch_collide_nodes_t<Real, SELBM_D3Q27>(p, s) : launch_dss_collide_t<Real, SELBM_D3Q27>(p, s);
}

template bool split_stage_d3q27<float>(int, bool, const KParams<float> &, const SplitHost &, cudaStream_t, cudaError_t *);
template bool split_stage_d3q27<double>(int, bool, const KParams<double> &, const SplitHost &, cudaStream_t, cudaError_t *);
template cudaError_t split_collide_d3q27<float>(int, const KParams<float> &, cudaStream_t);
template cudaError_t split_collide_d3q27<double>(int, const KParams<double> &, cudaStream_t);

}  // namespace slb
