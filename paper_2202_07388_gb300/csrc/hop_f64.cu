// Stencil kernels with binary64 spinors, links and clover blocks (reset
// steps and the plain binary64 baseline solver).
#include "hop_impl.cuh"

namespace oq {
cudaError_t launch_hop_f64(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return dispatch_dag<P_F64, LINK_18>(L, a, s);
}
}  // namespace oq
