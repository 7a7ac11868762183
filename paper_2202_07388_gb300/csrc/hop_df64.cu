// Stencil kernels with binary64 storage and double-float arithmetic on the
// binary32 pipes (reset-step residuals; binary64 links and clover blocks).
#include "hop_impl.cuh"

namespace oq {
cudaError_t launch_hop_df64(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return dispatch_dag<P_DF64, LINK_18>(L, a, s);
}
}  // namespace oq
