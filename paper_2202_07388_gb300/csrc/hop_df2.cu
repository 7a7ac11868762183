// Double-float stencil kernels, 2 right-hand sides per thread (hop_df2.cuh).
#include "hop_df2.cuh"

namespace oq {
// (the links are the double-float split of the binary64 links, whatever
// format the gauge field was uploaded in, as for the one-rhs kernel)
cudaError_t launch_hop_df2(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return L.dagger ? df2_dispatch_mode_epi<true>(L, a, s) : df2_dispatch_mode_epi<false>(L, a, s);
}
}  // namespace oq
