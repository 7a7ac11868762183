// Stencil kernels with bf16 spinor storage, binary32 arithmetic and binary32
// links (18 or 12 reals) and clover blocks.
#include "hop_impl.cuh"

namespace oq {
cudaError_t launch_hop_bf16(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return L.link_fmt == LINK_12 ? dispatch_dag<P_BF16, LINK_12>(L, a, s) : dispatch_dag<P_BF16, LINK_18>(L, a, s);
}
}  // namespace oq
