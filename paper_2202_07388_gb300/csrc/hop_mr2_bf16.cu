// Stencil kernels with bfloat16 spinor storage, 2 right-hand sides per
// thread (hop_mr.cuh).
#include "hop_mr.cuh"

namespace oq {
cudaError_t launch_hop_mr2_bf16(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return mr_dispatch<P_BF16, 2>(L, a, s);
}
}  // namespace oq
