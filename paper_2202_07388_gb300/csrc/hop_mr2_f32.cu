// Stencil kernels with binary32 spinor storage, 2 right-hand sides per
// thread (hop_mr.cuh).
#include "hop_mr.cuh"

namespace oq {
cudaError_t launch_hop_mr2_f32(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return mr_dispatch<P_F32, 2>(L, a, s);
}
}  // namespace oq
