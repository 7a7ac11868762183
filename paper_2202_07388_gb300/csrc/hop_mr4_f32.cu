// Stencil kernels with binary32 spinor storage, 4 right-hand sides per
// thread (hop_mr.cuh).
#include "hop_mr.cuh"

namespace oq {
cudaError_t launch_hop_mr4_f32(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return mr_dispatch<P_F32, 4>(L, a, s);
}
}  // namespace oq
