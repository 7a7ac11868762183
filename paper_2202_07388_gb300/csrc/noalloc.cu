// oq_dw_hat_apply_noalloc: the even-odd operator Dhat (or Dhat^dag) with its
// odd-site intermediate in a fixed, file-scope device array instead of
// handle-owned memory, so that the call itself never allocates.
//
// The array is a static __device__ symbol: every GPU that loads the library
// holds OQ_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code
// cannot use the symbol's name as a device address (it names a host-side
// shadow), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made
// while that device is current.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/oq.h"
#include "ctx.h"

using namespace oq;

static __device__ __align__(256) unsigned char g_dwhat_noalloc_t[OQ_NOALLOC_SCRATCH_BYTES];

namespace {
const int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of the static scratch on the current device (looked up once)
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OQ_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return OQ_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dwhat_noalloc_t) != cudaSuccess || !p) return OQ_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return OQ_OK;
}
}  // namespace

extern "C" int oq_dw_hat_apply_noalloc(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs,
                                       int dagger, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !in_dev || !out_dev || prec < 0 || prec > 3 || nrhs < 1)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  // the scratch address is per device: only the handle's device may be current
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return OQ_ERR_CUDA;
  if (cur != h->device) return OQ_ERR_STATE;
  const size_t half = (size_t)spinor_half_bytes(L.g.Vh, prec);
  if (half * (size_t)nrhs > (size_t)OQ_NOALLOC_SCRATCH_BYTES) return OQ_ERR_ARG;  // does not fit the fixed scratch
  const char* a0 = (const char*)in_dev;
  const char* b0 = (const char*)out_dev;
  if (a0 < b0 + half * nrhs && b0 < a0 + half * nrhs) return OQ_ERR_ARG;
  void* t = nullptr;
  int rc = scratch_address(&t);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  HopArgs a = h->hop_args(lat, prec);
  a.nrhs = nrhs;
  a.in_stride = a.in2_stride = a.out_stride = (long)half;
  a.half_bytes = (long)half;
  // pass 1: t_o = A_oo^{-1} (-1/2 H_oe in_e), into the static scratch
  a.in = in_dev;
  a.out = t;
  a.p = 1;
  rc = h->run_hop(h->hop_launch(lat, prec, HOP_P1, dagger ? 1 : 0, EPI_NONE, nrhs), a, s);
  if (rc) return rc;
  // pass 2: out_e = A_ee in_e + 1/2 H_eo t_o
  a.in = t;
  a.in2 = in_dev;
  a.out = out_dev;
  a.p = 0;
  return h->run_hop(h->hop_launch(lat, prec, HOP_P2, dagger ? 1 : 0, EPI_NONE, nrhs), a, s);
}
