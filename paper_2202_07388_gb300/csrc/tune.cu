// Autotuner for the stencil launch shape: for one (lattice, precision,
// number of right-hand sides) it times every admissible CTA shape
// (bx sites x by right-hand sides, bx a multiple of 32, bx*by <= 256) of the
// full Dw and of both Dhat passes with CUDA events on scratch fields, and
// keeps the fastest shape per mode in the handle.  Later launches of that
// variant (any epilogue) use the chosen shape.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/oq.h"
#include "ctx.h"

using namespace oq;

namespace {

std::vector<std::pair<int, int>> candidates(int nrhs) {
  std::vector<std::pair<int, int>> c;
  const int bxs[] = {32, 64, 128, 256};
  for (int bx : bxs)
    for (int by = 1; by <= 8 && by <= nrhs; ++by) {
      if (bx * by > 256) continue;
      if (nrhs > 1 && by > 1 && nrhs % by != 0 && by != nrhs) continue;
      if (nrhs > 1 && by == 1 && bx < 64) continue;
      c.push_back({bx, by});
    }
  return c;
}

}  // namespace

extern "C" int oq_autotune(oq_handle h, int lat, int prec, int nrhs, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || prec < 0 || prec > 4 || nrhs < 1 || nrhs > 64)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover) return OQ_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t full = 2 * (size_t)spinor_half_bytes(L.g.Vh, prec) * nrhs;
  void *in = nullptr, *out = nullptr;
  int rc = h->workspace(lat, "tune_in", full, &in);
  if (!rc) rc = h->workspace(lat, "tune_out", full, &out);
  if (rc) return rc;
  if (cudaMemsetAsync(in, 0, full, s) != cudaSuccess) return OQ_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return OQ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return OQ_ERR_CUDA;
  }
  const size_t half = full / 2 / nrhs;
  const int modes[] = {HOP_DW, HOP_P1, HOP_P2};
  int ret = OQ_OK;
  for (int mode : modes) {
    HopArgs a = h->hop_args(lat, prec);
    a.nrhs = nrhs;
    a.in = in;
    a.in2 = in;
    a.out = out;
    a.p = mode == HOP_P1 ? 1 : 0;
    if (mode == HOP_DW) {
      a.in_stride = a.in2_stride = a.out_stride = (long)(2 * half);
      a.half_bytes = (long)half;
    } else {
      a.in_stride = a.in2_stride = a.out_stride = (long)half;
      a.half_bytes = (long)half;
    }
    float best = 1e30f;
    std::pair<int, int> best_shape{128, 1};
    int best_fmt = L.link_fmt;
    // binary32 kernels may also read the 18-real copy of 12-real links
    const bool two_fmts = prec != P_F64 && prec != P_DF64 && L.link_fmt == LINK_12 && L.u32_18.p;
    for (int fmt = L.link_fmt; fmt >= 0; fmt = (two_fmts && fmt == LINK_12) ? LINK_18 : -1) {
      for (auto c : candidates(nrhs)) {
        HopLaunch l = h->hop_launch(lat, prec, mode, 0, EPI_NONE, nrhs);
        l.bx = c.first;
        l.by = c.second;
        l.link_fmt = fmt;
        const HopArgs b = h->with_links(l, a);
        for (int w = 0; w < 2; ++w)
          if (launch_hop(l, b, s) != cudaSuccess) ret = OQ_ERR_CUDA;
        const int reps = 5;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r)
          if (launch_hop(l, b, s) != cudaSuccess) ret = OQ_ERR_CUDA;
        cudaEventRecord(e1, s);
        h->launches += 2 + reps;
        if (cudaEventSynchronize(e1) != cudaSuccess) ret = OQ_ERR_CUDA;
        if (ret) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best) {
          best = ms;
          best_shape = c;
          best_fmt = fmt;
        }
      }
      if (ret) break;
    }
    if (ret) break;
    h->tuned[TuneKey{lat, prec, mode, nrhs}] = best_shape;
    h->tuned_ms[TuneKey{lat, prec, mode, nrhs}] = best;
    h->tuned_fmt[TuneKey{lat, prec, mode, nrhs}] = best_fmt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ret;
}

extern "C" int oq_tune_get(oq_handle h, int lat, int prec, int mode, int nrhs, int* bx, int* by, float* ms,
                           int* link_fmt) {
  if (!h || !bx || !by || !ms || lat < 0 || lat >= (int)h->lats.size()) return OQ_ERR_ARG;
  auto it = h->tuned.find(TuneKey{lat, prec, mode, nrhs});
  if (it == h->tuned.end()) return OQ_ERR_STATE;
  *bx = it->second.first;
  *by = it->second.second;
  *ms = h->tuned_ms[TuneKey{lat, prec, mode, nrhs}];
  if (link_fmt) *link_fmt = h->tuned_fmt[TuneKey{lat, prec, mode, nrhs}];
  return OQ_OK;
}
