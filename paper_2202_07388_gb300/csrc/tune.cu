// Autotuner for the stencil launch shape: for one (lattice, precision,
// number of right-hand sides) it times every admissible launch of the full
// Dw and of both Dhat passes with CUDA events on scratch fields: CTA shapes
// (bx sites x by rows, bx a multiple of 32), one or several (2, 4)
// right-hand sides per thread with or without a register cap, and both
// binary32 link formats when the handle holds both.  The fastest launch per
// mode is kept in the handle and used by every later launch of that mode;
// pass 2 is also timed with its norm and CG-update epilogues (on scratch
// operands: alpha = 0, reductions only stored), which keep their own choice.
// oq_tune_set pins a launch by hand for every epilogue of a mode.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/oq.h"
#include "ctx.h"

using namespace oq;

namespace {

// Scratch fields for timing: a fixed pseudo-random pattern of values in
// [-1, 1) in the storage type (element k from an integer hash of k), so that
// the launches are timed on data like a solver's rather than on zeros.
// Double-float elements are (hi, 0) pairs.
__global__ void tune_fill_kernel(void* p, size_t n, int prec) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)k * 2654435761u ^ (uint32_t)(k >> 32) * 2246822519u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float v = (float)(int32_t)h * (1.f / 2147483648.f);
    switch (prec) {
      case P_F64: static_cast<double*>(p)[k] = (double)v; break;
      case P_F32: static_cast<float*>(p)[k] = v; break;
      case P_BF16: static_cast<__nv_bfloat16*>(p)[k] = __float2bfloat16_rn(v); break;
      case P_F16: static_cast<__half*>(p)[k] = __float2half_rn(v); break;
      default: static_cast<float2*>(p)[k] = make_float2(v, 0.f); break;  // double-float
    }
  }
}
cudaError_t tune_fill(void* p, size_t bytes, int prec, cudaStream_t s) {
  const size_t esize = (prec == P_F64 || prec == P_DF64) ? 8 : prec == P_F32 ? 4 : 2;
  const size_t n = bytes / esize;
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  tune_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, n, prec);
  return cudaGetLastError();
}

std::vector<TuneVal> candidates(int prec, int nrhs) {
  std::vector<TuneVal> c;
  const int bxs[] = {32, 64, 128, 256};
  for (int bx : bxs)
    for (int by = 1; by <= 8 && by <= nrhs; ++by) {
      if (bx * by > 256) continue;
      if (nrhs > 1 && by > 1 && nrhs % by != 0 && by != nrhs) continue;
      if (nrhs > 1 && by == 1 && bx < 64) continue;
      TuneVal v;
      v.bx = bx;
      v.by = by;
      c.push_back(v);
    }
  // double-float: the register-capped kernel (<= 128 threads per CTA)
  if (prec == P_DF64) {
    const size_t n0 = c.size();
    for (size_t k = 0; k < n0; ++k)
      if (c[k].bx * c[k].by <= 128)
        for (int cap = 1; cap <= 2; ++cap) {
          TuneVal v = c[k];
          v.regcap = cap;
          c.push_back(v);
        }
  }
  // double-float, two right-hand sides per thread (packed two-lane arithmetic)
  if (prec == P_DF64 && nrhs >= 2) {
    const int bxs2[] = {32, 64, 128};
    for (int cap = 0; cap < 2; ++cap)
      for (int bx : bxs2)
        for (int by = 1; by <= 2; ++by) {
          if (bx * by > 128 || 2 * by > nrhs) continue;
          TuneVal v;
          v.bx = bx;
          v.by = by;
          v.nr = 2;
          v.regcap = cap;
          c.push_back(v);
        }
  }
  // several right-hand sides per thread (binary32 arithmetic types)
  if (prec == P_F32 || prec == P_BF16 || prec == P_F16) {
    const int nrs[] = {2, 4};
    for (int nr : nrs) {
      if (nr > nrhs) continue;
      for (int cap = 0; cap < (nr == 2 ? 4 : 3); ++cap)
        for (int bx : bxs)
          for (int by = 1; by <= 2; ++by) {
            if (bx * by > 128 || by * nr > nrhs) continue;
            TuneVal v;
            v.bx = bx;
            v.by = by;
            v.nr = nr;
            v.regcap = cap;
            c.push_back(v);
          }
    }
  }
  return c;
}

bool valid_shape(const LatCtx& L, int prec, int nrhs, const TuneVal& v) {
  if (v.bx < 32 || v.bx % 32 != 0 || v.by < 1 || v.by > nrhs) return false;
  if (v.nr == 1) {
    if (v.bx * v.by > 256) return false;
    if (v.regcap != 0 && !(prec == P_DF64 && (v.regcap == 1 || v.regcap == 2) && v.bx * v.by <= 128))
      return false;
  } else if (v.nr == 2 && prec == P_DF64) {
    // two rhs per thread in packed double-float: <= 128 threads, regcap 0 / 1
    if (v.bx * v.by > 128 || 2 * v.by > nrhs || v.regcap < 0 || v.regcap > 1) return false;
  } else if (v.nr == 2 || v.nr == 4) {
    if (prec != P_F32 && prec != P_BF16 && prec != P_F16) return false;
    if (v.bx * v.by > 128 || v.regcap < 0 || v.regcap > 3 || (v.regcap == 3 && v.nr != 2)) return false;
    // staged hops (regcap 2, 3) read 12-real links
    if (v.regcap >= 2 && (v.link_fmt == LINK_18 || (v.link_fmt == -1 && L.link_fmt != LINK_12))) return false;
  } else {
    return false;
  }
  if (v.link_fmt != -1) {
    if (prec == P_F64 || prec == P_DF64) return false;
    if (v.link_fmt == LINK_12 && L.link_fmt != LINK_12) return false;
    if (v.link_fmt == LINK_18 && L.link_fmt == LINK_12 && !L.u32_18.p) return false;
    if (v.link_fmt != LINK_12 && v.link_fmt != LINK_18) return false;
  }
  return true;
}

}  // namespace

extern "C" int oq_autotune(oq_handle h, int lat, int prec, int nrhs, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || prec < 0 || prec > 4 || nrhs < 1 || nrhs > 64)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == P_DF64) {
    const int rc = h->ensure_df(lat, s);
    if (rc) return rc;
  }
  const size_t full = 2 * (size_t)spinor_half_bytes(L.g.Vh, prec) * nrhs;
  void *in = nullptr, *out = nullptr;
  int rc = h->workspace(lat, "tune_in", full, &in);
  if (!rc) rc = h->workspace(lat, "tune_out", full, &out);
  if (rc) return rc;
  if (tune_fill(in, full, prec, s) != cudaSuccess || tune_fill(out, full, prec, s) != cudaSuccess)
    return OQ_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return OQ_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return OQ_ERR_CUDA;
  }
  const size_t half = full / 2 / nrhs;
  int ret = OQ_OK;
  // scratch for the epilogue variants of pass 2: the CG update reads a state
  // with alpha = 0 (x and r do not change) and every reduction only stores
  const int XP = prec == P_F64 ? P_F64 : P_F32;
  void *xs = nullptr, *rs = nullptr, *cgs = nullptr;
  const bool epis = prec != P_DF64;
  if (epis) {
    rc = h->workspace(lat, "tune_x", (size_t)spinor_half_bytes(L.g.Vh, XP) * nrhs, &xs);
    if (!rc) rc = h->workspace(lat, "tune_r", half * nrhs, &rs);
    if (!rc) rc = h->workspace(lat, "tune_cg", sizeof(CgState) * nrhs, &cgs);
    if (!rc) rc = h->ensure_reduce(2 * nrhs, (L.g.Vh + 31) / 32);
    if (rc) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
    if (tune_fill(xs, (size_t)spinor_half_bytes(L.g.Vh, XP) * nrhs, XP, s) != cudaSuccess ||
        tune_fill(rs, half * nrhs, prec, s) != cudaSuccess ||
        cudaMemsetAsync(cgs, 0, sizeof(CgState) * nrhs, s) != cudaSuccess)  // mode RUN, alpha 0
      ret = OQ_ERR_CUDA;
  }
  struct Variant {
    int mode, epi;
  };
  std::vector<Variant> variants = {{HOP_DW, EPI_NONE}, {HOP_P1, EPI_NONE}, {HOP_P2, EPI_NONE}};
  if (epis) {
    variants.push_back({HOP_P2, EPI_NORM});
    variants.push_back({HOP_P2, EPI_CG});
  }
  for (const Variant var : variants) {
    if (ret) break;
    const int mode = var.mode;
    HopArgs a = h->hop_args(lat, prec);
    a.nrhs = nrhs;
    // distinct fields as in a solve: pass 2 reads its odd input from the first
    // half of `in` and its even in2 from the second (Dw: in2 is its input)
    a.in = in;
    a.in2 = mode == HOP_P2 ? (void*)((char*)in + half * nrhs) : in;
    a.out = out;
    a.p = mode == HOP_P1 ? 1 : 0;
    if (mode == HOP_DW) {
      a.in_stride = a.in2_stride = a.out_stride = (long)(2 * half);
      a.half_bytes = (long)half;
    } else {
      a.in_stride = a.in2_stride = a.out_stride = (long)half;
      a.half_bytes = (long)half;
    }
    if (var.epi != EPI_NONE) {
      a.red = h->red_args(FIN_STORE, MODE_RUN);
      if (var.epi == EPI_CG) {
        a.out = nullptr;
        a.cg = (CgState*)cgs;
        a.gate = MODE_RUN;
        a.ep_x = xs;
        a.ep_x_stride = (long)spinor_half_bytes(L.g.Vh, XP);
        a.ep_p = out;  // the CG update writes no out: the search direction p
        a.ep_p_stride = (long)half;
        a.ep_r = rs;
        a.ep_r_stride = (long)half;
      }
    }
    TuneVal best;
    best.ms = 1e30f;
    // binary32 kernels may also read the 18-real copy of 12-real links
    const bool two_fmts = prec != P_F64 && prec != P_DF64 && L.link_fmt == LINK_12 && L.u32_18.p;
    for (int fmt = L.link_fmt; fmt >= 0; fmt = (two_fmts && fmt == LINK_12) ? LINK_18 : -1) {
      for (TuneVal c : candidates(prec, nrhs)) {
        if (c.regcap >= 2 && c.nr > 1 && fmt != LINK_12) continue;  // staged hops read 12-real links
        HopLaunch l = h->hop_launch(lat, prec, mode, 0, var.epi, nrhs);
        l.bx = c.bx;
        l.by = c.by;
        l.nr = c.nr;
        l.regcap = c.regcap;
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
        if (ms < best.ms) {
          best = c;
          best.link_fmt = fmt;
          best.ms = ms;
        }
      }
      if (ret) break;
    }
    if (ret) break;
    h->tuned[TuneKey{lat, prec, mode, nrhs, var.epi}] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ret;
}

extern "C" int oq_tune_get_epi(oq_handle h, int lat, int prec, int mode, int epi, int nrhs, int* bx, int* by,
                               float* ms, int* link_fmt, int* nr, int* regcap) {
  if (!h || !bx || !by || !ms || lat < 0 || lat >= (int)h->lats.size() || epi < EPI_NONE || epi > EPI_CG)
    return OQ_ERR_ARG;
  // the launch lookup's rule: an epilogue without a launch of its own runs the mode's plain one
  auto it = h->tuned.find(TuneKey{lat, prec, mode, nrhs, epi});
  if (it == h->tuned.end()) it = h->tuned.find(TuneKey{lat, prec, mode, nrhs, EPI_NONE});
  if (it == h->tuned.end()) return OQ_ERR_STATE;
  const TuneVal& v = it->second;
  *bx = v.bx;
  *by = v.by;
  *ms = v.ms;
  if (link_fmt) *link_fmt = v.link_fmt >= 0 ? v.link_fmt : h->lats[lat].link_fmt;
  if (nr) *nr = v.nr;
  if (regcap) *regcap = v.regcap;
  return OQ_OK;
}

extern "C" int oq_tune_get(oq_handle h, int lat, int prec, int mode, int nrhs, int* bx, int* by, float* ms,
                           int* link_fmt, int* nr, int* regcap) {
  return oq_tune_get_epi(h, lat, prec, mode, EPI_NONE, nrhs, bx, by, ms, link_fmt, nr, regcap);
}

extern "C" int oq_tune_set(oq_handle h, int lat, int prec, int mode, int nrhs, int bx, int by, int nr, int regcap,
                           int link_fmt) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || prec < 0 || prec > 4 || mode < 0 || mode > 2 || nrhs < 1 ||
      nrhs > 64)
    return OQ_ERR_ARG;
  const LatCtx& L = h->lats[lat];
  if (!L.has_gauge) return OQ_ERR_STATE;
  TuneVal v;
  v.bx = bx;
  v.by = by;
  v.nr = nr;
  v.regcap = regcap;
  v.link_fmt = link_fmt;
  v.ms = 0.f;
  if (!valid_shape(L, prec, nrhs, v)) return OQ_ERR_ARG;
  // the pinned launch serves every epilogue of the mode
  const int epis[] = {EPI_NORM, EPI_CG, EPI_RESID64};
  for (int e : epis) h->tuned.erase(TuneKey{lat, prec, mode, nrhs, e});
  h->tuned[TuneKey{lat, prec, mode, nrhs, EPI_NONE}] = v;
  return OQ_OK;
}
