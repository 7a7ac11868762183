// Deterministic grid reductions in binary64 with a fused "finisher".
//
// Every CTA reduces its threads' partial sums per right-hand side (warp
// shuffles -- binary32 for binary32 site values, see warp_total -- then
// binary64 through shared memory), writes one binary64 partial per (rhs,
// CTA), and the last CTA to arrive (atomic ticket) sums the partials of that
// rhs in a fixed order with one warp (16 loads in flight per lane) and runs
// the finisher that turns the sum into solver scalars (CG alpha / beta,
// restart norms).  The order of the additions never depends on timing, so
// results are bitwise reproducible.
#pragma once
#include "oq_internal.h"

namespace oq {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// the same tree in binary32 (sums of 32 binary32 site values; binary64
// arithmetic runs at 1/64 of the binary32 rate on GB300)
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of part[0 .. n) by one warp in a fixed order: lane l adds the entries
// l + 32 j into 16 accumulators (j mod 16, the ragged end into the first),
// combined pairwise, then across the warp.  The 16 loads of a round are
// independent, so they are in flight together: the partials were written by
// other CTAs of the launch and are read from L2 (ld.global.cg, no L1 copy)
// after the ticket's fence.
__device__ __forceinline__ double warp_sum_partials(const double* part, unsigned n, int lane) {
  constexpr int U = 16;
  double acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = 0.0;
  unsigned b = (unsigned)lane;
  for (; b + (U - 1) * 32 < n; b += U * 32) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = __ldcg(part + b + u * 32);
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] += v[u];
  }
  for (; b < n; b += 32) acc[0] += __ldcg(part + b);
#pragma unroll
  for (int w = U / 2; w > 0; w >>= 1)
#pragma unroll
    for (int u = 0; u < w; ++u) acc[u] += acc[u + w];
  return warp_sum(acc[0]);
}

// The sum of a warp's values: binary32 values (per-site sums of binary32
// fields, e.g. 24 squares) are summed over the warp in binary32 (32 terms),
// binary64 values in binary64; either way the result and everything beyond
// the warp are binary64.
__device__ __forceinline__ double warp_total(float v) { return (double)warp_sum_f(v); }
__device__ __forceinline__ double warp_total(double v) { return warp_sum(v); }

__device__ __forceinline__ void run_finisher(const RedArgs& ra, int rhs, double sum) {
  CgState* st = ra.cg ? ra.cg + rhs : nullptr;
  if (ra.fin != FIN_STORE && st->mode != ra.gate) return;  // rhs was not live in this launch
  switch (ra.fin) {
    case FIN_STORE:
      ra.result[rhs] = sum;
      break;
    case FIN_ALPHA:
      st->pAp = sum;
      if (!(sum > 0.0) || !isfinite(sum)) {
        st->alpha = 0.0;
        st->mode = MODE_RESET;
        st->reason = isfinite(sum) ? WHY_BREAKDOWN : WHY_NONFINITE;
      } else {
        st->alpha = st->rr / sum;
      }
      break;
    case FIN_BETA: {
      double rr_new = sum;
      st->steps += 1;
      if (!isfinite(rr_new)) {
        st->mode = MODE_RESET;
        st->reason = WHY_NONFINITE;
      } else if (rr_new <= st->tol2) {
        st->mode = MODE_RESET;
        st->reason = WHY_TOL;
      } else if (rr_new <= st->delta2 * st->rr_start) {
        st->mode = MODE_RESET;
        st->reason = WHY_DELTA;
      } else if (st->steps >= st->nmx) {
        st->mode = MODE_RESET;
        st->reason = WHY_NMX;
      } else {
        st->beta = rr_new / st->rr;
      }
      st->rr = rr_new;
      break;
    }
    case FIN_RESTART:
      st->rr = sum;
      st->rr_start = sum;
      st->mode = MODE_RUN;
      st->reason = WHY_NONE;
      break;
    case FIN_RD2:
      st->rd2 = sum;
      break;
  }
}

// Called by all threads of a CTA of shape (bx, by): thread (tx, ty) holds v
// (binary32 or binary64, see warp_total) for right-hand side `rhs` (one rhs
// per row).  `cta` numbers this CTA among
// the `ncta` CTAs that contribute to the same rhs.  smem needs bx*by/32 doubles.
// off: the rhs is gated off in this launch (its solver state is not in the
// launch's mode).  Every CTA of the launch sees the same state (it changes
// only in the finisher of the last CTA), so all of them skip the rhs: no
// partial, no ticket, no finisher.
template <typename T>
__device__ __forceinline__ void grid_reduce(T v, const RedArgs& ra, int rhs, int nrhs, double* smem, unsigned cta,
                                            unsigned ncta, bool off = false) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nw = blockDim.x >> 5;  // warps per rhs row (blockDim.x % 32 == 0)
  const double w = warp_total(v);
  if ((tx & 31) == 0) smem[ty * nw + (tx >> 5)] = w;
  __syncthreads();
  if (tx < 32) {
    bool last = false;
    double s = 0.0;
    if (rhs < nrhs && !off) {
      if (tx == 0) {
        for (int w = 0; w < nw; ++w) s += smem[ty * nw + w];
        ra.partials[(long)rhs * ncta + cta] = s;
        __threadfence();
        unsigned t = atomicAdd(ra.counters + rhs, 1u);
        last = (t == ncta - 1);
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        __threadfence();
        const double acc = warp_sum_partials(ra.partials + (long)rhs * ncta, ncta, tx);
        if (tx == 0) {
          ra.counters[rhs] = 0u;
          run_finisher(ra, rhs, acc);
        }
      }
    }
  }
}

// grid_reduce for NR values per thread (right-hand sides rhs0 .. rhs0+NR-1
// of the thread's row): smem needs (blockDim.x / 32) * blockDim.y * NR doubles;
// off[k]: rhs0 + k is gated off in this launch (skipped by every CTA, as in
// grid_reduce); value types as in grid_reduce.
template <int NR, typename T>
__device__ __forceinline__ void grid_reduce_nr(const T (&v)[NR], const RedArgs& ra, int rhs0, int nrhs,
                                               double* smem, unsigned cta, unsigned ncta, const bool (&off)[NR]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const double s = warp_total(v[k]);
    if ((tx & 31) == 0) smem[(ty * NR + k) * nw + (tx >> 5)] = s;
  }
  __syncthreads();
  if (tx >= 32) return;
  for (int k = 0; k < NR; ++k) {
    const int rhs = rhs0 + k;
    if (rhs >= nrhs) break;
    if (off[k]) continue;
    bool last = false;
    if (tx == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += smem[(ty * NR + k) * nw + w];
      ra.partials[(long)rhs * ncta + cta] = s;
      __threadfence();
      const unsigned t = atomicAdd(ra.counters + rhs, 1u);
      last = (t == ncta - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      const double acc = warp_sum_partials(ra.partials + (long)rhs * ncta, ncta, tx);
      if (tx == 0) {
        ra.counters[rhs] = 0u;
        run_finisher(ra, rhs, acc);
      }
    }
  }
}

}  // namespace oq
