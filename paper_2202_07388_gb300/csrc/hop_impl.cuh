// The Wilson-clover stencil on even-odd ordered half lattices.
//
// One thread computes one output site of parity p for one right-hand side:
//
//   H psi(x) = sum_mu [ U_mu(x) (1 - g_mu) psi(x+mu) + U_mu(x-mu)^dag (1 + g_mu) psi(x-mu) ]
//
// (projectors swapped for the adjoint, since g5 (1 -/+ g_mu) g5 = (1 +/- g_mu)),
// with the two-component spin projection so that only half spinors are
// transported by the links, and the time-boundary factor on hops that cross
// x0 = T-1 <-> 0.  The mode picks what is done with H psi:
//
//   HOP_DW : out = A in2 - 1/2 H in                  (one parity of D psi)
//   HOP_P1 : out = A^{-1} (-1/2 H in)                (D_oo^{-1} D_oe psi_e)
//   HOP_P2 : out = A in2 + 1/2 H in                  (D_ee psi_e - D_eo t_o)
//
// and the epilogue fuses the vector work of the solvers into the store
// (norm of the output, the CG update of x and r, or the binary64 residual
// eta - out of a reset step) with a deterministic binary64 grid reduction.
#pragma once
#include "reduce.cuh"

namespace oq {

// Accumulate one transported hop: with weight w (times the time-boundary
// factor when the hop crosses it) for binary64 / binary32, where the weight
// folds into FMAs; double-float sums the hops unweighted (a sign flip for
// the boundary) and hop_site scales once by w = +-1/2 (exact).
template <int MU, int S, typename R>
__device__ __forceinline__ void hop_accum(Spinor<R>& acc, HalfSpinor<R>& t, R w, bool cr, float bc_t) {
  if constexpr (std::is_same<R, dfloat>::value) {
    if (cr && bc_t < 0.f) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) t.c[s][c] = -t.c[s][c];
    }
    accum_reconstruct<MU, S, R, false>(acc, t, w);
  } else {
    accum_reconstruct<MU, S>(acc, t, cr ? w * (R)bc_t : w);
  }
}

// fnext / fprev (sub-domain launches, this rhs and output parity): the time
// faces that replace the hops leaving the sub-domain (HopArgs::halo_next)
template <int P, int FMT, int MU, bool DAG>
__device__ __forceinline__ void hop_dir(const HopArgs& a, const char* in, int p, long i, const int x[4],
                                        Spinor<typename PrecTraits<P>::R>& acc,
                                        typename PrecTraits<P>::R w, const char* fnext = nullptr,
                                        const char* fprev = nullptr) {
  typedef typename PrecTraits<P>::R R;
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
  bool cr;
  // forward: U_mu(x) (1 -/+ g) psi(x + mu)
  {
    long j = eo_neighbour(a.g, x, MU, +1, &cr);
    HalfSpinor<R> h, t;
    float sg = a.g.bc_t;
    if (MU == 0 && cr && fnext) {
      // x0 = T-1: the projected neighbour comes from the next sub-domain
      const long Fs = a.g.Vh / a.g.L[0];
      load_half<R>(fnext, Fs, i - (long)x[0] * Fs, h);
      sg = a.halo_sign_next;
    } else {
      Spinor<R> nb;
      load_spinor<P>(in, a.g.Vh, j, nb);
      project<MU, SF>(nb, h);
    }
    Su3<R> u;
    load_link<R, FMT>(a.links, a.g.Vh, p, MU, i, u);
    su3_mul(u, h, t);
    hop_accum<MU, SF>(acc, t, w, cr, sg);
  }
  // backward: U_mu(x - mu)^dag (1 +/- g) psi(x - mu)
  {
    long j = eo_neighbour(a.g, x, MU, -1, &cr);
    HalfSpinor<R> t;
    float sg = a.g.bc_t;
    if (MU == 0 && cr && fprev) {
      // x0 = 0: link and projection were applied by the previous sub-domain
      load_half<R>(fprev, a.g.Vh / a.g.L[0], i, t);
      sg = a.halo_sign_prev;
    } else {
      Spinor<R> nb;
      load_spinor<P>(in, a.g.Vh, j, nb);
      HalfSpinor<R> h;
      project<MU, -SF>(nb, h);
      Su3<R> u;
      load_link<R, FMT>(a.links, a.g.Vh, 1 - p, MU, j, u);
      su3_dag_mul(u, h, t);
    }
    hop_accum<MU, -SF>(acc, t, w, cr, sg);
  }
}

// z * i^c for c in 0..3 (double-float): a swap of the parts for odd c and
// sign flips, all by selects
__device__ __forceinline__ cx<dfloat> rot_ic(const cx<dfloat>& z, int c) {
  const bool sw = c & 1;
  dfloat re = sw ? z.im : z.re, im = sw ? z.re : z.im;
  if (c == 1 || c == 2) re = -re;
  if (c >= 2) im = -im;
  return cx<dfloat>{re, im};
}

// The hopping sum in double-float as one runtime loop over the 8 hops: the
// fully unrolled double-float stencil is ~14k instructions, far beyond the
// instruction cache, while one loop body (~1k) stays resident.  The spin
// projection for hop (mu, projector sign S) is h0 = p0 + i^c0 p[q0],
// h1 = p1 + i^c1 p[q1], the reconstruction acc2 += i^d0 t[r0],
// acc3 += i^d1 t[r1] (the same linear maps as project / accum_reconstruct,
// as tables; S = +1 adds 2 to every power); a backward hop applies
// U(x - mu)^dag by conjugate-transposing the link in registers.
template <int P, int FMT, bool DAG>
__device__ __forceinline__ void hop_loop_df(const HopArgs& a, const char* in, int p, long i, const int x[4],
                                            Spinor<dfloat>& acc) {
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    const int sh = ((fwd ? SF : -SF) > 0) ? 2 : 0;
    bool cr;
    const long j = eo_neighbour_rt(a.g, x, mu, fwd ? +1 : -1, &cr);
    Spinor<dfloat> nb;
    load_spinor<P>(in, a.g.Vh, j, nb);
    Su3<dfloat> u;
    load_link<dfloat, FMT>(a.links, a.g.Vh, fwd ? p : 1 - p, mu, fwd ? i : j, u);
    if (!fwd) {
      Su3<dfloat> v = u;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) u.m[r][c] = conj(v.m[c][r]);
    }
    // projection tables (mu = 0..3): partners q0, q1 and powers of i
    const bool swq = (mu == 1 || mu == 2);       // q0 = 3, q1 = 2
    const int c0 = ((mu == 1 || mu == 3) ? 1 : 0) + sh;
    const int c1 = (mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 2 : 3) + sh;
    HalfSpinor<dfloat> h, t;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<dfloat> pa = swq ? nb.c[3][c] : nb.c[2][c];
      const cx<dfloat> pb = swq ? nb.c[2][c] : nb.c[3][c];
      const cx<dfloat> ra = rot_ic(pa, c0 & 3), rb = rot_ic(pb, c1 & 3);
      h.c[0][c] = cx<dfloat>{df_add_lazy(nb.c[0][c].re, ra.re), df_add_lazy(nb.c[0][c].im, ra.im)};
      h.c[1][c] = cx<dfloat>{df_add_lazy(nb.c[1][c].re, rb.re), df_add_lazy(nb.c[1][c].im, rb.im)};
    }
    su3_mul(u, h, t);
    if (cr && a.g.bc_t < 0.f) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) t.c[s][c] = -t.c[s][c];
    }
    // reconstruction tables: r0 = 1, r1 = 0 for mu = 1, 2
    const int d0 = (mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 2 : 3) + sh;
    const int d1 = (mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 0 : 1) + sh;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<dfloat> ta = rot_ic(swq ? t.c[1][c] : t.c[0][c], d0 & 3);
      const cx<dfloat> tb = rot_ic(swq ? t.c[0][c] : t.c[1][c], d1 & 3);
      const cx<dfloat> up[4] = {t.c[0][c], t.c[1][c], ta, tb};
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
        acc.c[s2][c] = cx<dfloat>{df_add_lazy(acc.c[s2][c].re, up[s2].re), df_add_lazy(acc.c[s2][c].im, up[s2].im)};
    }
  }
  // the hops were summed without renormalising
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc.c[s2][c] = cx<dfloat>{df_norm(acc.c[s2][c].re), df_norm(acc.c[s2][c].im)};
}

// value type of a site's reduction contribution: binary32 for the
// binary32-arithmetic types (their per-site norms are binary32 sums), else
// binary64 (see warp_total)
template <int P>
using RedT = typename std::conditional<P == P_F64 || P == P_DF64, double, float>::type;

// One output site i (parity p) of right-hand side rhs: the stencil, the
// clover term and the epilogue.  Returns the site's contribution to the
// epilogue's reduction (0 if none).
template <int P, int FMT, int MODE, bool DAG, int EPI>
__device__ __forceinline__ RedT<P> hop_site(const HopArgs& a, long i, int rhs, int p) {
  typedef typename PrecTraits<P>::R R;
  RedT<P> red = 0;
    int x[4];
    eo_coords(a.g, p, i, x);
    const long par_in = (MODE == HOP_DW) ? (long)(1 - p) * a.half_bytes : 0;
    const long par_out = (MODE == HOP_DW) ? (long)p * a.half_bytes : 0;
    const char* in = (const char*)a.in + rhs * a.in_stride + par_in;
    Spinor<R> acc;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc.c[s][c] = cx<R>{0, 0};
    const R w = (MODE == HOP_P2) ? (R)0.5 : (R)-0.5;
    constexpr bool DF = std::is_same<R, dfloat>::value;
    if constexpr (DF && MODE != HOP_P1) {
      // double-float: A in2 / w first (w = +-1/2, so the scaling is exact)
      // while few registers are live; the unweighted hops add onto it and
      // one final scaling by w gives A in2 + w H in
      Spinor<R> loc;
      load_spinor<P>((const char*)a.in2 + rhs * a.in2_stride + par_out, a.g.Vh, i, loc);
      clover_apply<R>(a.clov, a.g.Vh, p, i, loc, acc);
      const float iw = 1.f / w.hi;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          acc.c[s][c] = cx<R>{df_scale(acc.c[s][c].re, iw), df_scale(acc.c[s][c].im, iw)};
    }
    if constexpr (DF) {
      hop_loop_df<P, FMT, DAG>(a, in, p, i, x, acc);
    } else {
      const char* fn = nullptr;
      const char* fp = nullptr;
      if (a.halo_next) {  // sub-domain launch: faces of this rhs and output parity
        const long po = (MODE == HOP_DW) ? (long)p * a.halo_pstride : 0;
        fn = (const char*)a.halo_next + rhs * a.halo_stride + po;
        fp = (const char*)a.halo_prev + rhs * a.halo_stride + po;
      }
      hop_dir<P, FMT, 0, DAG>(a, in, p, i, x, acc, w, fn, fp);
      hop_dir<P, FMT, 1, DAG>(a, in, p, i, x, acc, w);
      hop_dir<P, FMT, 2, DAG>(a, in, p, i, x, acc, w);
      hop_dir<P, FMT, 3, DAG>(a, in, p, i, x, acc, w);
    }
    if constexpr (DF) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          acc.c[s][c] = cx<R>{df_scale(acc.c[s][c].re, w.hi), df_scale(acc.c[s][c].im, w.hi)};
    }

    Spinor<R> res;
    if constexpr (MODE == HOP_P1) {
      clover_apply<R>(a.cinv, a.g.Vh, p, i, acc, res);
    } else if constexpr (DF) {
      res = acc;
    } else {
      const char* in2 = (const char*)a.in2 + rhs * a.in2_stride + par_out;
      Spinor<R> loc, al;
      load_spinor<P>(in2, a.g.Vh, i, loc);
      clover_apply<R>(a.clov, a.g.Vh, p, i, loc, al);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) res.c[s][c] = al.c[s][c] + acc.c[s][c];
    }

    if constexpr (EPI == EPI_NONE || EPI == EPI_NORM) {
      store_spinor<P>((char*)a.out + rhs * a.out_stride + par_out, a.g.Vh, i, res);
      if constexpr (EPI == EPI_NORM) red = (RedT<P>)site_norm2(res);
    } else if constexpr (EPI == EPI_CG) {
      // q = res; x += alpha p; r -= alpha q  (x in F64 for F64 solves, else F32)
      constexpr int XP = (P == P_F64) ? P_F64 : P_F32;
      typedef typename PrecTraits<XP>::R RX;
      const CgState& st = a.cg[rhs];
      const R al = (R)st.alpha;
      Spinor<R> pv, rv;
      Spinor<RX> xv;
      load_spinor<P>((const char*)a.ep_p + rhs * a.ep_p_stride, a.g.Vh, i, pv);
      load_spinor<P>((const char*)a.ep_r + rhs * a.ep_r_stride, a.g.Vh, i, rv);
      load_spinor<XP>((const char*)a.ep_x + rhs * a.ep_x_stride, a.g.Vh, i, xv);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xv.c[s][c].re = fma((RX)al, (RX)pv.c[s][c].re, xv.c[s][c].re);
          xv.c[s][c].im = fma((RX)al, (RX)pv.c[s][c].im, xv.c[s][c].im);
          rv.c[s][c].re = fma(-al, res.c[s][c].re, rv.c[s][c].re);
          rv.c[s][c].im = fma(-al, res.c[s][c].im, rv.c[s][c].im);
        }
      // the norm of what is stored (rounded to the storage type)
      round_trip<P>(rv);
      store_spinor<XP>((char*)a.ep_x + rhs * a.ep_x_stride, a.g.Vh, i, xv);
      store_spinor<P>((char*)a.ep_r + rhs * a.ep_r_stride, a.g.Vh, i, rv);
      red = (RedT<P>)site_norm2(rv);
    } else if constexpr (EPI == EPI_RESID64) {
      Spinor<R> e;
      load_spinor<P>((const char*)a.ep_eta + rhs * a.ep_eta_stride, a.g.Vh, i, e);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) res.c[s][c] = e.c[s][c] - res.c[s][c];
      store_spinor<P>((char*)a.out + rhs * a.out_stride, a.g.Vh, i, res);
      if constexpr (P == P_DF64) {
        // the site's 24 squares summed in double-float, one conversion
        dfloat acc2(0.f);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) acc2 = fma(res.c[s][c].re, res.c[s][c].re, fma(res.c[s][c].im, res.c[s][c].im, acc2));
        red = (double)acc2;
      } else {
        double acc2 = 0.0;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double re = (double)res.c[s][c].re, im = (double)res.c[s][c].im;
            acc2 += re * re + im * im;
          }
        red = acc2;
      }
    }
  return red;
}

template <int P, int FMT, int MODE, bool DAG, int EPI>
__device__ __forceinline__ void hop_kernel_body(const HopArgs& a, double* red_smem) {
  // CTA = blockDim.x sites x blockDim.y right-hand sides (one rhs per row:
  // the rows read the same links and clover blocks, served by L1).  The
  // grid index runs fastest over the rhs tiles of one site block, then (for
  // HOP_DW) over the two parities, then over site blocks, so that CTAs that
  // read the same links are resident at the same time and share them in L2.
  const unsigned ntile = (a.nrhs + blockDim.y - 1) / blockDim.y;
  const unsigned tile = blockIdx.x % ntile;
  const unsigned rest = blockIdx.x / ntile;
  const long blk = (MODE == HOP_DW) ? (long)(rest >> 1) : (long)rest;
  const long i = blk * blockDim.x + threadIdx.x;
  const int rhs = tile * blockDim.y + threadIdx.y;
  const int p = (MODE == HOP_DW) ? (int)(rest & 1) : a.p;
  record_live(a);
  const bool off = a.cg && rhs < a.nrhs && a.cg[rhs].mode != a.gate;  // gated off by the solver state
  const bool live = (i < a.g.Vh) && (rhs < a.nrhs) && !off;
  RedT<P> red = 0;
  if (live) red = hop_site<P, FMT, MODE, DAG, EPI>(a, i, rhs, p);
  if constexpr (EPI != EPI_NONE) {
    grid_reduce(red, a.red, rhs, a.nrhs, red_smem, (unsigned)blk, gridDim.x / ntile, off);
  }
}

template <int P, int FMT, int MODE, bool DAG, int EPI>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs a) {
  extern __shared__ double red_smem[];
  hop_kernel_body<P, FMT, MODE, DAG, EPI>(a, red_smem);
}

// double-float only: at most 128 threads and 128 registers per thread, so
// that 16 warps fit on an SM (the tuner weighs it against hop_kernel), or
// 168 registers for 12 warps (fewer spills)
template <int P, int FMT, int MODE, bool DAG, int EPI>
__global__ void __launch_bounds__(128, 4) hop_kernel_capped(const HopArgs a) {
  extern __shared__ double red_smem[];
  hop_kernel_body<P, FMT, MODE, DAG, EPI>(a, red_smem);
}
template <int P, int FMT, int MODE, bool DAG, int EPI>
__global__ void __launch_bounds__(128, 3) hop_kernel_capped3(const HopArgs a) {
  extern __shared__ double red_smem[];
  hop_kernel_body<P, FMT, MODE, DAG, EPI>(a, red_smem);
}

// Batched form over several systems (lattices / operators of any size, one
// right-hand side each): a persistent grid walks a list of tiles
// (system, site block); every system has its own arguments, solver state and
// reduction scratch in device memory.  For HOP_DW the block index carries
// the parity in its lowest bit.
template <int P, int FMT, int MODE, bool DAG, int EPI>
__global__ void __launch_bounds__(256) hop_batch_kernel(const HopArgs* __restrict__ sys,
                                                        const int2* __restrict__ tiles, int ntiles) {
  extern __shared__ double red_smem[];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const HopArgs& a = sys[tl.x];
    const long blk = (MODE == HOP_DW) ? (long)(tl.y >> 1) : (long)tl.y;
    const int p = (MODE == HOP_DW) ? (tl.y & 1) : a.p;
    const long i = blk * blockDim.x + threadIdx.x;
    const bool off = a.cg && a.cg[0].mode != a.gate;  // the system is gated off by its solver state
    const bool live = i < a.g.Vh && !off;
    RedT<P> red = 0;
    if (live) red = hop_site<P, FMT, MODE, DAG, EPI>(a, i, 0, p);
    if constexpr (EPI != EPI_NONE) {
      const unsigned nblk = (unsigned)((a.g.Vh + blockDim.x - 1) / blockDim.x);
      grid_reduce(red, a.red, 0, 1, red_smem, (unsigned)blk, nblk, off);
    }
  }
}

template <int P, int FMT, int MODE, bool DAG, int EPI>
static cudaError_t launch_one(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  dim3 block(L.bx, L.by, 1);
  const unsigned nb = (unsigned)((a.g.Vh + L.bx - 1) / L.bx);
  const unsigned ntile = (unsigned)((a.nrhs + L.by - 1) / L.by);
  dim3 grid((MODE == HOP_DW ? 2u * nb : nb) * ntile, 1u, 1u);
  size_t smem = (EPI == EPI_NONE) ? 0 : sizeof(double) * (L.bx / 32) * L.by;
  if (L.sys) {
    dim3 bblock(L.bx, 1, 1);
    hop_batch_kernel<P, FMT, MODE, DAG, EPI><<<L.grid, bblock, (EPI == EPI_NONE) ? 0 : sizeof(double) * (L.bx / 32),
                                                s>>>(L.sys, L.tiles, L.ntiles);
    return cudaGetLastError();
  }
  if constexpr (P == P_DF64) {
    if (L.regcap) {
      if (L.bx * L.by > 128) return cudaErrorInvalidValue;
      if (L.regcap == 2)
        hop_kernel_capped3<P, FMT, MODE, DAG, EPI><<<grid, block, smem, s>>>(a);
      else
        hop_kernel_capped<P, FMT, MODE, DAG, EPI><<<grid, block, smem, s>>>(a);
      return cudaGetLastError();
    }
  }
  hop_kernel<P, FMT, MODE, DAG, EPI><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int FMT, bool DAG>
static cudaError_t dispatch_mode_epi(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  switch (L.mode) {
    case HOP_DW:
      if (L.epi == EPI_NONE) return launch_one<P, FMT, HOP_DW, DAG, EPI_NONE>(L, a, s);
      break;
    case HOP_P1:
      if (L.epi == EPI_NONE) return launch_one<P, FMT, HOP_P1, DAG, EPI_NONE>(L, a, s);
      break;
    case HOP_P2:
      if (L.epi == EPI_NONE) return launch_one<P, FMT, HOP_P2, DAG, EPI_NONE>(L, a, s);
      if constexpr (P != P_DF64) {
        if (L.epi == EPI_NORM) return launch_one<P, FMT, HOP_P2, DAG, EPI_NORM>(L, a, s);
        if (L.epi == EPI_CG) return launch_one<P, FMT, HOP_P2, DAG, EPI_CG>(L, a, s);
      }
      if constexpr (P == P_F64 || P == P_DF64)
        if (L.epi == EPI_RESID64) return launch_one<P, FMT, HOP_P2, DAG, EPI_RESID64>(L, a, s);
      break;
  }
  return cudaErrorInvalidValue;
}

template <int P, int FMT>
static cudaError_t dispatch_dag(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  return L.dagger ? dispatch_mode_epi<P, FMT, true>(L, a, s) : dispatch_mode_epi<P, FMT, false>(L, a, s);
}

}  // namespace oq
