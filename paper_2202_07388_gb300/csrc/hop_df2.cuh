// Double-float stencil passes with two right-hand sides per thread.
//
// The reset steps of the mixed-precision CGNE recompute the residual in
// double-float arithmetic (an unevaluated sum hi + lo of two binary32
// numbers; oq_device.cuh), one right-hand side per thread in hop_impl.cuh.
// Here a thread carries two right-hand sides: every binary32 operation of
// the double-float formulas acts on the pair at once as one packed two-lane
// instruction (FADD2 / FMUL2 / FFMA2 of sm_100-class GPUs), in the same order
// as the one-rhs kernel, so each lane's result is bit for bit that of the
// one-rhs kernel.  The links and clover blocks of a site are loaded once for
// both.  A packed instruction occupies the binary32 pipe as long as two
// scalar ones (the same flop rate); what it saves is issue slots and the
// loads, index arithmetic and link handling per right-hand side, which bound
// the one-rhs kernel (binary32 pipe ~55 % busy at ~75 % issue).
//
// Passes and epilogues: Dw (HOP_DW), Dhat pass 1 (HOP_P1), pass 2
// (HOP_P2), with the plain store or the binary64-residual epilogue of a reset
// step (eta - out, its double-float norm).
#pragma once
#include "hop_impl.cuh"

namespace oq {
namespace df2 {

typedef float2 F2;
__device__ __forceinline__ F2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add(F2 a, F2 b) { return __fadd2_rn(a, b); }
// RN(a - b): the product b * (-1) is exact, so one rounding as in a subtraction
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return __ffma2_rn(b, bc(-1.f), a); }
__device__ __forceinline__ F2 mul(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 neg(F2 a) { return make_float2(-a.x, -a.y); }

// lane k (k = 0, 1: the thread's two right-hand sides) holds hi.k + lo.k
struct D2 {
  F2 hi, lo;
};
struct C2 {
  D2 re, im;
};
__device__ __forceinline__ D2 dneg(D2 x) { return D2{neg(x.hi), neg(x.lo)}; }
__device__ __forceinline__ C2 cneg(C2 z) { return C2{dneg(z.re), dneg(z.im)}; }

// the error-free transformations and double-float operations of
// oq_device.cuh, lane by lane
__device__ __forceinline__ D2 two_sum(F2 a, F2 b) {
  const F2 s = add(a, b);
  const F2 bb = sub(s, a);
  return D2{s, add(sub(a, sub(s, bb)), sub(b, bb))};
}
__device__ __forceinline__ D2 fast_two_sum(F2 a, F2 b) {
  const F2 s = add(a, b);
  return D2{s, sub(b, sub(s, a))};
}
__device__ __forceinline__ D2 dadd(D2 x, D2 y) {
  const D2 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, add(s.lo, add(x.lo, y.lo)));
}
__device__ __forceinline__ D2 add_lazy(D2 x, D2 y) {
  const D2 s = two_sum(x.hi, y.hi);
  return D2{s.hi, add(s.lo, add(x.lo, y.lo))};
}
__device__ __forceinline__ D2 dnorm(D2 x) { return fast_two_sum(x.hi, x.lo); }
__device__ __forceinline__ D2 dscale(D2 x, float s) { return D2{mul(x.hi, bc(s)), mul(x.lo, bc(s))}; }
// a * b + c (both factors per lane)
__device__ __forceinline__ D2 dfma(D2 a, D2 b, D2 c) {
  const F2 p = mul(a.hi, b.hi);
  F2 e = fma2(a.hi, b.hi, neg(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  const D2 s = two_sum(c.hi, p);
  return fast_two_sum(s.hi, add(s.lo, add(c.lo, e)));
}

// lazy dot product (DfAcc) with a factor shared by the two lanes
struct Acc {
  F2 s, e;
};
__device__ __forceinline__ void acc_first(Acc& a, dfloat x, D2 y) {
  const F2 xh = bc(x.hi), xl = bc(x.lo);
  a.s = mul(xh, y.hi);
  F2 e = fma2(xh, y.hi, neg(a.s));
  e = fma2(xh, y.lo, e);
  a.e = fma2(xl, y.hi, e);
}
__device__ __forceinline__ void acc_add(Acc& a, dfloat x, D2 y) {
  const F2 xh = bc(x.hi), xl = bc(x.lo);
  const F2 p = mul(xh, y.hi);
  F2 e = fma2(xh, y.hi, neg(p));
  e = fma2(xh, y.lo, e);
  e = fma2(xl, y.hi, e);
  const D2 t = two_sum(a.s, p);
  a.s = t.hi;
  a.e = add(a.e, add(t.lo, e));
}
__device__ __forceinline__ D2 acc_get(const Acc& a) { return fast_two_sum(a.s, a.e); }

// z * i^c (selects and sign flips, as rot_ic)
__device__ __forceinline__ C2 rot_ic(const C2& z, int c) {
  const bool sw = c & 1;
  D2 re = sw ? z.im : z.re, im = sw ? z.re : z.im;
  if (c == 1 || c == 2) re = dneg(re);
  if (c >= 2) im = dneg(im);
  return C2{re, im};
}

// chunk k (= 3 spin + colour) of the two right-hand sides' double-float
// spinors at eo index j: one (re.hi, re.lo, im.hi, im.lo) float4 each
__device__ __forceinline__ C2 ld(const float4* b0, const float4* b1, long Vh, int k, long j) {
  const float4 v0 = ldg_nc(b0 + k * Vh + j), v1 = ldg_nc(b1 + k * Vh + j);
  return C2{D2{make_float2(v0.x, v1.x), make_float2(v0.y, v1.y)}, D2{make_float2(v0.z, v1.z), make_float2(v0.w, v1.w)}};
}
__device__ __forceinline__ void st(float4* b0, float4* b1, bool l0, bool l1, long Vh, int k, long i, const C2& z) {
  if (l0) b0[k * Vh + i] = make_float4(z.re.hi.x, z.re.lo.x, z.im.hi.x, z.im.lo.x);
  if (l1) b1[k * Vh + i] = make_float4(z.re.hi.y, z.re.lo.y, z.im.hi.y, z.im.lo.y);
}

// y = K x for clover block b of site i (parity p): clover_apply<dfloat>'s
// row-by-row lazy dot products, the block's reals loaded once for both lanes
__device__ __forceinline__ void clover_block(const void* base, long Vh, int p, long i, int b, const C2 (&x)[6],
                                             C2 (&y)[6]) {
  const float4* q = reinterpret_cast<const float4*>(base) + (long)p * 36 * Vh;
  dfloat d[6];
  cx<dfloat> off[15];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 w = ldg_nc(q + (18 * b + k) * Vh + i);
    d[2 * k] = dfloat(w.x, w.y);
    d[2 * k + 1] = dfloat(w.z, w.w);
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    const float4 w = ldg_nc(q + (18 * b + 3 + k) * Vh + i);
    off[k] = cx<dfloat>{dfloat(w.x, w.y), dfloat(w.z, w.w)};
  }
#pragma unroll
  for (int r0 = 0; r0 < 6; ++r0) {
    Acc re, im;
    acc_first(re, d[r0], x[r0].re);
    acc_first(im, d[r0], x[r0].im);
#pragma unroll
    for (int c0 = 0; c0 < 6; ++c0) {
      if (c0 == r0) continue;
      const int a0 = r0 < c0 ? r0 : c0, b0 = r0 < c0 ? c0 : r0;
      const int k = a0 * 5 - a0 * (a0 - 1) / 2 + (b0 - a0 - 1);
      const cx<dfloat> o2 = off[k];
      const dfloat oi = r0 < c0 ? o2.im : -o2.im;  // conj for the lower triangle
      acc_add(re, o2.re, x[c0].re);
      acc_add(re, -oi, x[c0].im);
      acc_add(im, o2.re, x[c0].im);
      acc_add(im, oi, x[c0].re);
    }
    y[r0] = C2{acc_get(re), acc_get(im)};
  }
}

// The 8 hops as one runtime loop (hop_loop_df for two lanes): the spin
// projection is formed colour by colour from the neighbour's chunks, and each
// colour row of U h is reconstructed onto acc as soon as it is formed, so
// neither the neighbour spinor nor the transported half spinor is held whole.
// Every acc entry receives the same lazy additions in the same order as in
// the one-rhs kernel.
template <bool DAG>
__device__ __forceinline__ void hop_loop(const HopArgs& a, const float4* in0, const float4* in1, int p, long i,
                                         const int x[4], C2 (&acc)[4][3]) {
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
  const long Vh = a.g.Vh;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int mu = k >> 1;
    const bool fwd = (k & 1) == 0;
    const int sh = ((fwd ? SF : -SF) > 0) ? 2 : 0;
    bool cr;
    const long j = eo_neighbour_rt(a.g, x, mu, fwd ? +1 : -1, &cr);
    Su3<dfloat> u;
    load_link<dfloat, LINK_18>(a.links, Vh, fwd ? p : 1 - p, mu, fwd ? i : j, u);
    if (!fwd) {
      const Su3<dfloat> v = u;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) u.m[r][c] = conj(v.m[c][r]);
    }
    const bool swq = (mu == 1 || mu == 2);
    const int c0 = ((mu == 1 || mu == 3) ? 1 : 0) + sh;
    const int c1 = (mu == 0 ? 0 : mu == 1 ? 1 : mu == 2 ? 2 : 3) + sh;
    C2 h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C2 n0 = ld(in0, in1, Vh, c, j), n1 = ld(in0, in1, Vh, 3 + c, j);
      const C2 n2 = ld(in0, in1, Vh, 6 + c, j), n3 = ld(in0, in1, Vh, 9 + c, j);
      const C2 ra = rot_ic(swq ? n3 : n2, c0 & 3), rb = rot_ic(swq ? n2 : n3, c1 & 3);
      h[0][c] = C2{add_lazy(n0.re, ra.re), add_lazy(n0.im, ra.im)};
      h[1][c] = C2{add_lazy(n1.re, rb.re), add_lazy(n1.im, rb.im)};
    }
    const bool flip = cr && a.g.bc_t < 0.f;
    const int d0 = (mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 2 : 3) + sh;
    const int d1 = (mu == 0 ? 0 : mu == 1 ? 3 : mu == 2 ? 0 : 1) + sh;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      C2 t[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        Acc re, im;
        acc_first(re, u.m[r][0].re, h[s][0].re);
        acc_add(re, -u.m[r][0].im, h[s][0].im);
        acc_first(im, u.m[r][0].re, h[s][0].im);
        acc_add(im, u.m[r][0].im, h[s][0].re);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
          acc_add(re, u.m[r][b].re, h[s][b].re);
          acc_add(re, -u.m[r][b].im, h[s][b].im);
          acc_add(im, u.m[r][b].re, h[s][b].im);
          acc_add(im, u.m[r][b].im, h[s][b].re);
        }
        t[s] = C2{acc_get(re), acc_get(im)};
        if (flip) t[s] = cneg(t[s]);
      }
      const C2 ta = rot_ic(swq ? t[1] : t[0], d0 & 3), tb = rot_ic(swq ? t[0] : t[1], d1 & 3);
      const C2 up[4] = {t[0], t[1], ta, tb};
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
        acc[s2][r] = C2{add_lazy(acc[s2][r].re, up[s2].re), add_lazy(acc[s2][r].im, up[s2].im)};
    }
  }
  // the hops were summed without renormalising
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[s2][c] = C2{dnorm(acc[s2][c].re), dnorm(acc[s2][c].im)};
}

// One output site i (parity p) for right-hand sides rhs0, rhs0 + 1: the
// double-float branch of hop_site.  red[k]: the residual epilogue's site
// norm of lane k.
template <int MODE, bool DAG, int EPI>
__device__ __forceinline__ void site(const HopArgs& a, long i, int rhs0, int p, const bool (&live)[2],
                                     double (&red)[2]) {
  const long Vh = a.g.Vh;
  int x[4];
  eo_coords(a.g, p, i, x);
  const long par_in = (MODE == HOP_DW) ? (long)(1 - p) * a.half_bytes : 0;
  const long par_out = (MODE == HOP_DW) ? (long)p * a.half_bytes : 0;
  // lanes past nrhs read the last right-hand side and store nothing
  const int r0 = rhs0 < a.nrhs ? rhs0 : a.nrhs - 1;
  const int r1 = rhs0 + 1 < a.nrhs ? rhs0 + 1 : a.nrhs - 1;
  const float4* in0 = reinterpret_cast<const float4*>((const char*)a.in + r0 * a.in_stride + par_in);
  const float4* in1 = reinterpret_cast<const float4*>((const char*)a.in + r1 * a.in_stride + par_in);
  const float w = (MODE == HOP_P2) ? 0.5f : -0.5f;
  C2 acc[4][3];
  if constexpr (MODE != HOP_P1) {
    // A in2 / w first (w = +-1/2: exact), the unweighted hops add onto it
    const float4* l0 = reinterpret_cast<const float4*>((const char*)a.in2 + r0 * a.in2_stride + par_out);
    const float4* l1 = reinterpret_cast<const float4*>((const char*)a.in2 + r1 * a.in2_stride + par_out);
    const float iw = 1.f / w;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      C2 xv[6], yv[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) xv[r] = ld(l0, l1, Vh, 6 * b + r, i);
      clover_block(a.clov, Vh, p, i, b, xv, yv);
#pragma unroll
      for (int r = 0; r < 6; ++r) acc[(6 * b + r) / 3][r % 3] = C2{dscale(yv[r].re, iw), dscale(yv[r].im, iw)};
    }
  } else {
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[s2][c] = C2{D2{bc(0.f), bc(0.f)}, D2{bc(0.f), bc(0.f)}};
  }
  hop_loop<DAG>(a, in0, in1, p, i, x, acc);
#pragma unroll
  for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[s2][c] = C2{dscale(acc[s2][c].re, w), dscale(acc[s2][c].im, w)};

  const int o0 = rhs0, o1 = rhs0 + 1;
  if constexpr (MODE == HOP_P1) {
    // out = A^{-1} (w H in), one clover block at a time, stored as formed
    float4* b0 = reinterpret_cast<float4*>((char*)a.out + o0 * a.out_stride);
    float4* b1 = reinterpret_cast<float4*>((char*)a.out + (live[1] ? o1 : o0) * a.out_stride);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      C2 xv[6], yv[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) xv[r] = acc[(6 * b + r) / 3][r % 3];
      clover_block(a.cinv, Vh, p, i, b, xv, yv);
#pragma unroll
      for (int r = 0; r < 6; ++r) st(b0, b1, live[0], live[1], Vh, 6 * b + r, i, yv[r]);
    }
  } else if constexpr (EPI == EPI_NONE) {
    float4* b0 = reinterpret_cast<float4*>((char*)a.out + o0 * a.out_stride + par_out);
    float4* b1 = reinterpret_cast<float4*>((char*)a.out + (live[1] ? o1 : o0) * a.out_stride + par_out);
#pragma unroll
    for (int k = 0; k < 12; ++k) st(b0, b1, live[0], live[1], Vh, k, i, acc[k / 3][k % 3]);
  } else if constexpr (EPI == EPI_RESID64) {
    // r = eta - out, stored, and its squared norm in double-float
    const float4* e0 = reinterpret_cast<const float4*>((const char*)a.ep_eta + r0 * a.ep_eta_stride);
    const float4* e1 = reinterpret_cast<const float4*>((const char*)a.ep_eta + r1 * a.ep_eta_stride);
    float4* b0 = reinterpret_cast<float4*>((char*)a.out + o0 * a.out_stride);
    float4* b1 = reinterpret_cast<float4*>((char*)a.out + (live[1] ? o1 : o0) * a.out_stride);
    D2 n2{bc(0.f), bc(0.f)};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const C2 e = ld(e0, e1, Vh, k, i);
      const C2 rr{dadd(e.re, dneg(acc[k / 3][k % 3].re)), dadd(e.im, dneg(acc[k / 3][k % 3].im))};
      st(b0, b1, live[0], live[1], Vh, k, i, rr);
      n2 = dfma(rr.re, rr.re, dfma(rr.im, rr.im, n2));
    }
    red[0] = (double)n2.hi.x + (double)n2.lo.x;
    red[1] = (double)n2.hi.y + (double)n2.lo.y;
  }
}

}  // namespace df2

// CTA = blockDim.x sites x blockDim.y rows of two right-hand sides (at most
// 128 threads); grid ordered as for hop_kernel.  CAP = 0: at most 255
// registers (8 warps per SM); CAP = 1: at most 168 (12 warps, some spilling).
template <int MODE, bool DAG, int EPI, int CAP>
__global__ void __launch_bounds__(128, CAP ? 3 : 2) hop_df2_kernel(const HopArgs a) {
  extern __shared__ double red_smem[];
  const unsigned per_cta = blockDim.y * 2;
  const unsigned ntile = (a.nrhs + per_cta - 1) / per_cta;
  const unsigned tile = blockIdx.x % ntile;
  const unsigned rest = blockIdx.x / ntile;
  const unsigned blk = (MODE == HOP_DW) ? (rest >> 1) : rest;
  const long i = (long)blk * blockDim.x + threadIdx.x;
  const int rhs0 = (int)(tile * blockDim.y + threadIdx.y) * 2;
  const int p = (MODE == HOP_DW) ? (int)(rest & 1) : a.p;
  record_live(a);
  bool live[2], off[2];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    off[k] = a.cg && rhs0 + k < a.nrhs && a.cg[rhs0 + k].mode != a.gate;  // gated off by the solver state
    live[k] = (i < a.g.Vh) && (rhs0 + k < a.nrhs) && !off[k];
    any |= live[k];
  }
  double red[2] = {0.0, 0.0};
  if (any) df2::site<MODE, DAG, EPI>(a, i, rhs0, p, live, red);
  if constexpr (EPI != EPI_NONE) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (!live[k]) red[k] = 0.0;
    grid_reduce_nr<2>(red, a.red, rhs0, a.nrhs, red_smem, blk, gridDim.x / ntile, off);
  }
}

template <int MODE, bool DAG, int EPI>
static cudaError_t launch_df2_one(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  if (L.bx % 32 != 0 || L.bx * L.by > 128 || L.by < 1) return cudaErrorInvalidValue;
  dim3 block(L.bx, L.by, 1);
  const unsigned nb = (unsigned)((a.g.Vh + L.bx - 1) / L.bx);
  const unsigned ntile = (unsigned)((a.nrhs + L.by * 2 - 1) / (L.by * 2));
  dim3 grid((MODE == HOP_DW ? 2u * nb : nb) * ntile, 1u, 1u);
  const size_t smem = (EPI == EPI_NONE) ? 0 : sizeof(double) * (L.bx / 32) * L.by * 2;
  if (L.regcap)
    hop_df2_kernel<MODE, DAG, EPI, 1><<<grid, block, smem, s>>>(a);
  else
    hop_df2_kernel<MODE, DAG, EPI, 0><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool DAG>
static cudaError_t df2_dispatch_mode_epi(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  switch (L.mode) {
    case HOP_DW:
      if (L.epi == EPI_NONE) return launch_df2_one<HOP_DW, DAG, EPI_NONE>(L, a, s);
      break;
    case HOP_P1:
      if (L.epi == EPI_NONE) return launch_df2_one<HOP_P1, DAG, EPI_NONE>(L, a, s);
      break;
    case HOP_P2:
      if (L.epi == EPI_NONE) return launch_df2_one<HOP_P2, DAG, EPI_NONE>(L, a, s);
      if (L.epi == EPI_RESID64) return launch_df2_one<HOP_P2, DAG, EPI_RESID64>(L, a, s);
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace oq
