// Multi-right-hand-side form of the Wilson-clover stencil (binary32
// arithmetic, F32 / BF16 / F16 spinor storage).
//
// One thread computes one output site for NR right-hand sides (NR even).
// What depends only on the site is done once for all NR: coordinates and
// neighbour indices (32-bit, by multiplication with precomputed
// reciprocals), the eight link loads and their 12-real reconstruction, and
// the clover block loads.  The spinor arithmetic runs on pairs of
// right-hand sides with the two-lane binary32 FMA / ADD / MUL of sm_100-class
// GPUs (one instruction for both right-hand sides, per-lane results equal
// to the scalar fmaf / fadd / fmul).  The operator, its modes and epilogues
// are those of hop_kernel (hop_impl.cuh):
//
//   HOP_DW : out = A in2 - 1/2 H in
//   HOP_P1 : out = A^{-1} (-1/2 H in)
//   HOP_P2 : out = A in2 + 1/2 H in
//
// with H the hopping term of Eq. (2.2) (projectors swapped for the adjoint),
// the time-boundary factor on hops across x0 = T-1 <-> 0, and the norm / CG
// update epilogues with deterministic binary64 grid reductions.
#pragma once
#include <type_traits>

#include "reduce.cuh"

namespace oq {
namespace mr {

typedef float2 F2;

__device__ __forceinline__ F2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add(F2 a, F2 b) { return __fadd2_rn(a, b); }
// a - b as a + (-1) b: one rounding, the same value as fsub
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return __ffma2_rn(b, bc(-1.f), a); }
__device__ __forceinline__ F2 mul(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 ffma(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }

// a complex number of two right-hand sides (lane x: first, lane y: second)
struct C2 {
  F2 re, im;
};
struct Sp2 {
  C2 c[4][3];  // [spin][colour]
};
struct Hs2 {
  C2 c[2][3];
};

__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {sub(a.re, b.re), sub(a.im, b.im)}; }
// a + i b, a - i b
__device__ __forceinline__ C2 cadd_i(C2 a, C2 b) { return {sub(a.re, b.im), add(a.im, b.re)}; }
__device__ __forceinline__ C2 csub_i(C2 a, C2 b) { return {add(a.re, b.im), sub(a.im, b.re)}; }

// spinor of site j, 32-bit offsets (chunk c at c*Vh + j)
template <int P>
__device__ __forceinline__ void load_sp(const char* base, uint32_t Vh, uint32_t j, Spinor<float>& s) {
  cx<float>* f = &s.c[0][0];
  if constexpr (P == P_F32) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float4 v = __ldg(b + (c * Vh + j));
      f[2 * c] = cx<float>{v.x, v.y};
      f[2 * c + 1] = cx<float>{v.z, v.w};
    }
  } else {
    const uint4* b = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 v = __ldg(b + (c * Vh + j));
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 z = (P == P_BF16) ? unpack_bf16x2(w[k]) : unpack_f16x2(w[k]);
        f[4 * c + k] = cx<float>{z.x, z.y};
      }
    }
  }
}

template <int P>
__device__ __forceinline__ void store_sp(char* base, uint32_t Vh, uint32_t i, const Spinor<float>& s) {
  const cx<float>* f = &s.c[0][0];
  if constexpr (P == P_F32) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; ++c)
      b[c * Vh + i] = make_float4(f[2 * c].re, f[2 * c].im, f[2 * c + 1].re, f[2 * c + 1].im);
  } else {
    uint4* b = reinterpret_cast<uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        w[k] = (P == P_BF16) ? pack_bf16x2(f[4 * c + k].re, f[4 * c + k].im)
                             : pack_f16x2(f[4 * c + k].re, f[4 * c + k].im);
      b[c * Vh + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// A site's spinor as loaded (16-byte chunks, not yet converted): 6 float4
// (F32) or 3 uint4 (BF16/F16); component k (= 3 spin + colour) on demand.
template <int P>
struct RawSp {
  static constexpr int NC = P == P_F32 ? 6 : 3;
  uint4 ch[NC];
  __device__ __forceinline__ void load(const char* base, uint32_t Vh, uint32_t j) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int c = 0; c < NC; ++c) ch[c] = __ldg(b + (c * Vh + j));
  }
  __device__ __forceinline__ cx<float> get(int k) const {
    if constexpr (P == P_F32) {
      const uint4 v = ch[k / 2];
      return (k & 1) ? cx<float>{__uint_as_float(v.z), __uint_as_float(v.w)}
                     : cx<float>{__uint_as_float(v.x), __uint_as_float(v.y)};
    } else {
      const uint4 v = ch[k / 4];
      const uint32_t w = (k % 4 == 0) ? v.x : (k % 4 == 1) ? v.y : (k % 4 == 2) ? v.z : v.w;
      const float2 z = (P == P_BF16) ? unpack_bf16x2(w) : unpack_f16x2(w);
      return cx<float>{z.x, z.y};
    }
  }
};

// Per-thread staging of the next hop's operands in shared memory: 16-byte
// asynchronous copies (cp.async) that hold no register while in flight.  A
// thread reads back only the slots it filled itself, so waiting for its own
// copy groups suffices (no barrier).  A thread's slots are contiguous (slot
// k of stage st at offset st * nslot + k, a compile-time constant) and the
// slot count per thread is odd, so the 8 threads of a 128-byte phase of a
// warp's 16-byte access fall in distinct bank groups.
__device__ __forceinline__ void cp16(uint4* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
struct Stage {
  uint4* mine;  // this thread's first slot
  __device__ __forceinline__ uint4* at(int st, int k, int nslot) const { return mine + (st * nslot + k); }
};

// squared norm of a site's binary32 spinor, summed in binary32
__device__ __forceinline__ float norm2f(const Spinor<float>& s) {
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc = fmaf(s.c[k][c].re, s.c[k][c].re, fmaf(s.c[k][c].im, s.c[k][c].im, acc));
  return acc;
}

__device__ __forceinline__ void join(const Spinor<float>& a, const Spinor<float>& b, Sp2& s) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s.c[k][c].re = make_float2(a.c[k][c].re, b.c[k][c].re);
      s.c[k][c].im = make_float2(a.c[k][c].im, b.c[k][c].im);
    }
}

template <int LANE>
__device__ __forceinline__ void lane(const Sp2& s, Spinor<float>& a) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      a.c[k][c] = LANE == 0 ? cx<float>{s.c[k][c].re.x, s.c[k][c].im.x} : cx<float>{s.c[k][c].re.y, s.c[k][c].im.y};
}

// link U_mu at eo site i of parity p (binary32, 18 or 12 reals), 32-bit offsets
template <int FMT>
__device__ __forceinline__ void load_u(const void* base, uint32_t Vh, int p, int mu, uint32_t i, Su3<float>& u) {
  if constexpr (FMT == LINK_18) {
    const float2* b = reinterpret_cast<const float2*>(base) + (size_t)((p * 4 + mu) * 9) * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float2 v = __ldg(b + (k * Vh + i));
      u.m[k / 3][k % 3] = cx<float>{v.x, v.y};
    }
  } else {
    const float4* b = reinterpret_cast<const float4*>(base) + (size_t)((p * 4 + mu) * 3) * Vh;
    const float4 a0 = __ldg(b + i), a1 = __ldg(b + (Vh + i)), a2 = __ldg(b + (2 * Vh + i));
    u.m[0][0] = {a0.x, a0.y};
    u.m[0][1] = {a0.z, a0.w};
    u.m[0][2] = {a1.x, a1.y};
    u.m[1][0] = {a1.z, a1.w};
    u.m[1][1] = {a2.x, a2.y};
    u.m[1][2] = {a2.z, a2.w};
    // row 2 = conj(row0 x row1)
    u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
    u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
    u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
  }
}

// 12-real link from its three 16-byte chunks (rows 0, 1 stored, row 2 rebuilt)
__device__ __forceinline__ void link12_from(const float4 a0, const float4 a1, const float4 a2, Su3<float>& u) {
  u.m[0][0] = {a0.x, a0.y};
  u.m[0][1] = {a0.z, a0.w};
  u.m[0][2] = {a1.x, a1.y};
  u.m[1][0] = {a1.z, a1.w};
  u.m[1][1] = {a2.x, a2.y};
  u.m[1][2] = {a2.z, a2.w};
  u.m[2][0] = conj(u.m[0][1] * u.m[1][2] - u.m[0][2] * u.m[1][1]);
  u.m[2][1] = conj(u.m[0][2] * u.m[1][0] - u.m[0][0] * u.m[1][2]);
  u.m[2][2] = conj(u.m[0][0] * u.m[1][1] - u.m[0][1] * u.m[1][0]);
}

// acc[.][a] += wt * reconstruction (projector 1 -/+ g_mu, S = -1 / +1) of
// the transported colour-a components h0, h1 (spins 0, 1): every update is
// one FMA with +-wt (wt = the hop weight +-1/2, times the time-boundary
// factor for mu = 0).  The lower components are l0, l1 of the projector's
// reconstruction: mu = 0: (h0, h1); 1: (-i h1, -i h0); 2: (-h1, h0);
// 3: (-i h0, i h1); all negated for S = +1.
template <int MU, int S>
__device__ __forceinline__ void accum_col(Sp2& acc, int a, const C2& h0, const C2& h1, F2 wt) {
  const F2 nw = mul(wt, bc(-1.f));
  const F2 pos = S < 0 ? wt : nw, neg = S < 0 ? nw : wt;
  acc.c[0][a] = {ffma(wt, h0.re, acc.c[0][a].re), ffma(wt, h0.im, acc.c[0][a].im)};
  acc.c[1][a] = {ffma(wt, h1.re, acc.c[1][a].re), ffma(wt, h1.im, acc.c[1][a].im)};
  C2& l0 = acc.c[2][a];
  C2& l1 = acc.c[3][a];
  if constexpr (MU == 0) {
    l0 = {ffma(pos, h0.re, l0.re), ffma(pos, h0.im, l0.im)};
    l1 = {ffma(pos, h1.re, l1.re), ffma(pos, h1.im, l1.im)};
  } else if constexpr (MU == 1) {
    l0 = {ffma(pos, h1.im, l0.re), ffma(neg, h1.re, l0.im)};
    l1 = {ffma(pos, h0.im, l1.re), ffma(neg, h0.re, l1.im)};
  } else if constexpr (MU == 2) {
    l0 = {ffma(neg, h1.re, l0.re), ffma(neg, h1.im, l0.im)};
    l1 = {ffma(pos, h0.re, l1.re), ffma(pos, h0.im, l1.im)};
  } else {
    l0 = {ffma(pos, h0.im, l0.re), ffma(neg, h0.re, l0.im)};
    l1 = {ffma(neg, h1.im, l1.re), ffma(pos, h1.re, l1.im)};
  }
}

// Binary16 spin projection from the stored halves: a +/- b of two binary16
// parts as one exact conversion and one mixed-precision add (binary16 operand,
// binary32 result, one rounding) -- the same value as converting both parts
// and adding in binary32, with one conversion instead of two.
// hi: the imaginary part (upper half of the packed word).
__device__ __forceinline__ unsigned short half_of(uint32_t w, bool hi) {
  return (unsigned short)(hi ? (w >> 16) : (w & 0xffffu));
}
template <bool AHI, bool BHI, bool PLUS>
__device__ __forceinline__ float mix_f16(uint32_t wa, uint32_t wb) {
  const unsigned short a = half_of(wa, AHI), b = half_of(wb, BHI);
  float d, t;
  if constexpr (PLUS) {
    asm("cvt.f32.f16 %0, %1;" : "=f"(t) : "h"(a));
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(b), "f"(t));
  } else {
    asm("cvt.f32.f16 %0, %1;" : "=f"(t) : "h"(b));
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(t));
  }
  return d;
}
__device__ __forceinline__ uint32_t word_of(const RawSp<P_F16>& n, int k) {
  const uint4 v = n.ch[k / 4];
  return (k % 4 == 0) ? v.x : (k % 4 == 1) ? v.y : (k % 4 == 2) ? v.z : v.w;
}
// h = upper (spin U) + or - the partner (spin L), straight (re with re) or
// crossed (re with im: the factor i of the projector); SRE / SIM the signs
template <int U, int L, bool CROSS, int SRE, int SIM>
__device__ __forceinline__ C2 proj_f16(const RawSp<P_F16>& n0, const RawSp<P_F16>& n1, int a) {
  const uint32_t u0 = word_of(n0, 3 * U + a), l0 = word_of(n0, 3 * L + a);
  const uint32_t u1 = word_of(n1, 3 * U + a), l1 = word_of(n1, 3 * L + a);
  C2 h;
  h.re = make_float2(mix_f16<false, CROSS, (SRE > 0)>(u0, l0), mix_f16<false, CROSS, (SRE > 0)>(u1, l1));
  h.im = make_float2(mix_f16<true, !CROSS, (SIM > 0)>(u0, l0), mix_f16<true, !CROSS, (SIM > 0)>(u1, l1));
  return h;
}

// One hop for a pair of right-hand sides, with little live state: the
// projection reads the loaded chunks (n0, n1) directly, and each colour row
// of U h (or U^dag h) is accumulated into acc as soon as it is formed, so
// neither the converted neighbour spinor nor the transported half spinor is
// held whole.  Same linear maps as project, su3 and accum_col.
// MIX (binary16 only): the projection by mixed-precision adds (proj_f16);
// the kernels with the CG-update epilogue keep the converting form, which
// needs fewer registers there
template <int P, int MU, int S, bool UD, bool MIX = true>
__device__ __forceinline__ void hop_pair(const Su3<float>& u, const RawSp<P>& n0, const RawSp<P>& n1, Sp2& acc,
                                         F2 wt) {
  Hs2 h;
  if constexpr (P == P_F16 && MIX) {
    // the projectors' tables (as for the binary32 forms below): partner spin,
    // crossing by the factor i, signs of the real and imaginary parts
    constexpr int SP = S < 0 ? +1 : -1, SM = -SP;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if constexpr (MU == 0) {
        h.c[0][a] = proj_f16<0, 2, false, SP, SP>(n0, n1, a);
        h.c[1][a] = proj_f16<1, 3, false, SP, SP>(n0, n1, a);
      } else if constexpr (MU == 1) {
        h.c[0][a] = proj_f16<0, 3, true, SM, SP>(n0, n1, a);
        h.c[1][a] = proj_f16<1, 2, true, SM, SP>(n0, n1, a);
      } else if constexpr (MU == 2) {
        h.c[0][a] = proj_f16<0, 3, false, SP, SP>(n0, n1, a);
        h.c[1][a] = proj_f16<1, 2, false, SM, SM>(n0, n1, a);
      } else {
        h.c[0][a] = proj_f16<0, 2, true, SM, SP>(n0, n1, a);
        h.c[1][a] = proj_f16<1, 3, true, SP, SM>(n0, n1, a);
      }
    }
  } else {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    C2 pc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const cx<float> z0 = n0.get(3 * s + a), z1 = n1.get(3 * s + a);
      pc[s] = {make_float2(z0.re, z1.re), make_float2(z0.im, z1.im)};
    }
    if constexpr (MU == 0) {
      if constexpr (S < 0) { h.c[0][a] = cadd(pc[0], pc[2]); h.c[1][a] = cadd(pc[1], pc[3]); }
      else                 { h.c[0][a] = csub(pc[0], pc[2]); h.c[1][a] = csub(pc[1], pc[3]); }
    } else if constexpr (MU == 1) {
      if constexpr (S < 0) { h.c[0][a] = cadd_i(pc[0], pc[3]); h.c[1][a] = cadd_i(pc[1], pc[2]); }
      else                 { h.c[0][a] = csub_i(pc[0], pc[3]); h.c[1][a] = csub_i(pc[1], pc[2]); }
    } else if constexpr (MU == 2) {
      if constexpr (S < 0) { h.c[0][a] = cadd(pc[0], pc[3]); h.c[1][a] = csub(pc[1], pc[2]); }
      else                 { h.c[0][a] = csub(pc[0], pc[3]); h.c[1][a] = cadd(pc[1], pc[2]); }
    } else {
      if constexpr (S < 0) { h.c[0][a] = cadd_i(pc[0], pc[2]); h.c[1][a] = csub_i(pc[1], pc[3]); }
      else                 { h.c[0][a] = csub_i(pc[0], pc[2]); h.c[1][a] = cadd_i(pc[1], pc[3]); }
    }
  }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    C2 t[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C2 y;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float ur = UD ? u.m[b][a].re : u.m[a][b].re;
        const float ui = UD ? -u.m[b][a].im : u.m[a][b].im;
        const C2 x = h.c[s][b];
        if (b == 0) {
          y.re = mul(bc(ur), x.re);
          y.im = mul(bc(ur), x.im);
        } else {
          y.re = ffma(bc(ur), x.re, y.re);
          y.im = ffma(bc(ur), x.im, y.im);
        }
        y.re = ffma(bc(-ui), x.im, y.re);
        y.im = ffma(bc(ui), x.re, y.im);
      }
      t[s] = y;
    }
    accum_col<MU, S>(acc, a, t[0], t[1], wt);
  }
}

// One Hermitian 6x6 clover block of a site (binary32 storage: 6 diagonal
// reals, then 15 upper off-diagonal complex entries row by row).
struct Blk {
  float d[6];
  cx<float> off[15];
};

__device__ __forceinline__ void load_blk(const void* base, uint32_t Vh, int p, int b, uint32_t i, Blk& k) {
  const float4* q = reinterpret_cast<const float4*>(base) + (size_t)(p * 18) * Vh;
  float r[36];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const float4 w = __ldg(q + ((9 * b + c) * Vh + i));
    r[4 * c] = w.x;
    r[4 * c + 1] = w.y;
    r[4 * c + 2] = w.z;
    r[4 * c + 3] = w.w;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) k.d[c] = r[c];
#pragma unroll
  for (int c = 0; c < 15; ++c) k.off[c] = cx<float>{r[6 + 2 * c], r[7 + 2 * c]};
}

__device__ __forceinline__ void blk_from(const float4 (&w)[9], Blk& k) {
  float r[36];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    r[4 * c] = w[c].x;
    r[4 * c + 1] = w[c].y;
    r[4 * c + 2] = w[c].z;
    r[4 * c + 3] = w[c].w;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) k.d[c] = r[c];
#pragma unroll
  for (int c = 0; c < 15; ++c) k.off[c] = cx<float>{r[6 + 2 * c], r[7 + 2 * c]};
}

// y = K x for one block (x, y: the 6 components 3*spin_local + colour)
__device__ __forceinline__ void blk_apply(const Blk& k, const C2* x, C2* y) {
#pragma unroll
  for (int r = 0; r < 6; ++r) y[r] = {mul(bc(k.d[r]), x[r].re), mul(bc(k.d[r]), x[r].im)};
  int n = 0;
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = r + 1; c < 6; ++c) {
      const cx<float> o = k.off[n++];
      // y[r] += o x[c]
      y[r].re = ffma(bc(o.re), x[c].re, ffma(bc(-o.im), x[c].im, y[r].re));
      y[r].im = ffma(bc(o.re), x[c].im, ffma(bc(o.im), x[c].re, y[r].im));
      // y[c] += conj(o) x[r]
      y[c].re = ffma(bc(o.re), x[r].re, ffma(bc(o.im), x[r].im, y[c].re));
      y[c].im = ffma(bc(o.re), x[r].im, ffma(bc(-o.im), x[r].re, y[c].im));
    }
}

// eo coordinates of site i (parity p), 32-bit
__device__ __forceinline__ void coords(const Geom& g, int p, uint32_t i, int x[4]) {
  uint32_t q = geom_div(i, g.dm[0], g.ds[0]);
  const int k = (int)(i - q * (uint32_t)g.Lh3);
  uint32_t t = q;
  q = geom_div(t, g.dm[1], g.ds[1]);
  x[2] = (int)(t - q * (uint32_t)g.L[2]);
  t = q;
  q = geom_div(t, g.dm[2], g.ds[2]);
  x[1] = (int)(t - q * (uint32_t)g.L[1]);
  x[0] = (int)q;
  x[3] = 2 * k + ((p + x[0] + x[1] + x[2]) & 1);
}

// Per-thread work of hop_mr_kernel: the NR/2 lane pairs of one output site.
// PF: the operands of hop k + 1 (neighbour spinors of the NR right-hand
// sides and the 12-real link) are copied into the thread's shared-memory
// stage (k + 1) % 2 while hop k is computed, and pass 1 stages its inverse
// clover blocks the same way after the last hop (stg: 2 stages of
// NR * chunks + 3 slots).  Staged pass 2 and Dw first copy in2 (into
// NR * chunks / 2 extra slots of each stage) and the two clover blocks (into
// the stages' hop slots) and form A in2 from there before the hops, the
// summation order of the unstaged kernel; hop 0's operands are copied once
// block 0 has been read.
template <int P, int FMT, int MODE, bool DAG, int EPI, int NR, bool PF>
__device__ __forceinline__ void site(const HopArgs& a, uint32_t i, int rhs0, int p, const bool (&live)[NR],
                                     float (&red)[NR], const Stage& stg) {
  static_assert(!PF || FMT == LINK_12, "staged hops read 12-real links");
  constexpr int NP = NR / 2;
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
  const Geom& g = a.g;
  const uint32_t Vh = (uint32_t)g.Vh;
  int x[4];
  coords(g, p, i, x);
  // neighbour eo indices: a hop along mu = 0, 1, 2 moves the lexicographic
  // index by an even stride (L[3] is even), i.e. the eo index by half of it;
  // along mu = 3 the eo index is that of the row start plus x3' / 2
  const uint32_t s2 = (uint32_t)g.Lh3, s1 = s2 * (uint32_t)g.L[2], s0 = s1 * (uint32_t)g.L[1];
  const uint32_t st[3] = {s0, s1, s2};
  uint32_t jf[4], jb[4];
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const uint32_t wrap = (uint32_t)(g.L[mu] - 1) * st[mu];
    jf[mu] = x[mu] == g.L[mu] - 1 ? i - wrap : i + st[mu];
    jb[mu] = x[mu] == 0 ? i + wrap : i - st[mu];
  }
  // C* boundaries: a wrapped hop along x2 or x3 also moves x1 by half its extent
  const uint32_t h1 = (uint32_t)(g.L[1] >> 1) * s1;
  const uint32_t dcs = x[1] < (g.L[1] >> 1) ? h1 : (uint32_t)0 - h1;
  if (g.cs_shift & 4) {
    if (x[2] == g.L[2] - 1) jf[2] += dcs;
    if (x[2] == 0) jb[2] += dcs;
  }
  {
    const uint32_t row = i - (uint32_t)(x[3] >> 1);
    const int xf = x[3] + 1 == g.L[3] ? 0 : x[3] + 1;
    const int xb = x[3] == 0 ? g.L[3] - 1 : x[3] - 1;
    const uint32_t s3 = (g.cs_shift & 8) ? dcs : 0u;
    jf[3] = row + (uint32_t)(xf >> 1) + (x[3] + 1 == g.L[3] ? s3 : 0u);
    jb[3] = row + (uint32_t)(xb >> 1) + (x[3] == 0 ? s3 : 0u);
  }
  const F2 sf = bc(x[0] == g.L[0] - 1 ? g.bc_t : 1.f);  // forward time hop crosses the boundary
  const F2 sb = bc(x[0] == 0 ? g.bc_t : 1.f);

  const long par_in = (MODE == HOP_DW) ? (long)(1 - p) * a.half_bytes : 0;
  const long par_out = (MODE == HOP_DW) ? (long)p * a.half_bytes : 0;
  const char* in[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const int r = rhs0 + k < a.nrhs ? rhs0 + k : a.nrhs - 1;  // clamp: lanes past nrhs are not stored
    in[k] = (const char*)a.in + (long)r * a.in_stride + par_in;
  }

  // staged operands of hop H (mu = H / 2, forward for even H)
  constexpr int SC = RawSp<P>::NC;
  constexpr int NSLOT = NR * SC + 3;
  constexpr bool LOC = PF && MODE != HOP_P1;  // in2 and the blocks of A staged too
  // staged pass 2 and Dw: each stage has E more slots, which hold half of in2
  constexpr int E = LOC ? NR * SC / 2 : 0;
  constexpr int NS = NSLOT + E;  // slots per stage
  auto prefetch = [&](auto h_c, int st) {
    constexpr int H = decltype(h_c)::value;
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    const uint32_t j = FWD ? jf[MU] : jb[MU];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int c = 0; c < SC; ++c)
        cp16(stg.at(st, k * SC + c, NS), reinterpret_cast<const uint4*>(in[k]) + (c * Vh + j));
    const float4* b = reinterpret_cast<const float4*>(a.links) + (size_t)(((FWD ? p : 1 - p) * 4 + MU) * 3) * Vh;
    const uint32_t li = FWD ? i : j;
#pragma unroll
    for (int c = 0; c < 3; ++c) cp16(stg.at(st, NR * SC + c, NS), b + (c * Vh + li));
    cp_commit();
  };
  // clover block b of this site (9 chunks) into slots off .. off + 8 of stage st
  auto copy_blk = [&](const void* base, int b, int st, int off) {
    const float4* q = reinterpret_cast<const float4*>(base) + (size_t)(p * 18) * Vh;
#pragma unroll
    for (int c = 0; c < 9; ++c) cp16(stg.at(st, off + c, NS), q + ((9 * b + c) * Vh + i));
  };
  auto prefetch_blk = [&](const void* base, int b, int st) {
    copy_blk(base, b, st, 0);
    cp_commit();
  };
  // chunk f of in2 (f = k * SC + c for right-hand side k): the last E slots of stage f / E
  auto loc_at = [&](int f) { return f < E ? stg.at(0, NSLOT + f, NS) : stg.at(1, NSLOT + f - E, NS); };
  if constexpr (LOC) {
    // in2 and clover block 0 (into stage 0's hop slots), then block 1 (stage 1's)
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int r = rhs0 + k < a.nrhs ? rhs0 + k : a.nrhs - 1;
      const uint4* l = reinterpret_cast<const uint4*>((const char*)a.in2 + (long)r * a.in2_stride + par_out);
#pragma unroll
      for (int c = 0; c < SC; ++c) cp16(loc_at(k * SC + c), l + (c * Vh + i));
    }
    copy_blk(a.clov, 0, 0, 0);
    cp_commit();
    copy_blk(a.clov, 1, 1, 0);
    cp_commit();
  } else if constexpr (PF) {
    prefetch(std::integral_constant<int, 0>{}, 0);
  }

  // The weighted hops accumulate onto acc: for pass 2 and Dw onto A in2,
  // formed first while few registers are live (the site-local spinors stay
  // in their loaded chunks until their clover block is multiplied), for
  // pass 1 onto zero, then multiplied by A^{-1}.
  const F2 w = bc(MODE == HOP_P2 ? 0.5f : -0.5f);
  Sp2 acc[NP];
  if constexpr (LOC) {
    // acc = A in2, block b from stage b; hop 0's operands are copied into
    // stage 0 once block 0 has been read, in flight while block 1 is applied
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      cp_wait<1>();
      float4 w9[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) w9[c] = *reinterpret_cast<const float4*>(stg.at(b, c, NS));
      if (b == 0) prefetch(std::integral_constant<int, 0>{}, 0);
      Blk k;
      blk_from(w9, k);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        RawSp<P> l0, l1;
#pragma unroll
        for (int c = 0; c < SC; ++c) {
          l0.ch[c] = *loc_at((2 * q) * SC + c);
          l1.ch[c] = *loc_at((2 * q + 1) * SC + c);
        }
        C2 xv[6], yv[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          const cx<float> z0 = l0.get(6 * b + r), z1 = l1.get(6 * b + r);
          xv[r] = {make_float2(z0.re, z1.re), make_float2(z0.im, z1.im)};
        }
        blk_apply(k, xv, yv);
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[q].c[2 * b + r / 3][r % 3] = yv[r];
      }
    }
  } else if constexpr (MODE == HOP_P1) {
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[q].c[s][c] = {bc(0.f), bc(0.f)};
  } else {
    RawSp<P> loc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int r = rhs0 + k < a.nrhs ? rhs0 + k : a.nrhs - 1;
      loc[k].load((const char*)a.in2 + (long)r * a.in2_stride + par_out, Vh, i);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      Blk k;
      load_blk(a.clov, Vh, p, b, i, k);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        C2 xv[6], yv[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          const cx<float> z0 = loc[2 * q].get(6 * b + r), z1 = loc[2 * q + 1].get(6 * b + r);
          xv[r] = {make_float2(z0.re, z1.re), make_float2(z0.im, z1.im)};
        }
        blk_apply(k, xv, yv);
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[q].c[2 * b + r / 3][r % 3] = yv[r];
      }
    }
  }
  const F2 wf = mul(w, sf), wb = mul(w, sb);

  auto hop = [&](auto mu_c) {
    constexpr int MU = decltype(mu_c)::value;
    Su3<float> u;
    // forward: U_mu(x) (1 -/+ g) psi(x + mu)
    load_u<FMT>(a.links, Vh, p, MU, i, u);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      RawSp<P> n0, n1;
      n0.load(in[2 * q], Vh, jf[MU]);
      n1.load(in[2 * q + 1], Vh, jf[MU]);
      hop_pair<P, MU, SF, false, EPI != EPI_CG>(u, n0, n1, acc[q], MU == 0 ? wf : w);
    }
    // backward: U_mu(x - mu)^dag (1 +/- g) psi(x - mu)
    load_u<FMT>(a.links, Vh, 1 - p, MU, jb[MU], u);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      RawSp<P> n0, n1;
      n0.load(in[2 * q], Vh, jb[MU]);
      n1.load(in[2 * q + 1], Vh, jb[MU]);
      hop_pair<P, MU, -SF, true, EPI != EPI_CG>(u, n0, n1, acc[q], MU == 0 ? wb : w);
    }
  };
  // staged form: wait for hop H's copies while hop H + 1's are in flight
  auto step = [&](auto h_c) {
    constexpr int H = decltype(h_c)::value;
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    constexpr int st = H & 1;
    if constexpr (H < 7) {
      prefetch(std::integral_constant<int, H + 1>{}, (H + 1) & 1);
      cp_wait<1>();
    } else if constexpr (MODE == HOP_P1) {
      prefetch_blk(a.cinv, 0, 0);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    Su3<float> u;
    link12_from(*reinterpret_cast<const float4*>(stg.at(st, NR * SC, NS)),
                *reinterpret_cast<const float4*>(stg.at(st, NR * SC + 1, NS)),
                *reinterpret_cast<const float4*>(stg.at(st, NR * SC + 2, NS)), u);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      RawSp<P> n0, n1;
#pragma unroll
      for (int c = 0; c < SC; ++c) {
        n0.ch[c] = *stg.at(st, (2 * q) * SC + c, NS);
        n1.ch[c] = *stg.at(st, (2 * q + 1) * SC + c, NS);
      }
      hop_pair<P, MU, FWD ? SF : -SF, !FWD, EPI != EPI_CG>(u, n0, n1, acc[q], MU == 0 ? (FWD ? wf : wb) : w);
    }
  };
  if constexpr (PF) {
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
    step(std::integral_constant<int, 2>{});
    step(std::integral_constant<int, 3>{});
    step(std::integral_constant<int, 4>{});
    step(std::integral_constant<int, 5>{});
    step(std::integral_constant<int, 6>{});
    step(std::integral_constant<int, 7>{});
  } else {
    hop(std::integral_constant<int, 0>{});
    hop(std::integral_constant<int, 1>{});
    hop(std::integral_constant<int, 2>{});
    hop(std::integral_constant<int, 3>{});
  }

  Sp2 (&res)[NP] = acc;
  if constexpr (MODE == HOP_P1 && PF) {
    // res = A^{-1} (w H in): block 0 was staged with the last hop, block 1
    // is staged while block 0 is applied
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (b == 0) {
        prefetch_blk(a.cinv, 1, 1);
        cp_wait<1>();
      } else {
        cp_wait<0>();
      }
      float4 w9[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) w9[c] = *reinterpret_cast<const float4*>(stg.at(b, c, NS));
      Blk k;
      blk_from(w9, k);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        C2 xv[6], yv[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) xv[r] = acc[q].c[2 * b + r / 3][r % 3];
        blk_apply(k, xv, yv);
#pragma unroll
        for (int r = 0; r < 6; ++r) res[q].c[2 * b + r / 3][r % 3] = yv[r];
      }
    }
  } else if constexpr (MODE == HOP_P1) {
    // res = A^{-1} (w H in), in place one clover block at a time
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      Blk k;
      load_blk(a.cinv, Vh, p, b, i, k);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        C2 xv[6], yv[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) xv[r] = acc[q].c[2 * b + r / 3][r % 3];
        blk_apply(k, xv, yv);
#pragma unroll
        for (int r = 0; r < 6; ++r) res[q].c[2 * b + r / 3][r % 3] = yv[r];
      }
    }
  }

  if constexpr (EPI == EPI_NONE || EPI == EPI_NORM) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      Spinor<float> o0, o1;
      lane<0>(res[q], o0);
      lane<1>(res[q], o1);
      if (live[2 * q]) store_sp<P>((char*)a.out + (long)(rhs0 + 2 * q) * a.out_stride + par_out, Vh, i, o0);
      if (live[2 * q + 1])
        store_sp<P>((char*)a.out + (long)(rhs0 + 2 * q + 1) * a.out_stride + par_out, Vh, i, o1);
      if constexpr (EPI == EPI_NORM) {
        red[2 * q] = norm2f(o0);
        red[2 * q + 1] = norm2f(o1);
      }
    }
  } else if constexpr (EPI == EPI_CG) {
    // q = res; x += alpha p (x binary32); r -= alpha q; norm of the stored r.
    // One right-hand side at a time, from the loaded chunks, so that little
    // besides the result stays live.
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int rr = rhs0 + k < a.nrhs ? rhs0 + k : a.nrhs - 1;
      const float al = (float)a.cg[rr].alpha;
      RawSp<P> pv, rv;
      RawSp<P_F32> xv;
      pv.load((const char*)a.ep_p + (long)rr * a.ep_p_stride, Vh, i);
      rv.load((const char*)a.ep_r + (long)rr * a.ep_r_stride, Vh, i);
      xv.load((const char*)a.ep_x + (long)rr * a.ep_x_stride, Vh, i);
      Spinor<float> xo, ro;
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        const C2 qv = res[k / 2].c[m / 3][m % 3];
        const float qre = (k & 1) ? qv.re.y : qv.re.x, qim = (k & 1) ? qv.im.y : qv.im.x;
        const cx<float> pm = pv.get(m), rm = rv.get(m), xm = xv.get(m);
        xo.c[m / 3][m % 3] = cx<float>{fmaf(al, pm.re, xm.re), fmaf(al, pm.im, xm.im)};
        ro.c[m / 3][m % 3] = cx<float>{fmaf(-al, qre, rm.re), fmaf(-al, qim, rm.im)};
      }
      round_trip<P>(ro);
      if (live[k]) {
        store_sp<P_F32>((char*)a.ep_x + (long)rr * a.ep_x_stride, Vh, i, xo);
        store_sp<P>((char*)a.ep_r + (long)rr * a.ep_r_stride, Vh, i, ro);
        red[k] = norm2f(ro);
      }
    }
  }
}

}  // namespace mr

// CTA = blockDim.x sites x blockDim.y groups of NR right-hand sides
// (at most 128 threads); grid ordered as for hop_kernel (rhs tiles of one
// site block adjacent).  CAP = 1 caps the registers (128 for NR = 2, 168 for
// NR = 4: at least 16 / 12 warps per SM, with some spilling); CAP = 0 lets
// the compiler keep all neighbour loads of a site in flight.
// CAP = 2: the register cap of CAP = 1 and the hop operands staged in
// shared memory (site<..., PF = true>; 12-real links only).  CAP = 3 (NR = 2):
// staged with the cap of 168 registers (12 warps per SM): fewer spills, which
// the pass-2 kernels gain more from than from the extra warps.
template <int NR, int CAP>
struct MrBounds {
  static constexpr int min_blocks = CAP == 0 ? 1 : (NR == 2 && CAP != 3) ? 4 : 3;
};
// 16-byte slots per thread of a staged launch: 2 stages of NR * chunks + 3,
// for pass 2 and Dw of NR * chunks / 2 more (the site-local spinors); rounded
// up to an odd count
template <int P, int NR, int MODE>
constexpr int mr_stage_slots() {
  constexpr int sc = P == P_F32 ? 6 : 3;
  return (2 * (NR * sc + 3 + (MODE == HOP_P1 ? 0 : NR * sc / 2))) | 1;
}
template <int P, int NR, int MODE>
constexpr size_t mr_stage_bytes(int nthr) {
  return (size_t)mr_stage_slots<P, NR, MODE>() * 16 * nthr;
}
// the per-thread slots of a launch (staged: CAP = 2, 3)
template <int P, int NR, int MODE, int CAP>
constexpr int mr_slots() {
  return CAP >= 2 ? mr_stage_slots<P, NR, MODE>() : 0;
}
template <int P, int FMT, int MODE, bool DAG, int EPI, int NR, int CAP>
__global__ void __launch_bounds__(128, (MrBounds<NR, CAP>::min_blocks)) hop_mr_kernel(const HopArgs a) {
  extern __shared__ double dyn_smem[];
  constexpr bool PF = CAP >= 2;
  constexpr int NSL = mr_slots<P, NR, MODE, CAP>();
  const uint32_t nthr = blockDim.x * blockDim.y;
  // the threads' slots first, then the reduction scratch
  double* red_smem = dyn_smem + (size_t)NSL * 16 * nthr / sizeof(double);
  mr::Stage stg{reinterpret_cast<uint4*>(dyn_smem) + (size_t)(threadIdx.y * blockDim.x + threadIdx.x) * NSL};
  const unsigned per_cta = blockDim.y * NR;
  const unsigned ntile = (a.nrhs + per_cta - 1) / per_cta;
  const unsigned tile = blockIdx.x % ntile;
  const unsigned rest = blockIdx.x / ntile;
  const unsigned blk = (MODE == HOP_DW) ? (rest >> 1) : rest;
  const uint32_t i = blk * blockDim.x + threadIdx.x;
  const int rhs0 = (int)(tile * blockDim.y + threadIdx.y) * NR;
  const int p = (MODE == HOP_DW) ? (int)(rest & 1) : a.p;
  record_live(a);
  bool live[NR], off[NR];
  bool any = false;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    off[k] = a.cg && rhs0 + k < a.nrhs && a.cg[rhs0 + k].mode != a.gate;  // gated off by the solver state
    live[k] = (i < (uint32_t)a.g.Vh) && (rhs0 + k < a.nrhs) && !off[k];
    any |= live[k];
  }
  float red[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) red[k] = 0.f;
  if (any) mr::site<P, FMT, MODE, DAG, EPI, NR, PF>(a, i, rhs0, p, live, red, stg);
  if constexpr (EPI != EPI_NONE) {
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (!live[k]) red[k] = 0.f;
    grid_reduce_nr<NR>(red, a.red, rhs0, a.nrhs, red_smem, blk, gridDim.x / ntile, off);
  }
}

// a staged launch (CAP 2, 3): the threads' slots, then `smem` bytes of
// reduction scratch; above 48 KiB the kernel is allowed the device's opt-in
// limit (once per instantiation)
template <int P, int FMT, int MODE, bool DAG, int EPI, int NR, int CAP>
static cudaError_t launch_mr_smem(dim3 grid, dim3 block, size_t smem, const HopArgs& a, cudaStream_t s) {
  const size_t bytes = smem + (size_t)mr_slots<P, NR, MODE, CAP>() * 16 * block.x * block.y;
  static bool attr = false;
  if (!attr && bytes > 48 * 1024) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(hop_mr_kernel<P, FMT, MODE, DAG, EPI, NR, CAP>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  hop_mr_kernel<P, FMT, MODE, DAG, EPI, NR, CAP><<<grid, block, bytes, s>>>(a);
  return cudaGetLastError();
}

template <int P, int FMT, int MODE, bool DAG, int EPI, int NR>
static cudaError_t launch_mr_one(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  if (L.bx % 32 != 0 || L.bx * L.by > 128 || L.by < 1) return cudaErrorInvalidValue;
  dim3 block(L.bx, L.by, 1);
  const unsigned nb = (unsigned)((a.g.Vh + L.bx - 1) / L.bx);
  const unsigned ntile = (unsigned)((a.nrhs + L.by * NR - 1) / (L.by * NR));
  dim3 grid((MODE == HOP_DW ? 2u * nb : nb) * ntile, 1u, 1u);
  const size_t smem = (EPI == EPI_NONE) ? 0 : sizeof(double) * (L.bx / 32) * L.by * NR;
  if (L.regcap == 2) {
    if constexpr (FMT == LINK_12)
      return launch_mr_smem<P, FMT, MODE, DAG, EPI, NR, 2>(grid, block, smem, a, s);
    return cudaErrorInvalidValue;
  }
  if (L.regcap == 3) {
    if constexpr (FMT == LINK_12 && NR == 2)
      return launch_mr_smem<P, FMT, MODE, DAG, EPI, NR, 3>(grid, block, smem, a, s);
    return cudaErrorInvalidValue;
  }
  if (L.regcap)
    hop_mr_kernel<P, FMT, MODE, DAG, EPI, NR, 1><<<grid, block, smem, s>>>(a);
  else
    hop_mr_kernel<P, FMT, MODE, DAG, EPI, NR, 0><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int FMT, bool DAG, int NR>
static cudaError_t mr_dispatch_mode_epi(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  switch (L.mode) {
    case HOP_DW:
      if (L.epi == EPI_NONE) return launch_mr_one<P, FMT, HOP_DW, DAG, EPI_NONE, NR>(L, a, s);
      break;
    case HOP_P1:
      if (L.epi == EPI_NONE) return launch_mr_one<P, FMT, HOP_P1, DAG, EPI_NONE, NR>(L, a, s);
      break;
    case HOP_P2:
      if (L.epi == EPI_NONE) return launch_mr_one<P, FMT, HOP_P2, DAG, EPI_NONE, NR>(L, a, s);
      if (L.epi == EPI_NORM) return launch_mr_one<P, FMT, HOP_P2, DAG, EPI_NORM, NR>(L, a, s);
      if (L.epi == EPI_CG) return launch_mr_one<P, FMT, HOP_P2, DAG, EPI_CG, NR>(L, a, s);
      break;
  }
  return cudaErrorInvalidValue;
}

template <int P, int NR>
static cudaError_t mr_dispatch(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  if (L.link_fmt == LINK_12)
    return L.dagger ? mr_dispatch_mode_epi<P, LINK_12, true, NR>(L, a, s)
                    : mr_dispatch_mode_epi<P, LINK_12, false, NR>(L, a, s);
  return L.dagger ? mr_dispatch_mode_epi<P, LINK_18, true, NR>(L, a, s)
                  : mr_dispatch_mode_epi<P, LINK_18, false, NR>(L, a, s);
}

}  // namespace oq
