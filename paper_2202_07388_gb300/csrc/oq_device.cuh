// Device-side building blocks: complex numbers, lattice geometry on the
// even-odd ordered half lattices, and the packed (chunk-major SoA) storage
// of spinors, links and clover blocks in every supported precision.
//
// Packed layouts (Vh = V/2 sites per parity; eo index i = lex(x) >> 1):
//   spinor  : 24 reals/site, stored as chunks of 16 bytes, chunk-major:
//             chunk c of site i at base[c*Vh + i].  Real index r of the site
//             vector = 2*(3*spin + colour) + (0 re | 1 im).
//             F64: 12 chunks (double2), DF64: 12 chunks (float4 = re.hi,
//             re.lo, im.hi, im.lo), F32: 6 chunks (float4), BF16/F16: 3
//             chunks (8 halves each).
//   links   : U_mu(x) at [parity(x)][mu][chunk][Vh];
//             18-real: 9 chunks (F64 double2 / DF64 float4 / F32 float2),
//             element a*3+b;
//             12-real (F32, SU(3) only): 3 float4 chunks holding rows 0 and 1,
//             row 2 = conj(row0 x row1).
//   clover  : per site two Hermitian 6x6 blocks (chirality +, -), each as
//             6 real diagonal entries then the 15 upper off-diagonal complex
//             entries in row-major order (36 reals/block, 72 reals/site);
//             F64: 36 double2 chunks, DF64: 36 float4 chunks (two reals
//             as hi, lo, hi, lo), F32: 18 float4 chunks, [parity][chunk][Vh].
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace oq {

// P_DF64: "double-float" values (an unevaluated sum hi + lo of two binary32
// numbers with |lo| <= ulp(hi)/2, ~48 significant bits) stored as (hi, lo)
// pairs in the 8 bytes of a binary64 value, with arithmetic on the binary32
// pipes, for the reset-step residuals on a GPU whose binary64 rate is far
// below its binary32 rate.  Operands are split from binary64 once (links,
// clover, the solution vector), never inside the stencil.
enum Prec : int { P_F64 = 0, P_F32 = 1, P_BF16 = 2, P_F16 = 3, P_DF64 = 4 };

// ---------------------------------------------------------------------------
// double-float arithmetic from error-free transformations: Knuth's two-sum,
// Dekker's fast two-sum and the FMA two-product.  Sums use the "sloppy"
// double-word addition (two-sum of the high parts, the low parts added,
// renormalised), whose absolute error is a few u^2 (|x| + |y|), u = 2^-24:
// the operands' own magnitudes bound every error of a stencil sum, which is
// the accuracy a residual recomputation needs.  A product is added to an
// accumulator with one renormalisation in all (Joldes, Muller, Popescu, ACM
// TOMS 44, 2017, for the building blocks).  Explicit _rn intrinsics keep the
// compiler from contracting or reassociating the compensated steps.
// ---------------------------------------------------------------------------
struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ dfloat(float a) : hi(a), lo(0.f) {}
  __host__ __device__ dfloat(int a) : hi((float)a), lo(0.f) {}
  __device__ dfloat(double a) {
    hi = __double2float_rn(a);
    lo = __double2float_rn(a - (double)hi);
  }
  __device__ dfloat(float h, float l) : hi(h), lo(l) {}
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfloat(s, e);
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) {
  x = x + y;
  return x;
}
// a * b + c: the two-product of the high parts with the cross terms, added
// to c by a two-sum of the high parts, one renormalisation at the end
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfloat s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(c.lo, e)));
}
// A dot product of double-float numbers accumulated lazily: s is the running
// sum of the high products (each added by a two-sum), e collects the
// two-sum errors and the low parts of every product in binary32; one
// renormalisation at the end.  12 binary32 operations per term instead of
// the 15 of a renormalised fma.
struct DfAcc {
  float s, e;
};
__device__ __forceinline__ void dfa_first(DfAcc& a, dfloat x, dfloat y) {  // a = x y
  a.s = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -a.s);
  e = __fmaf_rn(x.hi, y.lo, e);
  a.e = __fmaf_rn(x.lo, y.hi, e);
}
__device__ __forceinline__ void dfa_add(DfAcc& a, dfloat x, dfloat y) {  // a += x y
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const dfloat t = df_two_sum(a.s, p);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, e));
}
__device__ __forceinline__ dfloat dfa_get(const DfAcc& a) { return df_fast_two_sum(a.s, a.e); }
// x + y without the final renormalisation: the two-sum of the high parts
// and the low parts added to its error (8 operations instead of 11).  The
// low part may exceed ulp(hi)/2 by a few ulp; a product or another lazy sum
// takes such a value as it is, and df_norm restores the normal form.
__device__ __forceinline__ dfloat df_add_lazy(dfloat x, dfloat y) {
  const dfloat s = df_two_sum(x.hi, y.hi);
  return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat df_norm(dfloat x) { return df_fast_two_sum(x.hi, x.lo); }
// x * 2^k for a power of two s = 2^k: exact, both parts scaled
__device__ __forceinline__ dfloat df_scale(dfloat x, float s) { return dfloat(x.hi * s, x.lo * s); }
using ::fma;  // keep the float / double overloads visible next to the dfloat one
enum LinkFmt : int { LINK_18 = 0, LINK_12 = 1 };

// ---------------------------------------------------------------------------
// complex
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
  R re, im;
};
template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cx<R> times_mi(cx<R> a) { return {a.im, -a.re}; }
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cfmac(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}

template <typename R>
struct Spinor {
  cx<R> c[4][3];  // [spin][colour]
};
template <typename R>
struct HalfSpinor {
  cx<R> c[2][3];
};
template <typename R>
struct Su3 {
  cx<R> m[3][3];
};

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geom {
  int L[4];   // L[0] = T (slowest) ... L[3] (fastest); all even
  int Lh3;    // L[3] / 2
  long Vh;    // V / 2
  float bc_t; // fermion factor for hops across the time boundary (-1 antiperiodic)
  // 32-bit division by Lh3, L[2], L[1] (in that order) as n / d =
  // (n * dm) >> ds, exact for n < 2^31 (geom_init_div)
  uint32_t dm[3];
  int ds[3];
  // C* boundaries (orbifold form): bit mu (2 or 3) set = a hop across the
  // x_mu boundary also moves x1 by L[1] / 2 (the lattice is doubled in x1,
  // its second half holding the charge-conjugate copy)
  int cs_shift;
};

// x1 after a hop along mu that wrapped (C* boundaries shift it by half the doubled extent)
__host__ __device__ __forceinline__ int cs_x1(const Geom& g, int mu, int x1) {
  if (!((g.cs_shift >> mu) & 1)) return x1;
  const int h = g.L[1] >> 1;
  return x1 < h ? x1 + h : x1 - h;
}

// Multipliers for geom's 32-bit divisions: for d >= 1 let l be the smallest
// integer with 2^l >= d, m = ceil(2^(31+l) / d) (< 2^32) and s = 31 + l.
// With m d = 2^s + e, 0 <= e < d <= 2^l, n m / 2^s = n/d + n e / (d 2^s) and
// the second term is below 1/d for n < 2^31, so the floor is floor(n / d).
__host__ __device__ inline void geom_div_magic(uint32_t d, uint32_t* m, int* s) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  *m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
  *s = 31 + l;
}
__host__ __device__ inline void geom_init_div(Geom& g) {
  const uint32_t d[3] = {(uint32_t)g.Lh3, (uint32_t)g.L[2], (uint32_t)g.L[1]};
  for (int k = 0; k < 3; ++k) geom_div_magic(d[k], &g.dm[k], &g.ds[k]);
}
__device__ __forceinline__ uint32_t geom_div(uint32_t n, uint32_t m, int s) {
  return (uint32_t)(((unsigned long long)n * m) >> s);
}

// coordinates of eo site i of parity p
__device__ __forceinline__ void eo_coords(const Geom& g, int p, long i, int x[4]) {
  long t = i;
  int k = (int)(t % g.Lh3);
  t /= g.Lh3;
  x[2] = (int)(t % g.L[2]);
  t /= g.L[2];
  x[1] = (int)(t % g.L[1]);
  x[0] = (int)(t / g.L[1]);
  x[3] = 2 * k + ((p + x[0] + x[1] + x[2]) & 1);
}

__device__ __forceinline__ long eo_index(const Geom& g, const int x[4]) {
  long lex = (((long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
  return lex >> 1;
}

// eo index of x + d*mu (periodic wrap); *crossed = 1 if the hop crosses the
// time boundary
__device__ __forceinline__ long eo_neighbour(const Geom& g, const int x[4], int mu, int d, bool* crossed) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  int v = y[mu] + d;
  bool c = false;
  if (v == g.L[mu]) { v = 0; c = true; }
  if (v < 0) { v = g.L[mu] - 1; c = true; }
  y[mu] = v;
  if (c) y[1] = cs_x1(g, mu, y[1]);
  *crossed = c && (mu == 0);
  return eo_index(g, y);
}

// eo_neighbour for a runtime direction, without indexing a local array
__device__ __forceinline__ long eo_neighbour_rt(const Geom& g, const int x[4], int mu, int d, bool* crossed) {
  const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
  const int xm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
  int v = xm + d;
  bool c = false;
  if (v == L) { v = 0; c = true; }
  if (v < 0) { v = L - 1; c = true; }
  *crossed = c && (mu == 0);
  const int y0 = mu == 0 ? v : x[0], y2 = mu == 2 ? v : x[2], y3 = mu == 3 ? v : x[3];
  const int y1 = mu == 1 ? v : (c ? cs_x1(g, mu, x[1]) : x[1]);
  const long lex = (((long)y0 * g.L[1] + y1) * g.L[2] + y2) * g.L[3] + y3;
  return lex >> 1;
}

// ---------------------------------------------------------------------------
// storage types
// ---------------------------------------------------------------------------
template <int P> struct PrecTraits;
template <> struct PrecTraits<P_F64> { typedef double R; typedef double2 Chunk; static const int nchunk = 12; static const int bytes = 8; };
template <> struct PrecTraits<P_F32> { typedef float R;  typedef float4 Chunk;  static const int nchunk = 6;  static const int bytes = 4; };
template <> struct PrecTraits<P_BF16> { typedef float R; typedef uint4 Chunk;   static const int nchunk = 3;  static const int bytes = 2; };
template <> struct PrecTraits<P_F16> { typedef float R;  typedef uint4 Chunk;   static const int nchunk = 3;  static const int bytes = 2; };
template <> struct PrecTraits<P_DF64> { typedef dfloat R; typedef float4 Chunk;  static const int nchunk = 12; static const int bytes = 8; };

template <typename T>
__device__ __forceinline__ T ldg_nc(const T* p) { return __ldg(p); }

__device__ __forceinline__ float2 unpack_bf16x2(uint32_t w) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
  return __bfloat1622float2(h);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_f16x2(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Load the 12 complex components of site i from a packed spinor field.
template <int P>
__device__ __forceinline__ void load_spinor(const void* base, long Vh, long i,
                                            Spinor<typename PrecTraits<P>::R>& s) {
  typedef typename PrecTraits<P>::R R;
  cx<R>* f = &s.c[0][0];
  if constexpr (P == P_F64) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 v = ldg_nc(b + c * Vh + i);
      f[c] = cx<R>{R(v.x), R(v.y)};
    }
  } else if constexpr (P == P_DF64) {
    // one complex per chunk: (re.hi, re.lo, im.hi, im.lo)
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      float4 v = ldg_nc(b + c * Vh + i);
      f[c] = cx<R>{dfloat(v.x, v.y), dfloat(v.z, v.w)};
    }
  } else if constexpr (P == P_F32) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 v = ldg_nc(b + c * Vh + i);
      f[2 * c] = cx<R>{v.x, v.y};
      f[2 * c + 1] = cx<R>{v.z, v.w};
    }
  } else {
    const uint4* b = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint4 v = ldg_nc(b + c * Vh + i);
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 z = (P == P_BF16) ? unpack_bf16x2(w[k]) : unpack_f16x2(w[k]);
        f[4 * c + k] = cx<R>{z.x, z.y};
      }
    }
  }
}

template <int P>
__device__ __forceinline__ void store_spinor(void* base, long Vh, long i,
                                             const Spinor<typename PrecTraits<P>::R>& s) {
  typedef typename PrecTraits<P>::R R;
  const cx<R>* f = &s.c[0][0];
  if constexpr (P == P_F64) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; ++c) b[c * Vh + i] = make_double2((double)f[c].re, (double)f[c].im);
  } else if constexpr (P == P_DF64) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int c = 0; c < 12; ++c) b[c * Vh + i] = make_float4(f[c].re.hi, f[c].re.lo, f[c].im.hi, f[c].im.lo);
  } else if constexpr (P == P_F32) {
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

// sum of the 24 squares of one site (in the arithmetic type), as binary64
template <typename R>
__device__ __forceinline__ double site_norm2(const Spinor<R>& s) {
  R acc = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc += s.c[k][c].re * s.c[k][c].re + s.c[k][c].im * s.c[k][c].im;
  return (double)acc;
}

// Round a binary32 spinor held in registers to the storage type P and back,
// i.e. the value a store_spinor<P> / load_spinor<P> pair would give, without
// re-reading memory written by the same kernel.
template <int P, typename R>
__device__ __forceinline__ void round_trip(Spinor<R>& s) {
  if constexpr (P == P_BF16) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 z = unpack_bf16x2(pack_bf16x2(s.c[a][c].re, s.c[a][c].im));
        s.c[a][c] = cx<R>{z.x, z.y};
      }
  } else if constexpr (P == P_F16) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 z = unpack_f16x2(pack_f16x2(s.c[a][c].re, s.c[a][c].im));
        s.c[a][c] = cx<R>{z.x, z.y};
      }
  }
}

// Load link U_mu at eo site i of parity p.  R = float for F32 storage,
// double for F64 storage.
template <typename R, int FMT>
__device__ __forceinline__ void load_link(const void* base, long Vh, int p, int mu, long i, Su3<R>& u) {
  if constexpr (std::is_same<R, dfloat>::value) {
    // split binary64 links: one complex element per (re.hi, re.lo, im.hi, im.lo) chunk
    const float4* b = reinterpret_cast<const float4*>(base) + ((long)(p * 4 + mu) * 9) * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 v = ldg_nc(b + k * Vh + i);
      u.m[k / 3][k % 3] = cx<R>{dfloat(v.x, v.y), dfloat(v.z, v.w)};
    }
  } else if constexpr (sizeof(R) == 8) {
    const double2* b = reinterpret_cast<const double2*>(base) + ((long)(p * 4 + mu) * 9) * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = ldg_nc(b + k * Vh + i);
      u.m[k / 3][k % 3] = cx<R>{v.x, v.y};
    }
  } else if constexpr (FMT == LINK_18) {
    const float2* b = reinterpret_cast<const float2*>(base) + ((long)(p * 4 + mu) * 9) * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 v = ldg_nc(b + k * Vh + i);
      u.m[k / 3][k % 3] = cx<R>{v.x, v.y};
    }
  } else {
    const float4* b = reinterpret_cast<const float4*>(base) + ((long)(p * 4 + mu) * 3) * Vh;
    float4 a0 = ldg_nc(b + i), a1 = ldg_nc(b + Vh + i), a2 = ldg_nc(b + 2 * Vh + i);
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

// y = U h  (colour matvec on both spin components of a half spinor)
template <typename R>
__device__ __forceinline__ void su3_mul(const Su3<R>& u, const HalfSpinor<R>& h, HalfSpinor<R>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = u.m[a][0] * h.c[s][0];
      cfma(acc, u.m[a][1], h.c[s][1]);
      cfma(acc, u.m[a][2], h.c[s][2]);
      y.c[s][a] = acc;
    }
}

// y = U^dag h
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const Su3<R>& u, const HalfSpinor<R>& h, HalfSpinor<R>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = cmulc(u.m[0][a], h.c[s][0]);
      cfmac(acc, u.m[1][a], h.c[s][1]);
      cfmac(acc, u.m[2][a], h.c[s][2]);
      y.c[s][a] = acc;
    }
}

// double-float forms: each output real is one 6-term dot product
__device__ __forceinline__ void su3_mul(const Su3<dfloat>& u, const HalfSpinor<dfloat>& h, HalfSpinor<dfloat>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      DfAcc re, im;
      dfa_first(re, u.m[a][0].re, h.c[s][0].re);
      dfa_add(re, -u.m[a][0].im, h.c[s][0].im);
      dfa_first(im, u.m[a][0].re, h.c[s][0].im);
      dfa_add(im, u.m[a][0].im, h.c[s][0].re);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        dfa_add(re, u.m[a][b].re, h.c[s][b].re);
        dfa_add(re, -u.m[a][b].im, h.c[s][b].im);
        dfa_add(im, u.m[a][b].re, h.c[s][b].im);
        dfa_add(im, u.m[a][b].im, h.c[s][b].re);
      }
      y.c[s][a] = cx<dfloat>{dfa_get(re), dfa_get(im)};
    }
}
__device__ __forceinline__ void su3_dag_mul(const Su3<dfloat>& u, const HalfSpinor<dfloat>& h,
                                            HalfSpinor<dfloat>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      DfAcc re, im;  // sum_b conj(U_ba) h_b
      dfa_first(re, u.m[0][a].re, h.c[s][0].re);
      dfa_add(re, u.m[0][a].im, h.c[s][0].im);
      dfa_first(im, u.m[0][a].re, h.c[s][0].im);
      dfa_add(im, -u.m[0][a].im, h.c[s][0].re);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        dfa_add(re, u.m[b][a].re, h.c[s][b].re);
        dfa_add(re, u.m[b][a].im, h.c[s][b].im);
        dfa_add(im, u.m[b][a].re, h.c[s][b].im);
        dfa_add(im, -u.m[b][a].im, h.c[s][b].re);
      }
      y.c[s][a] = cx<dfloat>{dfa_get(re), dfa_get(im)};
    }
}

// ---------------------------------------------------------------------------
// clover blocks
// ---------------------------------------------------------------------------
// Multiply the two Hermitian 6x6 blocks of site i (parity p) onto psi:
// out = A psi.  Block b acts on spins 2b, 2b+1 (index 3*spin_local+colour).
template <typename R>
__device__ __forceinline__ void clover_apply(const void* base, long Vh, int p, long i,
                                             const Spinor<R>& in, Spinor<R>& out) {
  const cx<R>* v = &in.c[0][0];
  cx<R>* o = &out.c[0][0];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    R d[6];
    cx<R> off[15];
    if constexpr (std::is_same<R, dfloat>::value) {
      // split binary64 clover: chunk k holds reals 2k, 2k+1 as (hi, lo, hi, lo)
      const float4* q = reinterpret_cast<const float4*>(base) + (long)p * 36 * Vh;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float4 w = ldg_nc(q + (18 * b + k) * Vh + i);
        d[2 * k] = dfloat(w.x, w.y);
        d[2 * k + 1] = dfloat(w.z, w.w);
      }
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        float4 w = ldg_nc(q + (18 * b + 3 + k) * Vh + i);
        off[k] = cx<R>{dfloat(w.x, w.y), dfloat(w.z, w.w)};
      }
    } else if constexpr (sizeof(R) == 8) {
      const double2* q = reinterpret_cast<const double2*>(base) + (long)p * 36 * Vh;
      // block b occupies chunks 18b .. 18b+17: 3 chunks of diagonal, 15 off
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double2 w = ldg_nc(q + (18 * b + k) * Vh + i);
        d[2 * k] = w.x;
        d[2 * k + 1] = w.y;
      }
#pragma unroll
      for (int k = 0; k < 15; ++k) {
        double2 w = ldg_nc(q + (18 * b + 3 + k) * Vh + i);
        off[k] = cx<R>{w.x, w.y};
      }
    } else {
      const float4* q = reinterpret_cast<const float4*>(base) + (long)p * 18 * Vh;
      float r[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        float4 w = ldg_nc(q + (9 * b + k) * Vh + i);
        r[4 * k] = w.x;
        r[4 * k + 1] = w.y;
        r[4 * k + 2] = w.z;
        r[4 * k + 3] = w.w;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) d[k] = r[k];
#pragma unroll
      for (int k = 0; k < 15; ++k) off[k] = cx<R>{r[6 + 2 * k], r[7 + 2 * k]};
    }
    const cx<R>* x = v + 6 * b;
    cx<R>* y = o + 6 * b;
    if constexpr (std::is_same<R, dfloat>::value) {
      // row r: d_r x_r + sum_{c > r} K_rc x_c + sum_{c < r} conj(K_cr) x_c,
      // off-diagonal K_rc (r < c) at index k(r, c) of the row-major upper triangle
#pragma unroll
      for (int r0 = 0; r0 < 6; ++r0) {
        DfAcc re, im;
        dfa_first(re, d[r0], x[r0].re);
        dfa_first(im, d[r0], x[r0].im);
#pragma unroll
        for (int c0 = 0; c0 < 6; ++c0) {
          if (c0 == r0) continue;
          const int a0 = r0 < c0 ? r0 : c0, b0 = r0 < c0 ? c0 : r0;
          const int k = a0 * 5 - a0 * (a0 - 1) / 2 + (b0 - a0 - 1);
          const cx<R> o2 = off[k];
          const R oi = r0 < c0 ? o2.im : -o2.im;  // conj for the lower triangle
          dfa_add(re, o2.re, x[c0].re);
          dfa_add(re, -oi, x[c0].im);
          dfa_add(im, o2.re, x[c0].im);
          dfa_add(im, oi, x[c0].re);
        }
        y[r0] = cx<R>{dfa_get(re), dfa_get(im)};
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < 6; ++r0) y[r0] = d[r0] * x[r0];
      int k = 0;
#pragma unroll
      for (int r0 = 0; r0 < 6; ++r0)
#pragma unroll
        for (int c0 = r0 + 1; c0 < 6; ++c0) {
          cfma(y[r0], off[k], x[c0]);
          cfmac(y[c0], off[k], x[r0]);
          ++k;
        }
    }
  }
}

// ---------------------------------------------------------------------------
// spin projection (chiral basis) for the hop along direction mu.
// S = -1: (1 - g_mu) psi, S = +1: (1 + g_mu) psi.  The projected spinor is
// (h0, h1, l0, l1) with the half spinor h and lower components l fixed
// linear functions of h; only h is transported.
// ---------------------------------------------------------------------------
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Spinor<R>& p, HalfSpinor<R>& h) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> p0 = p.c[0][a], p1 = p.c[1][a], p2 = p.c[2][a], p3 = p.c[3][a];
    if constexpr (MU == 0) {
      if constexpr (S < 0) { h.c[0][a] = p0 + p2; h.c[1][a] = p1 + p3; }
      else                 { h.c[0][a] = p0 - p2; h.c[1][a] = p1 - p3; }
    } else if constexpr (MU == 1) {
      if constexpr (S < 0) { h.c[0][a] = p0 + times_i(p3); h.c[1][a] = p1 + times_i(p2); }
      else                 { h.c[0][a] = p0 - times_i(p3); h.c[1][a] = p1 - times_i(p2); }
    } else if constexpr (MU == 2) {
      if constexpr (S < 0) { h.c[0][a] = p0 + p3; h.c[1][a] = p1 - p2; }
      else                 { h.c[0][a] = p0 - p3; h.c[1][a] = p1 + p2; }
    } else {
      if constexpr (S < 0) { h.c[0][a] = p0 + times_i(p2); h.c[1][a] = p1 - times_i(p3); }
      else                 { h.c[0][a] = p0 - times_i(p2); h.c[1][a] = p1 + times_i(p3); }
    }
  }
}

// acc += w * (1 -/+ g_mu)-reconstruction of the transported half spinor h
// (SCALE = false: w = 1, no multiplication)
// A time face of a sub-domain: one half spinor (2 spins x 3 colours) per
// site of one parity of one time slice, Fs = Vh / L0 sites, 16-byte chunks
// stored chunk-major ([chunk][Fs]): binary64 6 chunks (one complex each),
// binary32 3 chunks (two complex each); component k = 3 spin + colour.
template <typename R>
__device__ __forceinline__ void load_half(const void* base, long Fs, long f, HalfSpinor<R>& h) {
  cx<R>* c = &h.c[0][0];
  if constexpr (sizeof(R) == 8) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 v = b[k * Fs + f];
      c[k] = cx<R>{v.x, v.y};
    }
  } else {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 v = b[k * Fs + f];
      c[2 * k] = cx<R>{v.x, v.y};
      c[2 * k + 1] = cx<R>{v.z, v.w};
    }
  }
}
template <typename R>
__device__ __forceinline__ void store_half(void* base, long Fs, long f, const HalfSpinor<R>& h) {
  const cx<R>* c = &h.c[0][0];
  if constexpr (sizeof(R) == 8) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k * Fs + f] = make_double2(c[k].re, c[k].im);
  } else {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k * Fs + f] = make_float4(c[2 * k].re, c[2 * k].im, c[2 * k + 1].re, c[2 * k + 1].im);
  }
}

template <int MU, int S, typename R, bool SCALE = true>
__device__ __forceinline__ void accum_reconstruct(Spinor<R>& acc, const HalfSpinor<R>& h, R w) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> h0 = h.c[0][a], h1 = h.c[1][a];
    if constexpr (SCALE) {
      h0 = w * h0;
      h1 = w * h1;
    }
    acc.c[0][a] = acc.c[0][a] + h0;
    acc.c[1][a] = acc.c[1][a] + h1;
    cx<R> l0, l1;
    if constexpr (MU == 0) { l0 = h0; l1 = h1; }
    else if constexpr (MU == 1) { l0 = times_mi(h1); l1 = times_mi(h0); }
    else if constexpr (MU == 2) { l0 = -h1; l1 = h0; }
    else { l0 = times_mi(h0); l1 = times_i(h1); }
    if constexpr (S > 0) { l0 = -l0; l1 = -l1; }
    acc.c[2][a] = acc.c[2][a] + l0;
    acc.c[3][a] = acc.c[3][a] + l1;
  }
}

}  // namespace oq
