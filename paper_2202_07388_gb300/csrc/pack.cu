// Layout conversion kernels: canonical binary64 links and spinors (site
// lexicographic, time slowest) to the packed even-odd chunk-major device
// layouts, with rounding to the storage precision (round to nearest even)
// and an optional per-field scale for the 16-bit formats.
#include "oq_internal.h"
#include "oq_kernels.h"

namespace oq {

__device__ __forceinline__ long lex_of(const Geom& g, const int x[4]) {
  return (((long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// one thread per (eo site, parity, mu); u18 (optional) receives an 18-real
// binary32 copy next to a 12-real one; A (optional) multiplies the link by
// exp(i q A_mu(x)) (QCD+QED), uclov / au1 (optional) keep the link before
// the phase and the angle
// cs_l1 > 0 (C* boundaries): canon holds the physical links of L1 = cs_l1
// (half the doubled extent g.L[1]); the sites x1 >= cs_l1 of the doubled
// lattice get the charge-conjugate copy: the complex conjugate link (and the
// U(1) angle negated)
__global__ void pack_links_kernel(Geom g, const double2* __restrict__ canon, double2* __restrict__ u64,
                                  void* __restrict__ u32, int fmt, float2* __restrict__ u18,
                                  const double* __restrict__ A, double q, double2* __restrict__ uclov,
                                  double* __restrict__ au1, int cs_l1) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  const int mu = blockIdx.z;
  if (i >= g.Vh) return;
  int x[4];
  eo_coords(g, p, i, x);
  bool mirror = false;
  long lex = lex_of(g, x);
  if (cs_l1 > 0) {
    mirror = x[1] >= cs_l1;
    const int x1 = mirror ? x[1] - cs_l1 : x[1];
    lex = (((long)x[0] * cs_l1 + x1) * g.L[2] + x[2]) * g.L[3] + x[3];
  }
  const double2* src = canon + (lex * 4 + mu) * 9;
  double2 m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = mirror ? make_double2(src[k].x, -src[k].y) : src[k];
  if (uclov) {
    double2* d = uclov + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k * g.Vh + i] = m[k];
  }
  if (A) {
    const double a = mirror ? -A[lex * 4 + mu] : A[lex * 4 + mu];
    double sn, cs;
    sincos(q * a, &sn, &cs);
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = make_double2(m[k].x * cs - m[k].y * sn, m[k].x * sn + m[k].y * cs);
    au1[(long)(p * 4 + mu) * g.Vh + i] = a;
  }
  double2* d64 = u64 + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
  for (int k = 0; k < 9; ++k) d64[k * g.Vh + i] = m[k];
  if (!u32) return;  // binary64 links only
  if (fmt == LINK_18) {
    float2* d = reinterpret_cast<float2*>(u32) + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k * g.Vh + i] = make_float2((float)m[k].x, (float)m[k].y);
  } else {
    float4* d = reinterpret_cast<float4*>(u32) + ((long)(p * 4 + mu) * 3) * g.Vh;
    d[i] = make_float4((float)m[0].x, (float)m[0].y, (float)m[1].x, (float)m[1].y);
    d[g.Vh + i] = make_float4((float)m[2].x, (float)m[2].y, (float)m[3].x, (float)m[3].y);
    d[2 * g.Vh + i] = make_float4((float)m[4].x, (float)m[4].y, (float)m[5].x, (float)m[5].y);
    if (u18) {
      float2* e = u18 + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
      for (int k = 0; k < 9; ++k) e[k * g.Vh + i] = make_float2((float)m[k].x, (float)m[k].y);
    }
  }
}

cudaError_t pack_links(const Geom& g, const double* canon, double* u64, void* u32, int fmt, void* u18,
                       const double* A, double q, double* uclov, double* au1, cudaStream_t s, int cs_l1) {
  dim3 block(128), grid((unsigned)((g.Vh + 127) / 128), 2, 4);
  pack_links_kernel<<<grid, block, 0, s>>>(g, reinterpret_cast<const double2*>(canon),
                                           reinterpret_cast<double2*>(u64), u32, fmt,
                                           reinterpret_cast<float2*>(u18), A, q,
                                           reinterpret_cast<double2*>(uclov), au1, cs_l1);
  return cudaGetLastError();
}

// one thread per (eo site, parity): the time-like link U_0(x) of the slices
// x0 = 0 (hops 0 <-> 1) and x0 = T-1 (hops T-1 <-> T, i.e. across the
// boundary) becomes zero in every hopping copy, so that no hop reaches the
// x0 = 0 slice, where Schroedinger-functional quark fields vanish
__global__ void sf_mask_links_kernel(Geom g, double2* __restrict__ u64, void* __restrict__ u32, int fmt,
                                     float2* __restrict__ u18) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (i >= g.Vh) return;
  int x[4];
  eo_coords(g, p, i, x);
  if (x[0] != 0 && x[0] != g.L[0] - 1) return;
  const int mu = 0;
  double2* d64 = u64 + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
  for (int k = 0; k < 9; ++k) d64[k * g.Vh + i] = make_double2(0.0, 0.0);
  if (fmt == LINK_18) {
    float2* d = reinterpret_cast<float2*>(u32) + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k * g.Vh + i] = make_float2(0.f, 0.f);
  } else {
    float4* d = reinterpret_cast<float4*>(u32) + ((long)(p * 4 + mu) * 3) * g.Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k * g.Vh + i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (u18) {
    float2* e = u18 + ((long)(p * 4 + mu) * 9) * g.Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k * g.Vh + i] = make_float2(0.f, 0.f);
  }
}

cudaError_t sf_mask_links(const Geom& g, double* u64, void* u32, int fmt, void* u18, cudaStream_t s) {
  dim3 block(128), grid((unsigned)((g.Vh + 127) / 128), 2);
  sf_mask_links_kernel<<<grid, block, 0, s>>>(g, reinterpret_cast<double2*>(u64), u32, fmt,
                                              reinterpret_cast<float2*>(u18));
  return cudaGetLastError();
}

// one thread per (eo site, parity, rhs).  blockIdx.y = parity index within
// the subset, blockIdx.z = rhs.
template <int P>
__global__ void pack_spinor_kernel(Geom g, const double2* __restrict__ canon, char* __restrict__ out,
                                   int subset, long canon_stride, long out_stride, double scale, int half) {
  typedef typename PrecTraits<P>::R R;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  const int p = (subset == 2) ? (int)blockIdx.y : subset;
  const int rhs = blockIdx.z;
  int x[4];
  eo_coords(g, p, i, x);
  // half: the canonical field holds one parity only, site lex / 2 (the sites
  // of one parity alternate along x3, L3 even)
  const double2* src = canon + rhs * canon_stride + (half ? lex_of(g, x) >> 1 : lex_of(g, x)) * 12;
  // Schroedinger-functional lattices: the field vanishes at x0 = 0
  if (g.bc_t == 0.f && x[0] == 0) scale = 0.0;
  Spinor<R> s;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = src[k];
    s.c[k / 3][k % 3] = cx<R>{(R)(v.x * scale), (R)(v.y * scale)};
  }
  char* dst = out + rhs * out_stride + ((subset == 2) ? (long)p * spinor_half_bytes(g.Vh, P) : 0);
  if constexpr (P == P_BF16 || P == P_F16) {
    // round binary64 -> 16-bit directly (no intermediate binary32 rounding)
    uint4* b = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double2 v = src[4 * c + k];
        double re = v.x * scale, im = v.y * scale;
        if constexpr (P == P_BF16) {
          __nv_bfloat16 a = __double2bfloat16(re), bb = __double2bfloat16(im);
          w[k] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(bb) << 16);
        } else {
          __half a = __double2half(re), bb = __double2half(im);
          w[k] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(bb) << 16);
        }
      }
      b[c * g.Vh + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    store_spinor<P>(dst, g.Vh, i, s);
  }
}

template <int P>
__global__ void unpack_spinor_kernel(Geom g, const char* __restrict__ in, double2* __restrict__ canon,
                                     int subset, long in_stride, long canon_stride, double inv_scale, int half) {
  typedef typename PrecTraits<P>::R R;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  const int p = (subset == 2) ? (int)blockIdx.y : subset;
  const int rhs = blockIdx.z;
  int x[4];
  eo_coords(g, p, i, x);
  const char* src = in + rhs * in_stride + ((subset == 2) ? (long)p * spinor_half_bytes(g.Vh, P) : 0);
  Spinor<R> s;
  load_spinor<P>(src, g.Vh, i, s);
  double2* dst = canon + rhs * canon_stride + (half ? lex_of(g, x) >> 1 : lex_of(g, x)) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k)
    dst[k] = make_double2((double)s.c[k / 3][k % 3].re * inv_scale, (double)s.c[k / 3][k % 3].im * inv_scale);
}

// Even-site (or odd-site) canonical fields: the site of eo index i sits at
// position i (lex / 2), so the 128 sites of a CTA are one contiguous run of
// 128 x 12 double2.  The run moves between the canonical field and shared
// memory with consecutive threads on consecutive 16-byte chunks (coalesced,
// which matters when the field is page-locked host memory read or written
// over the host-device link), and each thread converts its own site from
// there.  Shared rows of 13 chunks keep the per-site accesses free of bank
// conflicts.  blockDim.x = 128.
constexpr int HB = 128, HROW = 13;

template <int P>
__global__ void __launch_bounds__(HB) pack_half_kernel(Geom g, const double2* __restrict__ canon,
                                                       char* __restrict__ out, int p, long canon_stride,
                                                       long out_stride, double scale) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double2 sm[HB * HROW];
  const int t = threadIdx.x, rhs = blockIdx.z;
  const long i0 = (long)blockIdx.x * HB;
  const int nsite = (int)(g.Vh - i0 < HB ? g.Vh - i0 : HB);
  const double2* src = canon + rhs * canon_stride + i0 * 12;
  for (int e = t; e < nsite * 12; e += HB) sm[(e / 12) * HROW + e % 12] = src[e];
  __syncthreads();
  if (t >= nsite) return;
  const long i = i0 + t;
  double sc = scale;
  if (g.bc_t == 0.f) {  // Schroedinger-functional lattices: the field vanishes at x0 = 0
    int x[4];
    eo_coords(g, p, i, x);
    if (x[0] == 0) sc = 0.0;
  }
  char* dst = out + rhs * out_stride;
  if constexpr (P == P_BF16 || P == P_F16) {
    uint4* b = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 v = sm[t * HROW + 4 * c + k];
        const double re = v.x * sc, im = v.y * sc;
        if constexpr (P == P_BF16) {
          __nv_bfloat16 a = __double2bfloat16(re), bb = __double2bfloat16(im);
          w[k] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(bb) << 16);
        } else {
          __half a = __double2half(re), bb = __double2half(im);
          w[k] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(bb) << 16);
        }
      }
      b[c * g.Vh + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    Spinor<R> sp;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double2 v = sm[t * HROW + k];
      sp.c[k / 3][k % 3] = cx<R>{(R)(v.x * sc), (R)(v.y * sc)};
    }
    store_spinor<P>(dst, g.Vh, i, sp);
  }
}

template <int P>
__global__ void __launch_bounds__(HB) unpack_half_kernel(Geom g, const char* __restrict__ in,
                                                         double2* __restrict__ canon, long in_stride,
                                                         long canon_stride, double inv_scale) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double2 sm[HB * HROW];
  const int t = threadIdx.x, rhs = blockIdx.z;
  const long i0 = (long)blockIdx.x * HB;
  const int nsite = (int)(g.Vh - i0 < HB ? g.Vh - i0 : HB);
  if (t < nsite) {
    Spinor<R> sp;
    load_spinor<P>(in + rhs * in_stride, g.Vh, i0 + t, sp);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      sm[t * HROW + k] = make_double2((double)sp.c[k / 3][k % 3].re * inv_scale,
                                      (double)sp.c[k / 3][k % 3].im * inv_scale);
  }
  __syncthreads();
  double2* dst = canon + rhs * canon_stride + i0 * 12;
  for (int e = t; e < nsite * 12; e += HB) dst[e] = sm[(e / 12) * HROW + e % 12];
}

cudaError_t pack_spinor(const Geom& g, int prec, int subset, const double* canon, void* out, double scale,
                        int nrhs, long canon_stride_d2, long out_stride_bytes, cudaStream_t s, int half) {
  if (half && subset == 2) return cudaErrorInvalidValue;
  if (half) {
    dim3 hb(HB), hg((unsigned)((g.Vh + HB - 1) / HB), 1, nrhs);
    const double2* c = reinterpret_cast<const double2*>(canon);
    char* o = reinterpret_cast<char*>(out);
    switch (prec) {
      case P_F64: pack_half_kernel<P_F64><<<hg, hb, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale); break;
      case P_F32: pack_half_kernel<P_F32><<<hg, hb, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale); break;
      case P_BF16: pack_half_kernel<P_BF16><<<hg, hb, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale); break;
      case P_F16: pack_half_kernel<P_F16><<<hg, hb, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale); break;
      case P_DF64: pack_half_kernel<P_DF64><<<hg, hb, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  dim3 block(128), grid((unsigned)((g.Vh + 127) / 128), subset == 2 ? 2 : 1, nrhs);
  const double2* c = reinterpret_cast<const double2*>(canon);
  char* o = reinterpret_cast<char*>(out);
  switch (prec) {
    case P_F64: pack_spinor_kernel<P_F64><<<grid, block, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale, half); break;
    case P_F32: pack_spinor_kernel<P_F32><<<grid, block, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale, half); break;
    case P_BF16: pack_spinor_kernel<P_BF16><<<grid, block, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale, half); break;
    case P_F16: pack_spinor_kernel<P_F16><<<grid, block, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale, half); break;
    case P_DF64: pack_spinor_kernel<P_DF64><<<grid, block, 0, s>>>(g, c, o, subset, canon_stride_d2, out_stride_bytes, scale, half); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t unpack_spinor(const Geom& g, int prec, int subset, const void* in, double* canon, double scale,
                          int nrhs, long in_stride_bytes, long canon_stride_d2, cudaStream_t s, int half) {
  if (half && subset == 2) return cudaErrorInvalidValue;
  if (half) {
    dim3 hb(HB), hg((unsigned)((g.Vh + HB - 1) / HB), 1, nrhs);
    double2* c = reinterpret_cast<double2*>(canon);
    const char* i = reinterpret_cast<const char*>(in);
    const double inv = 1.0 / scale;
    switch (prec) {
      case P_F64: unpack_half_kernel<P_F64><<<hg, hb, 0, s>>>(g, i, c, in_stride_bytes, canon_stride_d2, inv); break;
      case P_F32: unpack_half_kernel<P_F32><<<hg, hb, 0, s>>>(g, i, c, in_stride_bytes, canon_stride_d2, inv); break;
      case P_BF16: unpack_half_kernel<P_BF16><<<hg, hb, 0, s>>>(g, i, c, in_stride_bytes, canon_stride_d2, inv); break;
      case P_F16: unpack_half_kernel<P_F16><<<hg, hb, 0, s>>>(g, i, c, in_stride_bytes, canon_stride_d2, inv); break;
      case P_DF64: unpack_half_kernel<P_DF64><<<hg, hb, 0, s>>>(g, i, c, in_stride_bytes, canon_stride_d2, inv); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  dim3 block(128), grid((unsigned)((g.Vh + 127) / 128), subset == 2 ? 2 : 1, nrhs);
  double2* c = reinterpret_cast<double2*>(canon);
  const char* i = reinterpret_cast<const char*>(in);
  const double inv = 1.0 / scale;
  switch (prec) {
    case P_F64: unpack_spinor_kernel<P_F64><<<grid, block, 0, s>>>(g, i, c, subset, in_stride_bytes, canon_stride_d2, inv, half); break;
    case P_F32: unpack_spinor_kernel<P_F32><<<grid, block, 0, s>>>(g, i, c, subset, in_stride_bytes, canon_stride_d2, inv, half); break;
    case P_BF16: unpack_spinor_kernel<P_BF16><<<grid, block, 0, s>>>(g, i, c, subset, in_stride_bytes, canon_stride_d2, inv, half); break;
    case P_F16: unpack_spinor_kernel<P_F16><<<grid, block, 0, s>>>(g, i, c, subset, in_stride_bytes, canon_stride_d2, inv, half); break;
    case P_DF64: unpack_spinor_kernel<P_DF64><<<grid, block, 0, s>>>(g, i, c, subset, in_stride_bytes, canon_stride_d2, inv, half); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// binary64 array -> double-float pairs (hi = rn(x), lo = rn(x - hi)), element
// by element: a binary64-layout field or table becomes its DF64 layout
__global__ void split_f64_kernel(const double* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const double x = in[k];
    const float hi = __double2float_rn(x);
    out[k] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}

cudaError_t split_f64(const double* in, void* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  split_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, reinterpret_cast<float2*>(out), n);
  return cudaGetLastError();
}

}  // namespace oq
