// Vector kernels on packed spinor fields: binary64 norms and dot products
// (Sec. 2, 2.1: reductions in binary64 whatever the storage type) and the
// vector steps of CGNE that are not fused into the stencil epilogue.
// One thread per site (all 24 reals), right-hand sides on gridDim.y.
#include "reduce.cuh"
#include "oq_kernels.h"

namespace oq {

static const int RED_BX = 256;

int reduce_grid(long nsites) {
  long g = (nsites + RED_BX - 1) / RED_BX;
  const long cap = 152L * 8;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

template <int P>
__global__ void __launch_bounds__(RED_BX) norm2_kernel(const char* x, long Vh, long stride, int nrhs, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[RED_BX / 32];
  const int rhs = blockIdx.y;
  double acc = 0.0;
  const char* xb = x + rhs * stride;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += (long)gridDim.x * blockDim.x) {
    Spinor<R> s;
    load_spinor<P>(xb, Vh, i, s);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc += (double)s.c[a][c].re * s.c[a][c].re + (double)s.c[a][c].im * s.c[a][c].im;
  }
  grid_reduce(acc, ra, rhs, nrhs, smem, blockIdx.x, gridDim.x);
}

template <int P>
__global__ void __launch_bounds__(RED_BX) dot_kernel(const char* x, const char* y, long Vh, long stride, int nrhs,
                                                     RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[RED_BX / 32];
  const int rhs = blockIdx.y;
  double re = 0.0, im = 0.0;
  const char* xb = x + rhs * stride;
  const char* yb = y + rhs * stride;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += (long)gridDim.x * blockDim.x) {
    Spinor<R> a, b;
    load_spinor<P>(xb, Vh, i, a);
    load_spinor<P>(yb, Vh, i, b);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        re += (double)a.c[s][c].re * b.c[s][c].re + (double)a.c[s][c].im * b.c[s][c].im;
        im += (double)a.c[s][c].re * b.c[s][c].im - (double)a.c[s][c].im * b.c[s][c].re;
      }
  }
  grid_reduce(re, ra, 2 * rhs, 2 * nrhs, smem, blockIdx.x, gridDim.x);
  __syncthreads();
  grid_reduce(im, ra, 2 * rhs + 1, 2 * nrhs, smem, blockIdx.x, gridDim.x);
}

// nsites = number of sites of the field (Vh for a half field, 2 Vh for a full one:
// a full packed field is two consecutive half fields, which is the same
// chunk-major layout with 2 Vh sites only if read per half; handled by the
// caller passing half fields).
cudaError_t reduce_norm2(int prec, const void* x, long Vh, long stride_bytes, int nrhs, const RedArgs& ra,
                         cudaStream_t s) {
  dim3 grid(reduce_grid(Vh), nrhs), block(RED_BX);
  const char* xx = (const char*)x;
  switch (prec) {
    case P_F64: norm2_kernel<P_F64><<<grid, block, 0, s>>>(xx, Vh, stride_bytes, nrhs, ra); break;
    case P_F32: norm2_kernel<P_F32><<<grid, block, 0, s>>>(xx, Vh, stride_bytes, nrhs, ra); break;
    case P_BF16: norm2_kernel<P_BF16><<<grid, block, 0, s>>>(xx, Vh, stride_bytes, nrhs, ra); break;
    case P_F16: norm2_kernel<P_F16><<<grid, block, 0, s>>>(xx, Vh, stride_bytes, nrhs, ra); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t reduce_dot(int prec, const void* x, const void* y, long Vh, long stride_bytes, int nrhs,
                       const RedArgs& ra, cudaStream_t s) {
  dim3 grid(reduce_grid(Vh), nrhs), block(RED_BX);
  const char* xx = (const char*)x;
  const char* yy = (const char*)y;
  switch (prec) {
    case P_F64: dot_kernel<P_F64><<<grid, block, 0, s>>>(xx, yy, Vh, stride_bytes, nrhs, ra); break;
    case P_F32: dot_kernel<P_F32><<<grid, block, 0, s>>>(xx, yy, Vh, stride_bytes, nrhs, ra); break;
    case P_BF16: dot_kernel<P_BF16><<<grid, block, 0, s>>>(xx, yy, Vh, stride_bytes, nrhs, ra); break;
    case P_F16: dot_kernel<P_F16><<<grid, block, 0, s>>>(xx, yy, Vh, stride_bytes, nrhs, ra); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CGNE vector steps
// ---------------------------------------------------------------------------

// p = r + beta p   (right-hand sides in MODE_RUN).  hist (diagnostics,
// nullable): thread 0 of each rhs records the recursive residual
// sqrt(rr) * scale of the regular step just done at hist[rhs][steps - 1]
// (launched after every step's CG update and before any restart, so a
// gated-off rhs only rewrites its last entry with the same value)
template <int P>
__global__ void __launch_bounds__(256) cg_p_kernel(char* p, const char* r, long Vh, long stride, const CgState* cg,
                                                   double* hist, int hcap) {
  typedef typename PrecTraits<P>::R R;
  const int rhs = blockIdx.y;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (hist && i == 0) {
    const CgState& c = cg[rhs];
    if (c.steps >= 1 && c.steps <= hcap) hist[(long)rhs * hcap + c.steps - 1] = sqrt(c.rr) * c.scale;
  }
  if (i >= Vh || cg[rhs].mode != MODE_RUN) return;
  const R beta = (R)cg[rhs].beta;
  Spinor<R> pv, rv;
  load_spinor<P>(p + rhs * stride, Vh, i, pv);
  load_spinor<P>(r + rhs * stride, Vh, i, rv);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pv.c[s][c].re = fma(beta, pv.c[s][c].re, rv.c[s][c].re);
      pv.c[s][c].im = fma(beta, pv.c[s][c].im, rv.c[s][c].im);
    }
  store_spinor<P>(p + rhs * stride, Vh, i, pv);
}

cudaError_t cg_update_p(int prec, void* p, const void* r, long Vh, long stride, int nrhs, const CgState* cg,
                        cudaStream_t s, double* hist, int hcap) {
  dim3 grid((unsigned)((Vh + 255) / 256), nrhs), block(256);
  char* pp = (char*)p;
  const char* rr = (const char*)r;
  switch (prec) {
    case P_F64: cg_p_kernel<P_F64><<<grid, block, 0, s>>>(pp, rr, Vh, stride, cg, hist, hcap); break;
    case P_F32: cg_p_kernel<P_F32><<<grid, block, 0, s>>>(pp, rr, Vh, stride, cg, hist, hcap); break;
    case P_BF16: cg_p_kernel<P_BF16><<<grid, block, 0, s>>>(pp, rr, Vh, stride, cg, hist, hcap); break;
    case P_F16: cg_p_kernel<P_F16><<<grid, block, 0, s>>>(pp, rr, Vh, stride, cg, hist, hcap); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// x_d += scale * x_s   (right-hand sides in MODE_RESET)
template <int XP>
__global__ void __launch_bounds__(256) cg_accx_kernel(char* xd, const char* xs, long Vh, long sd, long ss,
                                                      const CgState* cg, char* xdf) {
  typedef typename PrecTraits<XP>::R RX;
  const int rhs = blockIdx.y;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh || cg[rhs].mode != MODE_RESET) return;
  const double sc = cg[rhs].scale;
  Spinor<double> d;
  Spinor<RX> v;
  load_spinor<P_F64>(xd + rhs * sd, Vh, i, d);
  load_spinor<XP>(xs + rhs * ss, Vh, i, v);
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d.c[s][c].re = fma(sc, (double)v.c[s][c].re, d.c[s][c].re);
      d.c[s][c].im = fma(sc, (double)v.c[s][c].im, d.c[s][c].im);
    }
  store_spinor<P_F64>(xd + rhs * sd, Vh, i, d);
  if (xdf) {
    // the double-float split of the new x_d, in the binary64 layout: one
    // (re.hi, re.lo, im.hi, im.lo) chunk where x_d holds one double2
    float4* o = reinterpret_cast<float4*>(xdf + rhs * sd);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double re = d.c[k / 3][k % 3].re, im = d.c[k / 3][k % 3].im;
      const float rh = __double2float_rn(re), ih = __double2float_rn(im);
      o[k * Vh + i] = make_float4(rh, __double2float_rn(re - (double)rh), ih, __double2float_rn(im - (double)ih));
    }
  }
}

cudaError_t cg_accumulate_x(int xprec, double* xd, const void* xs, long Vh, long stride_xd, long stride_xs,
                            int nrhs, const CgState* cg, cudaStream_t s, void* xdf) {
  dim3 grid((unsigned)((Vh + 255) / 256), nrhs), block(256);
  if (xprec == P_F64)
    cg_accx_kernel<P_F64><<<grid, block, 0, s>>>((char*)xd, (const char*)xs, Vh, stride_xd, stride_xs, cg,
                                                 (char*)xdf);
  else
    cg_accx_kernel<P_F32><<<grid, block, 0, s>>>((char*)xd, (const char*)xs, Vh, stride_xd, stride_xs, cg,
                                                 (char*)xdf);
  return cudaGetLastError();
}

// r_s = p = r_d / scale in the small type, x_s = 0, ||r_s||^2 -> FIN_RESTART.
// RD: storage of r_d (P_F64 after a binary64 reset, P_DF64 after a
// double-float one).  For the binary32-arithmetic types the site's squares
// are summed in binary32 (as in the stencil epilogues), converted once.
template <int P, int XP, int RD>
__global__ void __launch_bounds__(256) cg_restart_kernel(const char* rd, char* rs, char* p, char* xs, long Vh,
                                                         long sd, long ss, long sx, int nrhs, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  typedef typename PrecTraits<XP>::R RX;
  __shared__ double smem[256 / 32];
  const int rhs = blockIdx.y;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < Vh && ra.cg[rhs].mode == MODE_RESET) {
    const double inv = 1.0 / ra.cg[rhs].scale;
    Spinor<R> v;
    Spinor<RX> z;
    if constexpr (RD == P_DF64) {
      Spinor<dfloat> d;
      load_spinor<P_DF64>(rd + rhs * sd, Vh, i, d);
      const float invf = (float)inv;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if constexpr (P == P_F64) {  // binary64 phase of a precision ladder: keep both words
            v.c[s][c] = cx<R>{((double)d.c[s][c].re.hi + (double)d.c[s][c].re.lo) * inv,
                              ((double)d.c[s][c].im.hi + (double)d.c[s][c].im.lo) * inv};
          } else {
            v.c[s][c] = cx<R>{(R)(__fadd_rn(d.c[s][c].re.hi, d.c[s][c].re.lo) * invf),
                              (R)(__fadd_rn(d.c[s][c].im.hi, d.c[s][c].im.lo) * invf)};
          }
        }
    } else {
      Spinor<double> d;
      load_spinor<P_F64>(rd + rhs * sd, Vh, i, d);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) v.c[s][c] = cx<R>{(R)(d.c[s][c].re * inv), (R)(d.c[s][c].im * inv)};
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) z.c[s][c] = cx<RX>{0, 0};
    round_trip<P>(v);  // the norm below is that of the stored (rounded) values
    store_spinor<P>(rs + rhs * ss, Vh, i, v);
    store_spinor<P>(p + rhs * ss, Vh, i, v);
    store_spinor<XP>(xs + rhs * sx, Vh, i, z);
    acc = site_norm2(v);
  }
  grid_reduce(acc, ra, rhs, nrhs, smem, blockIdx.x, gridDim.x);
}

cudaError_t cg_restart(int prec, const void* rd, int rd_prec, void* rs, void* p, void* xs, int xprec, long Vh,
                       long stride_d, long stride_s, long stride_xs, int nrhs, const RedArgs& ra, cudaStream_t s) {
  dim3 grid((unsigned)((Vh + 255) / 256), nrhs), block(256);
  const char* d = (const char*)rd;
  char *r = (char*)rs, *pp = (char*)p, *x = (char*)xs;
#define OQ_RESTART(PP, XX, RR) \
  cg_restart_kernel<PP, XX, RR><<<grid, block, 0, s>>>(d, r, pp, x, Vh, stride_d, stride_s, stride_xs, nrhs, ra)
  if (rd_prec == P_DF64) {
    switch (prec) {
      case P_F64: OQ_RESTART(P_F64, P_F64, P_DF64); break;
      case P_F32: OQ_RESTART(P_F32, P_F32, P_DF64); break;
      case P_BF16: OQ_RESTART(P_BF16, P_F32, P_DF64); break;
      case P_F16: OQ_RESTART(P_F16, P_F32, P_DF64); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (prec) {
      case P_F64: OQ_RESTART(P_F64, P_F64, P_F64); break;
      case P_F32: OQ_RESTART(P_F32, P_F32, P_F64); break;
      case P_BF16: OQ_RESTART(P_BF16, P_F32, P_F64); break;
      case P_F16: OQ_RESTART(P_F16, P_F32, P_F64); break;
      default: return cudaErrorInvalidValue;
    }
  }
#undef OQ_RESTART
  (void)xprec;
  return cudaGetLastError();
}

// dst = src for right-hand sides in mode `gate` (binary64 half fields)
__global__ void __launch_bounds__(256) copy_gated_kernel(double2* dst, const double2* src, long n, long stride,
                                                         const CgState* cg, int gate) {
  const int rhs = blockIdx.y;
  if (cg[rhs].mode != gate) return;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    dst[rhs * stride + k] = src[rhs * stride + k];
}

cudaError_t cg_copy_gated(double* dst, const double* src, long n16, long stride16, int nrhs, const CgState* cg,
                          int gate, cudaStream_t s) {
  dim3 grid(reduce_grid(n16 / 4 + 1), nrhs), block(256);
  copy_gated_kernel<<<grid, block, 0, s>>>((double2*)dst, (const double2*)src, n16, stride16, cg, gate);
  return cudaGetLastError();
}

// y = a_k x + b_k y for right-hand side k (real coefficients), on the reals
// of packed binary64 or binary32 fields (the layout is irrelevant: every
// real is scaled the same way); n reals per right-hand side
struct AxpbyCoef {
  double a[64], b[64];
};
template <typename R>
__global__ void __launch_bounds__(256) axpby_kernel(const R* x, R* y, long n, const AxpbyCoef c) {
  const int rhs = blockIdx.y;
  const R a = (R)c.a[rhs], b = (R)c.b[rhs];
  const R* xr = x + rhs * n;
  R* yr = y + rhs * n;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    yr[k] = fma(a, xr[k], b * yr[k]);
}

cudaError_t axpby(int prec, const double* a, const void* x, const double* b, void* y, long n, int nrhs,
                  cudaStream_t s) {
  if (nrhs < 1 || nrhs > 64) return cudaErrorInvalidValue;
  AxpbyCoef c;
  for (int k = 0; k < nrhs; ++k) {
    c.a[k] = a[k];
    c.b[k] = b[k];
  }
  dim3 grid(reduce_grid(n / 24 + 1), nrhs), block(256);
  if (prec == P_F64)
    axpby_kernel<double><<<grid, block, 0, s>>>((const double*)x, (double*)y, n, c);
  else if (prec == P_F32)
    axpby_kernel<float><<<grid, block, 0, s>>>((const float*)x, (float*)y, n, c);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace oq
