// Time-split sub-domains (Sec. 3: the global lattice is divided into local
// lattices, one per process, and each application of the Dirac operator
// needs the field on the neighbouring boundary sites).
//
// A sub-domain lattice (oq_lattice.bc_t = OQ_BC_HALO) holds T_loc time
// slices of a larger lattice split along time.  Its hops that leave the
// sub-domain through the x0 = T_loc-1 / x0 = 0 faces read faces received from
// the next / previous sub-domain instead of the periodic wrap:
//
//   to the previous one: the projected half spinors (1 -/+ g0) psi of the
//     x0 = 0 slice (the previous one multiplies them by its own U_0);
//   to the next one:     U_0(x)^dag (1 +/- g0) psi(x) of the x0 = T_loc-1
//     slice (the link lives here, so it is applied here);
//
// 12 reals per boundary site and direction (the spin projection halves the
// data).  The face of the output parity p is made from the input field of
// parity 1 - p.  The clover term of a sub-domain needs the links one slice
// beyond each face: oq_gauge_upload_halo takes T_loc + 2 slices and the
// clover build runs on that extended lattice and keeps the interior.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"

namespace oq {

// one thread per (face site, slice, rhs): blockIdx.y = 0 the x0 = 0 slice
// (face to the previous sub-domain), 1 the x0 = T-1 slice (to the next one).
// in: packed half field of parity q (right-hand sides in_stride apart).
template <int P, int FMT, bool DAG>
__global__ void face_pack_kernel(Geom g, const char* __restrict__ in, long in_stride, const void* __restrict__ links,
                                 int q, char* __restrict__ to_prev, char* __restrict__ to_next, long fstride) {
  typedef typename PrecTraits<P>::R R;
  constexpr int SF = DAG ? +1 : -1;  // projector sign of the forward hop
  const long Fs = g.Vh / g.L[0];
  const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= Fs) return;
  const int rhs = blockIdx.z;
  const bool hi = blockIdx.y == 1;
  const long i = (hi ? (long)(g.L[0] - 1) * Fs : 0) + f;
  Spinor<R> nb;
  load_spinor<P>(in + rhs * in_stride, g.Vh, i, nb);
  HalfSpinor<R> h;
  if (!hi) {
    // the previous sub-domain's forward hop from its last slice lands here
    project<0, SF>(nb, h);
    store_half<R>(to_prev + rhs * fstride, Fs, f, h);
  } else {
    // the next sub-domain's backward hop from its first slice lands here
    project<0, -SF>(nb, h);
    Su3<R> u;
    load_link<R, FMT>(links, g.Vh, q, 0, i, u);
    HalfSpinor<R> t;
    su3_dag_mul(u, h, t);
    store_half<R>(to_next + rhs * fstride, Fs, f, t);
  }
}

template <int P>
static cudaError_t face_pack_p(const Geom& g, int fmt, const void* in, long in_stride, const void* links, int q,
                               int dagger, void* to_prev, void* to_next, long fstride, int nrhs, cudaStream_t s) {
  const long Fs = g.Vh / g.L[0];
  dim3 block(128), grid((unsigned)((Fs + 127) / 128), 2, (unsigned)nrhs);
  const char* x = (const char*)in;
  char* a = (char*)to_prev;
  char* b = (char*)to_next;
  if (P == P_F64 || fmt == LINK_18) {
    if (dagger)
      face_pack_kernel<P, LINK_18, true><<<grid, block, 0, s>>>(g, x, in_stride, links, q, a, b, fstride);
    else
      face_pack_kernel<P, LINK_18, false><<<grid, block, 0, s>>>(g, x, in_stride, links, q, a, b, fstride);
  } else {
    if (dagger)
      face_pack_kernel<P, LINK_12, true><<<grid, block, 0, s>>>(g, x, in_stride, links, q, a, b, fstride);
    else
      face_pack_kernel<P, LINK_12, false><<<grid, block, 0, s>>>(g, x, in_stride, links, q, a, b, fstride);
  }
  return cudaGetLastError();
}

static cudaError_t face_pack(int prec, const Geom& g, int fmt, const void* in, long in_stride, const void* links,
                             int q, int dagger, void* to_prev, void* to_next, long fstride, int nrhs,
                             cudaStream_t s) {
  switch (prec) {
    case P_F64: return face_pack_p<P_F64>(g, fmt, in, in_stride, links, q, dagger, to_prev, to_next, fstride, nrhs, s);
    case P_F32: return face_pack_p<P_F32>(g, fmt, in, in_stride, links, q, dagger, to_prev, to_next, fstride, nrhs, s);
    case P_BF16:
      return face_pack_p<P_BF16>(g, fmt, in, in_stride, links, q, dagger, to_prev, to_next, fstride, nrhs, s);
    case P_F16: return face_pack_p<P_F16>(g, fmt, in, in_stride, links, q, dagger, to_prev, to_next, fstride, nrhs, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace oq

using namespace oq;

namespace {

bool valid(oq_handle h, int lat) { return h && lat >= 0 && lat < (int)h->lats.size(); }

// bytes of one face (one parity, one right-hand side): 12 reals per boundary site
size_t face_bytes(const LatCtx& L, int prec) {
  const long Fs = L.g.Vh / L.g.L[0];
  return (size_t)Fs * 12 * (prec == P_F64 ? 8 : 4);
}

// binary32 link copy in the uploaded format (the faces and the halo launches
// read the same links)
const void* links_of(const LatCtx& L, int prec) { return prec == P_F64 ? L.u64.p : L.u32.p; }

// a stencil launch on a sub-domain: the tuned CTA shape with one rhs per
// thread (the halo hops live in the one-rhs kernel) on the uploaded links
HopLaunch halo_launch(oq_handle h, int lat, int prec, int mode, int dagger, int nrhs) {
  HopLaunch l = h->hop_launch(lat, prec, mode, dagger, EPI_NONE, nrhs);
  if (l.nr != 1) {
    l.nr = 1;
    if (l.bx * l.by > 256) l.by = 1;
  }
  l.regcap = 0;
  l.link_fmt = h->lats[lat].link_fmt;
  return l;
}

void set_halo(HopArgs& a, const oq_halo* halo, size_t fbytes, int nrhs) {
  a.halo_next = halo->from_next;
  a.halo_prev = halo->from_prev;
  a.halo_stride = (long)fbytes;
  a.halo_pstride = (long)fbytes * nrhs;
  a.halo_sign_next = (float)halo->sign_next;
  a.halo_sign_prev = (float)halo->sign_prev;
}

bool halo_ok(const oq_halo* halo) {
  return halo && halo->from_next && halo->from_prev && (halo->sign_next == 1.0 || halo->sign_next == -1.0) &&
         (halo->sign_prev == 1.0 || halo->sign_prev == -1.0);
}

}  // namespace

extern "C" size_t oq_face_bytes(oq_handle h, int lat, int prec) {
  if (!valid(h, lat) || prec < 0 || prec > 3) return 0;
  return face_bytes(h->lats[lat], prec);
}

extern "C" int oq_face_pack(oq_handle h, int lat, int prec, int subset, const void* in_dev, int nrhs, int dagger,
                            void* to_prev_dev, void* to_next_dev, void* stream) {
  if (!valid(h, lat) || prec < 0 || prec > 3 || subset < 0 || subset > 2 || !in_dev || !to_prev_dev ||
      !to_next_dev || nrhs < 1 || nrhs > 65535)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_gauge) return OQ_ERR_STATE;
  if (prec != P_F64 && L.link_fmt == LINK_12 && !L.u32.p) return OQ_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t fb = face_bytes(L, prec);
  const long half = (long)spinor_half_bytes(L.g.Vh, prec);
  if (subset != OQ_FULL) {
    // faces for the output parity 1 - subset
    if (face_pack(prec, L.g, L.link_fmt, in_dev, half, links_of(L, prec), subset, dagger, to_prev_dev, to_next_dev,
                  (long)fb, nrhs, s) != cudaSuccess)
      return OQ_ERR_CUDA;
    h->launches += 1;
    return OQ_OK;
  }
  // full fields: faces of output parity p (from input parity 1 - p) at p * nrhs faces
  for (int p = 0; p < 2; ++p) {
    const char* in = (const char*)in_dev + (long)(1 - p) * half;
    char* a = (char*)to_prev_dev + (size_t)p * nrhs * fb;
    char* b = (char*)to_next_dev + (size_t)p * nrhs * fb;
    if (face_pack(prec, L.g, L.link_fmt, in, 2 * half, links_of(L, prec), 1 - p, dagger, a, b, (long)fb, nrhs, s) !=
        cudaSuccess)
      return OQ_ERR_CUDA;
    h->launches += 1;
  }
  return OQ_OK;
}

extern "C" int oq_dw_apply_halo(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs,
                                int dagger, const oq_halo* halo, void* stream) {
  if (!valid(h, lat) || !in_dev || !out_dev || prec < 0 || prec > 3 || nrhs < 1 || !halo_ok(halo)) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover) return OQ_ERR_STATE;
  const size_t full = 2 * (size_t)spinor_half_bytes(L.g.Vh, prec);
  const char* x = (const char*)in_dev;
  const char* y = (const char*)out_dev;
  if (x < y + full * nrhs && y < x + full * nrhs) return OQ_ERR_ARG;
  HopArgs a = h->hop_args(lat, prec);
  a.in = in_dev;
  a.in2 = in_dev;
  a.out = out_dev;
  a.in_stride = a.in2_stride = a.out_stride = (long)full;
  a.half_bytes = (long)full / 2;
  a.nrhs = nrhs;
  set_halo(a, halo, face_bytes(L, prec), nrhs);
  return h->run_hop(halo_launch(h, lat, prec, HOP_DW, dagger ? 1 : 0, nrhs), a, (cudaStream_t)stream);
}

extern "C" int oq_dhat_pass(oq_handle h, int lat, int prec, int pass, const void* in_dev, const void* in2_dev,
                            void* out_dev, int nrhs, int dagger, const oq_halo* halo, void* stream) {
  if (!valid(h, lat) || !in_dev || !out_dev || prec < 0 || prec > 3 || nrhs < 1 || (pass != 1 && pass != 2))
    return OQ_ERR_ARG;
  if (pass == 2 && !in2_dev) return OQ_ERR_ARG;
  if (halo && !halo_ok(halo)) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover) return OQ_ERR_STATE;
  if (L.halo_t && !halo) return OQ_ERR_STATE;  // a sub-domain's time hops need the faces
  const size_t half = (size_t)spinor_half_bytes(L.g.Vh, prec);
  const char* x = (const char*)in_dev;
  const char* y = (const char*)out_dev;
  if (x < y + half * nrhs && y < x + half * nrhs) return OQ_ERR_ARG;
  HopArgs a = h->hop_args(lat, prec);
  a.in = in_dev;
  a.in2 = pass == 2 ? in2_dev : in_dev;
  a.out = out_dev;
  a.in_stride = a.in2_stride = a.out_stride = (long)half;
  a.half_bytes = (long)half;
  a.nrhs = nrhs;
  a.p = pass == 1 ? 1 : 0;
  if (halo) set_halo(a, halo, face_bytes(L, prec), nrhs);
  const int mode = pass == 1 ? HOP_P1 : HOP_P2;
  const HopLaunch l = halo ? halo_launch(h, lat, prec, mode, dagger ? 1 : 0, nrhs)
                           : h->hop_launch(lat, prec, mode, dagger ? 1 : 0, EPI_NONE, nrhs);
  return h->run_hop(l, a, (cudaStream_t)stream);
}

extern "C" int oq_gauge_upload_halo(oq_handle h, int lat, const double* U_ext_dev, int link_fmt, void* stream) {
  if (!valid(h, lat) || !U_ext_dev || (link_fmt != OQ_LINK_18 && link_fmt != OQ_LINK_12)) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.halo_t) return OQ_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const long Fs = L.g.Vh / L.g.L[0];
  // the hopping links: slices 0 .. T_loc-1 of the extended field (canonical
  // site x0 = 0 of the sub-domain starts one slice, 2 Fs sites of 72 reals, in)
  const long Fs_in = L.cstar ? Fs / 2 : Fs;  // C*: the uploaded links are the physical (undoubled) ones
  int rc = oq_gauge_upload(h, lat, U_ext_dev + (size_t)2 * Fs_in * 72, link_fmt, stream);
  if (rc) return rc;
  // the extended links for the clover build
  Geom ge = halo_ext_geom(L.g);
  rc = h->alloc(&L.uext, sizeof(double) * 2 * 4 * 18 * ge.Vh);
  if (rc) return rc;
  if (pack_links(ge, U_ext_dev, (double*)L.uext.p, nullptr, LINK_18, nullptr, nullptr, 0.0, nullptr, nullptr, s,
                 L.cstar ? L.g.L[1] / 2 : 0) != cudaSuccess)
    return OQ_ERR_CUDA;
  L.has_uext = true;
  return OQ_OK;
}

extern "C" int oq_axpby(oq_handle h, int lat, int prec, int subset, const double* a_host, const void* x_dev,
                        const double* b_host, void* y_dev, int nrhs, void* stream) {
  if (!valid(h, lat) || (prec != P_F64 && prec != P_F32) || subset < 0 || subset > 2 || !a_host || !b_host ||
      !x_dev || !y_dev || nrhs < 1 || nrhs > 64)
    return OQ_ERR_ARG;
  const long n = 24L * h->lats[lat].g.Vh * (subset == OQ_FULL ? 2 : 1);
  if (axpby(prec, a_host, x_dev, b_host, y_dev, n, nrhs, (cudaStream_t)stream) != cudaSuccess) return OQ_ERR_CUDA;
  h->launches += 1;
  return OQ_OK;
}
