// C ABI of the library: handle management, uploads, operator applications,
// reductions.  The solvers live in cgne.cu (and the later solver files).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"

using namespace oq;

namespace oq {
cudaError_t launch_hop(const HopLaunch& L, const HopArgs& a, cudaStream_t s) {
  if (L.nr != 1) {
    if (L.sys || (L.nr != 2 && L.nr != 4)) return cudaErrorInvalidValue;
    switch (L.prec) {
      case P_F32: return L.nr == 2 ? launch_hop_mr2_f32(L, a, s) : launch_hop_mr4_f32(L, a, s);
      case P_BF16: return L.nr == 2 ? launch_hop_mr2_bf16(L, a, s) : launch_hop_mr4_bf16(L, a, s);
      case P_F16: return L.nr == 2 ? launch_hop_mr2_f16(L, a, s) : launch_hop_mr4_f16(L, a, s);
      case P_DF64: return L.nr == 2 ? launch_hop_df2(L, a, s) : cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
  }
  switch (L.prec) {
    case P_F64: return launch_hop_f64(L, a, s);
    case P_F32: return launch_hop_f32(L, a, s);
    case P_BF16: return launch_hop_bf16(L, a, s);
    case P_F16: return launch_hop_f16(L, a, s);
    case P_DF64: return launch_hop_df64(L, a, s);
  }
  return cudaErrorInvalidValue;
}
}  // namespace oq

extern "C" const char* oq_error_string(int code) {
  switch (code) {
    case OQ_OK: return "ok";
    case OQ_ERR_ARG: return "invalid argument";
    case OQ_ERR_CUDA: return "CUDA error";
    case OQ_ERR_NOMEM: return "out of device memory";
    case OQ_ERR_TIMEOUT: return "bounded device wait timed out";
    case OQ_ERR_NONFINITE: return "non-finite value in a binary64 norm";
    case OQ_ERR_NOCONV: return "solver did not converge within nmx steps";
    case OQ_ERR_STATE: return "call out of order (gauge field or clover term missing)";
    default: return "unknown error";
  }
}

extern "C" int oq_create(oq_handle* out, const oq_lattice* lats, int nlat) {
  if (!out || !lats || nlat < 1 || nlat > 64) return OQ_ERR_ARG;
  *out = nullptr;
  for (int k = 0; k < nlat; ++k) {
    for (int mu = 0; mu < 4; ++mu)
      if (lats[k].L[mu] < 2 || (lats[k].L[mu] & 1)) return OQ_ERR_ARG;
    if (lats[k].bc_t != 1 && lats[k].bc_t != -1 && lats[k].bc_t != 0 && lats[k].bc_t != OQ_BC_HALO)
      return OQ_ERR_ARG;
    if (lats[k].cstar < 0 || lats[k].cstar > 3) return OQ_ERR_ARG;
    const double v = (double)lats[k].L[0] * lats[k].L[1] * lats[k].L[2] * lats[k].L[3] * (lats[k].cstar ? 2 : 1);
    if (v > (double)(1L << 29)) return OQ_ERR_ARG;  // Vh <= 2^28: 32-bit site offsets
  }
  oq_ctx* h = new (std::nothrow) oq_ctx();
  if (!h) return OQ_ERR_NOMEM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return OQ_ERR_CUDA;
  }
  h->lats.resize(nlat);
  for (int k = 0; k < nlat; ++k) {
    LatCtx& L = h->lats[k];
    for (int mu = 0; mu < 4; ++mu) L.g.L[mu] = lats[k].L[mu];
    // C* boundaries: the orbifold lattice doubled in x1, x2 / x3 wraps shifted
    L.cstar = lats[k].cstar;
    if (L.cstar) L.g.L[1] *= 2;
    L.g.cs_shift = (L.cstar >= 2 ? 4 : 0) | (L.cstar >= 3 ? 8 : 0);
    L.g.Lh3 = lats[k].L[3] / 2;
    L.g.Vh = (long)L.g.L[0] * L.g.L[1] * L.g.L[2] * L.g.L[3] / 2;
    L.halo_t = lats[k].bc_t == OQ_BC_HALO;
    L.g.bc_t = L.halo_t ? 1.0f : (float)lats[k].bc_t;  // a sub-domain's boundary factors come with its faces
    geom_init_div(L.g);
  }
  *out = h;
  return OQ_OK;
}

extern "C" int oq_destroy(oq_handle h) {
  if (!h) return OQ_ERR_ARG;
  cudaDeviceSynchronize();
  h->release();
  delete h;
  return OQ_OK;
}

extern "C" size_t oq_spinor_bytes(oq_handle h, int lat, int prec, int subset) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || prec < 0 || prec > 4 || subset < 0 || subset > 2) return 0;
  size_t half = (size_t)spinor_half_bytes(h->lats[lat].g.Vh, prec);
  return subset == OQ_FULL ? 2 * half : half;
}

// shared by oq_gauge_upload and oq_gauge_upload_qed (A_dev != nullptr)
static int gauge_upload(oq_handle h, int lat, const double* U_dev, const double* A_dev, double q, int link_fmt,
                        void* stream) {
  if (!h || !U_dev || lat < 0 || lat >= (int)h->lats.size()) return OQ_ERR_ARG;
  if (link_fmt != OQ_LINK_18 && link_fmt != OQ_LINK_12) return OQ_ERR_ARG;
  if (A_dev && (link_fmt != OQ_LINK_18 || !isfinite(q))) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  const bool sf = L.g.bc_t == 0.f;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n64 = sizeof(double) * 2 * 4 * 18 * L.g.Vh;
  const size_t n32 = sizeof(float) * 2 * 4 * (link_fmt == OQ_LINK_12 ? 12 : 18) * L.g.Vh;
  int rc = h->alloc(&L.u64, n64);
  if (rc) return rc;
  rc = h->alloc(&L.u32, n32);
  if (rc) return rc;
  // with 12-real links keep an 18-real binary32 copy as well: the tuner may
  // prefer it where the stencil is instruction-bound (many right-hand sides)
  if (link_fmt == OQ_LINK_12) {
    rc = h->alloc(&L.u32_18, sizeof(float) * 2 * 4 * 18 * L.g.Vh);
    if (rc) return rc;
  }
  // the clover's own copy of the links: unmasked (SF) or without the phase (QED)
  if (sf || A_dev) {
    rc = h->alloc(&L.uclov, n64);
    if (rc) return rc;
  }
  if (A_dev) {
    rc = h->alloc(&L.au1, sizeof(double) * 2 * 4 * L.g.Vh);
    if (rc) return rc;
  }
  L.link_fmt = link_fmt;
  void* u18 = link_fmt == OQ_LINK_12 ? L.u32_18.p : nullptr;
  if (pack_links(L.g, U_dev, (double*)L.u64.p, L.u32.p, link_fmt, u18, A_dev, q,
                 (sf || A_dev) ? (double*)L.uclov.p : nullptr, A_dev ? (double*)L.au1.p : nullptr,
                 s, L.cstar ? L.g.L[1] / 2 : 0) != cudaSuccess)
    return OQ_ERR_CUDA;
  if (sf && sf_mask_links(L.g, (double*)L.u64.p, L.u32.p, link_fmt, u18, s) != cudaSuccess) return OQ_ERR_CUDA;
  L.uclov_valid = sf || A_dev;
  L.has_u1 = A_dev != nullptr;
  L.qcharge = A_dev ? q : 0.0;
  L.has_gauge = true;
  L.has_clover = false;
  L.df_ready = false;
  L.has_uext = false;
  return OQ_OK;
}

extern "C" int oq_gauge_upload(oq_handle h, int lat, const double* U_dev, int link_fmt, void* stream) {
  return gauge_upload(h, lat, U_dev, nullptr, 0.0, link_fmt, stream);
}

extern "C" int oq_gauge_upload_qed(oq_handle h, int lat, const double* U_dev, const double* A_dev, double q,
                                   void* stream) {
  if (!A_dev) return OQ_ERR_ARG;
  return gauge_upload(h, lat, U_dev, A_dev, q, OQ_LINK_18, stream);
}

// Clover term of a sub-domain: built on the extended lattice (T_loc + 2
// slices) into scratch, then slice s + 1 of the extended parity 1 - q is
// slice s of parity q (one slice shifts the parity; the eo index shifts by
// the Fs = Vh / T_loc sites of a slice).  Blocks of A and A^{-1}: 36 (binary64)
// or 18 (binary32) chunks of 16 bytes per parity.
static int clover_build_halo(oq_handle h, int lat, double kappa, double csw, cudaStream_t s) {
  LatCtx& L = h->lats[lat];
  const Geom ge = halo_ext_geom(L.g);
  const long Fs = L.g.Vh / L.g.L[0];
  void *a64, *a32, *i64, *i32;
  const size_t n64 = sizeof(double) * 2 * 72 * ge.Vh, n32 = sizeof(float) * 2 * 72 * ge.Vh;
  int rc = h->workspace(lat, "clov_ext_a64", n64, &a64);
  if (!rc) rc = h->workspace(lat, "clov_ext_a32", n32, &a32);
  if (!rc) rc = h->workspace(lat, "clov_ext_i64", n64, &i64);
  if (!rc) rc = h->workspace(lat, "clov_ext_i32", n32, &i32);
  if (rc) return rc;
  if (build_clover(ge, (const double*)L.uext.p, nullptr, 0.0, 0, kappa, csw, 0.0, 1.0, (double*)a64, (float*)a32,
                   (double*)i64, (float*)i32, h->status_dev, s) != cudaSuccess)
    return OQ_ERR_CUDA;
  struct Part {
    void* dst;
    const void* src;
    int nch;
  } parts[] = {{L.a64.p, a64, 36}, {L.i64.p, i64, 36}, {L.a32.p, a32, 18}, {L.i32.p, i32, 18}};
  for (const Part& pt : parts)
    for (int q = 0; q < 2; ++q) {
      char* d = (char*)pt.dst + (size_t)q * pt.nch * L.g.Vh * 16;
      const char* src = (const char*)pt.src + ((size_t)(1 - q) * pt.nch * ge.Vh + Fs) * 16;
      if (cudaMemcpy2DAsync(d, (size_t)L.g.Vh * 16, src, (size_t)ge.Vh * 16, (size_t)L.g.Vh * 16, pt.nch,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return OQ_ERR_CUDA;
    }
  return OQ_OK;
}

extern "C" int oq_clover_build(oq_handle h, int lat, double kappa, double csw, void* stream) {
  oq_clover_params p;
  p.kappa = kappa;
  p.csw = csw;
  p.cF = 1.0;
  p.csw_qed = 0.0;
  p.qed_split = 0;
  return oq_clover_build_ex(h, lat, &p, stream);
}

extern "C" int oq_clover_build_ex(oq_handle h, int lat, const oq_clover_params* prm, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !prm) return OQ_ERR_ARG;
  const double kappa = prm->kappa, csw = prm->csw;
  if (!(kappa > 0.0) || !isfinite(csw) || !isfinite(prm->cF) || !isfinite(prm->csw_qed) ||
      (prm->qed_split != 0 && prm->qed_split != 1))
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_gauge) return OQ_ERR_STATE;
  if (prm->qed_split && !L.has_u1) return OQ_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n64 = sizeof(double) * 2 * 72 * L.g.Vh, n32 = sizeof(float) * 2 * 72 * L.g.Vh;
  int rc = h->alloc(&L.a64, n64);
  if (!rc) rc = h->alloc(&L.a32, n32);
  if (!rc) rc = h->alloc(&L.i64, n64);
  if (!rc) rc = h->alloc(&L.i32, n32);
  if (!rc) rc = h->ensure_scratch();
  if (rc) return rc;
  if (cudaMemsetAsync(h->status_dev, 0, sizeof(int), s) != cudaSuccess) return OQ_ERR_CUDA;
  if (L.halo_t) {
    // sub-domain: build on the lattice extended by one slice on each side
    // (every plaquette leaf of an interior site is there), keep the interior
    if (!L.has_uext) return OQ_ERR_STATE;
    if (prm->qed_split || prm->cF != 1.0) return OQ_ERR_ARG;
    rc = clover_build_halo(h, lat, kappa, csw, s);
    if (rc) return rc;
  } else {
    const double* links = L.uclov_valid ? (const double*)L.uclov.p : (const double*)L.u64.p;
    if (build_clover(L.g, links, L.has_u1 ? (const double*)L.au1.p : nullptr, L.qcharge, prm->qed_split, kappa, csw,
                     prm->csw_qed, prm->cF, (double*)L.a64.p, (float*)L.a32.p, (double*)L.i64.p, (float*)L.i32.p,
                     h->status_dev, s) != cudaSuccess)
      return OQ_ERR_CUDA;
  }
  int st = 0;
  if (cudaMemcpyAsync(&st, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return OQ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return OQ_ERR_CUDA;
  if (st) return OQ_ERR_NONFINITE;  // a singular clover block
  L.kappa = kappa;
  L.csw = csw;
  L.cF = prm->cF;
  L.csw_qed = prm->qed_split ? prm->csw_qed : 0.0;
  L.has_clover = true;
  L.df_ready = false;
  return OQ_OK;
}

static bool valid_lat(oq_handle h, int lat) { return h && lat >= 0 && lat < (int)h->lats.size(); }

extern "C" int oq_spinor_pack(oq_handle h, int lat, int prec, int subset, const double* canon_dev, void* packed_dev,
                              double scale, int nrhs, void* stream) {
  if (!valid_lat(h, lat) || !canon_dev || !packed_dev || prec < 0 || prec > 4 || subset < 0 || subset > 2 ||
      nrhs < 1 || !(scale != 0.0) || !isfinite(scale))
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  const long cstride = 2 * L.g.Vh * 12;  // double2 per canonical field
  const long ostride = (long)oq_spinor_bytes(h, lat, prec, subset);
  return pack_spinor(L.g, prec, subset, canon_dev, packed_dev, scale, nrhs, cstride, ostride, (cudaStream_t)stream) ==
                 cudaSuccess
             ? OQ_OK
             : OQ_ERR_CUDA;
}

extern "C" int oq_spinor_unpack(oq_handle h, int lat, int prec, int subset, const void* packed_dev, double* canon_dev,
                                double scale, int nrhs, void* stream) {
  if (!valid_lat(h, lat) || !canon_dev || !packed_dev || prec < 0 || prec > 4 || subset < 0 || subset > 2 ||
      nrhs < 1 || !(scale != 0.0) || !isfinite(scale))
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  const long cstride = 2 * L.g.Vh * 12;
  const long istride = (long)oq_spinor_bytes(h, lat, prec, subset);
  return unpack_spinor(L.g, prec, subset, packed_dev, canon_dev, scale, nrhs, istride, cstride,
                       (cudaStream_t)stream) == cudaSuccess
             ? OQ_OK
             : OQ_ERR_CUDA;
}

static bool overlap(const void* a, const void* b, size_t n) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + n && y < x + n;
}

extern "C" int oq_dw_apply(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs, int dagger,
                           void* stream) {
  if (!valid_lat(h, lat) || !in_dev || !out_dev || prec < 0 || prec > 4 || nrhs < 1) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // a sub-domain needs oq_dw_apply_halo
  const size_t full = oq_spinor_bytes(h, lat, prec, OQ_FULL);
  if (overlap(in_dev, out_dev, full * nrhs)) return OQ_ERR_ARG;
  if (prec == P_DF64) {
    const int rc = h->ensure_df(lat, (cudaStream_t)stream);
    if (rc) return rc;
  }
  HopArgs a = h->hop_args(lat, prec);
  a.in = in_dev;
  a.in2 = in_dev;
  a.out = out_dev;
  a.in_stride = a.in2_stride = a.out_stride = (long)full;
  a.half_bytes = (long)full / 2;
  a.nrhs = nrhs;
  HopLaunch hl = h->hop_launch(lat, prec, HOP_DW, dagger ? 1 : 0, EPI_NONE, nrhs);
  return h->run_hop(hl, a, (cudaStream_t)stream);
}

extern "C" int oq_dw_hat_apply(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs, int dagger,
                               void* stream) {
  if (!valid_lat(h, lat) || !in_dev || !out_dev || prec < 0 || prec > 4 || nrhs < 1) return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // a sub-domain needs oq_dhat_pass with faces
  const size_t half = oq_spinor_bytes(h, lat, prec, OQ_EVEN);
  if (overlap(in_dev, out_dev, half * nrhs)) return OQ_ERR_ARG;
  void* t = nullptr;
  int rc = h->workspace(lat, "dwhat_t", half * nrhs, &t);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == P_DF64) {
    rc = h->ensure_df(lat, s);
    if (rc) return rc;
  }
  HopArgs a = h->hop_args(lat, prec);
  a.nrhs = nrhs;
  a.in_stride = a.in2_stride = a.out_stride = (long)half;
  a.half_bytes = (long)half;
  // pass 1: t_o = A_oo^{-1} (-1/2 H_oe in_e)
  a.in = in_dev;
  a.out = t;
  a.p = 1;
  HopLaunch l1 = h->hop_launch(lat, prec, HOP_P1, dagger ? 1 : 0, EPI_NONE, nrhs);
  rc = h->run_hop(l1, a, s);
  if (rc) return rc;
  // pass 2: out_e = A_ee in_e + 1/2 H_eo t_o
  a.in = t;
  a.in2 = in_dev;
  a.out = out_dev;
  a.p = 0;
  HopLaunch l2 = h->hop_launch(lat, prec, HOP_P2, dagger ? 1 : 0, EPI_NONE, nrhs);
  return h->run_hop(l2, a, s);
}

static int reduce_common(oq_handle h, int lat, int prec, int subset, const void* x, const void* y, int nrhs,
                         double* out_host, void* stream) {
  if (!valid_lat(h, lat) || !x || !out_host || prec < 0 || prec > 3 || subset < 0 || subset > 2 || nrhs < 1)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  cudaStream_t s = (cudaStream_t)stream;
  const int nslot = (y ? 2 : 1) * nrhs;
  const int grid = reduce_grid(L.g.Vh);
  int rc = h->ensure_reduce(nslot * 2, grid);
  if (rc) return rc;
  const long half = (long)oq_spinor_bytes(h, lat, prec, OQ_EVEN);
  const long stride = (long)oq_spinor_bytes(h, lat, prec, subset);
  const int nparts = subset == OQ_FULL ? 2 : 1;
  for (int part = 0; part < nparts; ++part) {
    RedArgs ra = h->red_args(FIN_STORE, 0);
    ra.result = h->results + part * nslot;
    const char* xp = (const char*)x + part * half;
    cudaError_t e = y ? reduce_dot(prec, xp, (const char*)y + part * half, L.g.Vh, stride, nrhs, ra, s)
                      : reduce_norm2(prec, xp, L.g.Vh, stride, nrhs, ra, s);
    if (e != cudaSuccess) return OQ_ERR_CUDA;
  }
  if (cudaMemcpyAsync(h->results_host, h->results, sizeof(double) * nslot * nparts, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return OQ_ERR_CUDA;
  for (int k = 0; k < nslot; ++k) out_host[k] = h->results_host[k] + (nparts == 2 ? h->results_host[nslot + k] : 0.0);
  return OQ_OK;
}

extern "C" int oq_norm2(oq_handle h, int lat, int prec, int subset, const void* x_dev, int nrhs, double* out_host,
                        void* stream) {
  return reduce_common(h, lat, prec, subset, x_dev, nullptr, nrhs, out_host, stream);
}

extern "C" int oq_dot(oq_handle h, int lat, int prec, int subset, const void* x_dev, const void* y_dev, int nrhs,
                      double* out_host, void* stream) {
  if (!y_dev) return OQ_ERR_ARG;
  return reduce_common(h, lat, prec, subset, x_dev, y_dev, nrhs, out_host, stream);
}

extern "C" int oq_profile_start(oq_handle h) {
  if (!h) return OQ_ERR_ARG;
  for (auto& r : h->prof) {
    h->event_pool.push_back(r.e0);
    h->event_pool.push_back(r.e1);
  }
  h->prof.clear();
  // one live-count slot per launch (1 MiB: 262,144 launches; later launches
  // of the same profile are counted as all right-hand sides live)
  if (!h->prof_live) {
    const size_t n = (size_t)1 << 18;
    if (cudaMalloc(&h->prof_live, n * sizeof(unsigned)) != cudaSuccess) return OQ_ERR_NOMEM;
    h->prof_live_n = n;
  }
  h->prof_on = true;
  return OQ_OK;
}

extern "C" int oq_profile_stop(oq_handle h, oq_kernel_time* out, int max_entries, int* n_entries) {
  if (!h || !n_entries || (max_entries > 0 && !out)) return OQ_ERR_ARG;
  h->prof_on = false;
  if (cudaDeviceSynchronize() != cudaSuccess) return OQ_ERR_CUDA;
  std::vector<unsigned> live(h->prof.size() < h->prof_live_n ? h->prof.size() : h->prof_live_n);
  if (!live.empty() &&
      cudaMemcpy(live.data(), h->prof_live, live.size() * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return OQ_ERR_CUDA;
  std::vector<oq_kernel_time> agg;
  for (auto& r : h->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return OQ_ERR_CUDA;
    oq_kernel_time* t = nullptr;
    for (auto& a : agg)
      if (a.mode == r.mode && a.epi == r.epi && a.prec == r.prec && a.nr == r.nr && a.link_fmt == r.link_fmt &&
          a.dag == r.dag)
        t = &a;
    if (!t) {
      agg.push_back(oq_kernel_time{r.mode, r.epi, r.prec, 0, 0.0, 0.0, r.nr, r.link_fmt, r.dag, 0, 0.0, 0});
      t = &agg.back();
    }
    const unsigned nl = r.slot >= 0 ? live[r.slot] : (unsigned)r.nrhs;
    if (nl == 0) {
      // every right-hand side gated off: the launch moved no operand
      t->gated_launches += 1;
      t->gated_ms += ms;
    } else {
      t->launches += 1;
      t->total_ms += ms;
      t->bytes += r.fixed + r.per_rhs * nl;
      t->rhs_launches += nl;
    }
    h->event_pool.push_back(r.e0);
    h->event_pool.push_back(r.e1);
  }
  h->prof.clear();
  *n_entries = (int)agg.size();
  for (int k = 0; k < (int)agg.size() && k < max_entries; ++k) out[k] = agg[k];
  return OQ_OK;
}

extern "C" long long oq_kernel_launches(oq_handle h) { return h ? h->launches : -1; }

extern "C" int oq_set_option(oq_handle h, int key, int value) {
  if (!h) return OQ_ERR_ARG;
  switch (key) {
    case OQ_OPT_DF64_RESETS: h->df64_resets = value != 0; return OQ_OK;
    case OQ_OPT_TEST_TC_SKIP_MMA: h->hook_tc_skip_commit = value != 0; return OQ_OK;
    case OQ_OPT_NN_TENSOR_CORES: h->nn_tensor_cores = value != 0; return OQ_OK;
    case OQ_OPT_SAP_KERNEL:
      if (value < 0 || value > 2) return OQ_ERR_ARG;
      h->sap_kernel = value;
      return OQ_OK;
    case OQ_OPT_HISTORY: h->history = value != 0; return OQ_OK;
  }
  return OQ_ERR_ARG;
}

extern "C" int oq_solve_history(oq_handle h, int rhs, int kind, double* out_host, int cap, int* n) {
  if (!h || !n || cap < 0 || (cap > 0 && !out_host) || (kind != 0 && kind != 1)) return OQ_ERR_ARG;
  if (h->hist_nrhs == 0) return OQ_ERR_STATE;
  if (rhs < 0 || rhs >= h->hist_nrhs) return OQ_ERR_ARG;
  const std::vector<double>& v = kind == 0 ? h->hist_rec[rhs] : h->hist_reset[rhs];
  *n = kind == 0 ? (int)v.size() : (int)(v.size() / 2);
  const size_t m = v.size() < (size_t)cap ? v.size() : (size_t)cap;
  if (m) memcpy(out_host, v.data(), sizeof(double) * m);
  return OQ_OK;
}
